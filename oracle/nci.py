"""FP64 numerical-Cerenkov-instability (NCI) dispersion analysis of the hybrid
solver, written from the Appendix (Eqs. 2dmodesres, coupling, asym1 and the
definitions that follow them).

TEST INFRASTRUCTURE ONLY: used by tests/ and the benchmark's CPU baseline; the
product's batched GPU root solver shares no code with it.

For a cold plasma drifting at v0 along x1 (Lorentz factor gamma, plasma
frequency^2 wp2 in units of the reference plasma frequency), and a grid mode
(k1, k2) with time alias mu and x1 alias nu1, the numerical dispersion
relation of the Appendix is

  D(w) = [ (w' - k1' v0)^2 - (wp2/gamma^3) (-1)^mu S_j1 S_E1 w' / [w] ]
       * [ [w]^2 - [k]E1 [k]B1 - [k]E2 [k]B2
           - (wp2/gamma) (-1)^mu S_j2 (S_E2 [w] - S_B3 [k]E1 v0) / (w' - k1' v0) ]
       + C = 0,
  C = (wp2/gamma) (-1)^mu / [w] * { S_j1 S_E1 w' [k]E2 [k]B2 (v0^2 - 1)
       + S_j2 S_E2 [k]E2 [k]B2 (w' - k1' v0)
       + S_j1 [k]E2 (S_E2 [k]B1 k2 v0 - S_B3 k2 v0^2 [w]) },

with w' = w + mu 2 pi/dt, k1' = k1 + nu1 2 pi/dx1, [w] = sin(w dt/2)/(dt/2),
and for the hybrid solver [k]E1 = [k]B1 = k1 (plus the Sec. 4 bump when
used), [k]E2 = [k]B2 = sin(k2 dx2/2)/(dx2/2).

Readings of garbled or silent points:
  * s_{l,i} = (sin(k'_i dx_i/2) / (k'_i dx_i/2))^(l+1) with k' the aliased
    wavenumber (the printed form lacks the denominator's k');
  * the repeated "S_E1" of the interpolation list is S_E3 (unused in 2D);
  * S_B3 of the full relation carries B's time centring: S_B3(w) = S'_B3
    cos(w dt/2), with S'_B3 the printed spatial factor; the cubic's
    zeta0 + zeta1 dw' is exactly the expansion of cos(w dt/2) about the
    resonance, and only with this factor are the cubic's D2 and C2 the Taylor
    coefficients of xi0^2 D (pinned);
  * the current filter F(k1) and the j1 correction multiply S_j1
    (S_j1 <- S_j1 F corr) and the filter multiplies S_j2;
  * momentum-conserving interpolation, shape order l = 2 unless given;
  * the growth rate of an alias is max Im(w) over the roots in the disk
    |w - w_res| < (wp2/gamma)^(1/3) around the beam resonance w_res (the scale
    at which the cubic's cubic and constant terms balance; the fastest NCI
    roots lie within a tenth of it), 0 if none grows.

Root finding: the zeros of [w] F(w) (entire: the same zeros as F without its
poles) in the disk, by recursive subdivision of an enclosing rectangle with
the argument principle counting the zeros of each piece, and Newton's method
inside pieces that hold one zero.  The count over the whole region makes the
set complete by construction.

Pins (tests/test_oracle_nci_mlp.py, tests/test_golden_paper_values.py): the
printed cubic's D2 and C2 equal the Taylor coefficients of xi0^2 D at v0 -> 1
(this fixes the coupling term C and every symbol's place); the continuum limit
equals the eigenfrequencies of an independently written linearised cold
relativistic beam; planted sign errors in each group of C fail these; the
vacuum limit factorises; the resonance roots scale with sqrt(wp2); the (0,0)
modes grow far more slowly than the (0,+-1) modes and more slowly at smaller
dt (Sec. 4); the value Sec. 4 prints: zero (0,0) growth at the Table 1
parameters with the printed k1 modification, positive growth without it; the
root set's completeness (argument principle on the region's circle) and its
growth against a brute-force scan of |F|.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class NciParams:
    dt: float = 0.08
    dx1: float = 0.2
    dx2: float = 0.2
    gamma: float = 50.0
    wp2: float = 100.0            # n / n_p (Table 1)
    order: int = 2                # particle shape order l
    filt_kc: float = 0.0          # fraction of pi/dx1; 0 = no filter
    filt_w: float = 0.2
    correct_j1: bool = True
    kmod_l: float = 0.0           # Sec. 4 bump, fractions of k_g1
    kmod_u: float = 0.0
    kmod_max: float = 0.0
    solver: str = "hybrid"        # "hybrid" | "yee"

    @property
    def v0(self) -> float:
        return math.sqrt(1.0 - 1.0 / (self.gamma * self.gamma))


def sinc(x: float) -> float:
    return 1.0 if x == 0.0 else math.sin(x) / x


def filter_factor(P: NciParams, k1: float) -> float:
    if not (0.0 < P.filt_kc < 1.0):
        return 1.0
    kn = math.pi / P.dx1
    k = abs(k1)
    kc, w = P.filt_kc * kn, P.filt_w * kn
    if k <= kc - 0.5 * w:
        return 1.0
    if k >= kc + 0.5 * w:
        return 0.0
    c = math.cos(0.5 * math.pi * (k - kc + 0.5 * w) / w)
    return c * c


def kop1(P: NciParams, k1: float) -> float:
    """[k]E1 = [k]B1 of the solver at the fundamental k1."""
    if P.solver == "yee":
        return math.sin(0.5 * k1 * P.dx1) / (0.5 * P.dx1)
    k = k1
    if P.kmod_max != 0.0:
        kg = 2.0 * math.pi / P.dx1
        kl, ku = P.kmod_l * kg, P.kmod_u * kg
        km = 0.5 * (kl + ku)
        a = abs(k1)
        if kl <= a <= ku:
            c = math.cos(0.5 * math.pi * (a - km) / (kl - km))
            k = k1 + math.copysign(P.kmod_max * kg * c * c, k1)
    return k


@dataclass
class ModeSymbols:
    k1: float
    k2: float
    k1a: float        # aliased k1' = k1 + nu1 k_g1
    kE1: float        # [k]E1 = [k]B1
    kE2: float        # [k]E2 = [k]B2
    SE1: float
    SE2: float
    SB3: float
    Sj1: float
    Sj2: float
    mu: int
    nu1: int


def symbols(P: NciParams, k1: float, k2: float, mu: int, nu1: int) -> ModeSymbols:
    kg1 = 2.0 * math.pi / P.dx1
    k1a = k1 + nu1 * kg1
    l = P.order
    s1 = sinc(0.5 * k1a * P.dx1)
    s2 = sinc(0.5 * k2 * P.dx2)
    sl1, sl2 = s1 ** (l + 1), s2 ** (l + 1)
    sm1, sm2 = s1 ** l, s2 ** l                      # order l - 1
    sgn = -1.0 if (nu1 % 2) else 1.0
    SE1 = sl1 * sl2 * sgn
    SE2 = sl1 * sl2
    SB3 = sl1 * sl2 * sgn
    F = filter_factor(P, k1)
    corr = sinc(0.5 * k1 * P.dx1) * k1 / kop1(P, k1) if (P.correct_j1 and k1 != 0.0 and P.solver != "yee") else 1.0
    Sj1 = sm1 * sl2 * sgn * F * corr
    Sj2 = sl1 * sm2 * F
    kE1 = kop1(P, k1)
    kE2 = math.sin(0.5 * k2 * P.dx2) / (0.5 * P.dx2)
    return ModeSymbols(k1, k2, k1a, kE1, kE2, SE1, SE2, SB3, Sj1, Sj2, mu, nu1)


def wbracket(P: NciParams, w):
    """[w] = sin(w dt/2)/(dt/2), the leapfrog's time-difference symbol (numpy, complex)."""
    return np.sin(0.5 * w * P.dt) / (0.5 * P.dt)


def sb3_of(P: NciParams, m: ModeSymbols, w):
    """S_B3 of the full relation: the spatial interpolation factor times cos(w dt/2),
    the time centring of B (half a step away from E) at the particles' time level;
    the printed cubic's zeta0 + zeta1 dw' is exactly the expansion of this factor."""
    return m.SB3 * np.cos(0.5 * w * P.dt)


def F_of(P: NciParams, m: ModeSymbols, w):
    """D(w) (w' - k1' v0): the dispersion function (Eq. 2dmodesres with the coupling
    term) times the resonance factor, which removes D's pole at w' = k1' v0."""
    v0 = P.v0
    wg = 2.0 * math.pi / P.dt
    wp = w + m.mu * wg
    Delta = wp - m.k1a * v0
    wb = wbracket(P, w)
    SB3 = sb3_of(P, m, w)
    sgn = -1.0 if (m.mu % 2) else 1.0
    a = P.wp2 / P.gamma ** 3 * sgn
    b = P.wp2 / P.gamma * sgn
    K2 = m.kE1 * m.kE1 + m.kE2 * m.kE2
    first = Delta * Delta - a * m.Sj1 * m.SE1 * wp / wb
    second = (wb * wb - K2) * Delta - b * m.Sj2 * (m.SE2 * wb - SB3 * m.kE1 * v0)
    C = b / wb * (m.Sj1 * m.SE1 * wp * m.kE2 * m.kE2 * (v0 * v0 - 1.0)
                  + m.Sj2 * m.SE2 * m.kE2 * m.kE2 * Delta
                  + m.Sj1 * m.kE2 * (m.SE2 * m.kE1 * m.k2 * v0 - SB3 * m.k2 * v0 * v0 * wb))
    return first * second + C * Delta


def G_of(P: NciParams, m: ModeSymbols, w):
    """[w] F(w): the same zeros as F, without F's poles where [w] = 0 (an entire function
    of w, so the argument principle counts its zeros)."""
    return wbracket(P, w) * F_of(P, m, w)


def cubic_coeffs(P: NciParams, m: ModeSymbols):
    """A2, B2, C2, D2 of Eq. asym1 (v0 -> 1 in k~1; S'_B3 is the spatial factor m.SB3,
    zeta0 and zeta1 the expansion of B's time centring cos(w dt/2))."""
    wg = 2.0 * math.pi / P.dt
    kt = m.k1 + m.nu1 * (2.0 * math.pi / P.dx1) - m.mu * wg
    h = 0.5 * P.dt
    xi0 = math.sin(kt * h) / h
    xi1 = math.cos(kt * h)
    ze0 = math.cos(kt * h)
    ze1 = -math.sin(kt * h) * h
    sgn = -1.0 if (m.mu % 2) else 1.0
    b = P.wp2 / P.gamma * sgn
    kE1, kB1, kE2, kB2 = m.kE1, m.kE1, m.kE2, m.kE2
    A2 = 2.0 * xi0 ** 3 * xi1
    B2 = xi0 ** 2 * (xi0 ** 2 - kE1 * kB1 - kE2 * kB2 - b * m.Sj2 * (m.SE2 * xi1 - ze1 * m.SB3 * kE1))
    C2 = b * (xi0 ** 2 * m.Sj2 * (ze0 * m.SB3 * kE1 - m.SE2 * xi0) - xi1 * m.Sj1 * kE2 * m.k2 * m.SE2 * kB1
              + xi0 * kE2 * (m.Sj2 * m.SE2 * kB2 - m.Sj1 * m.k2 * ze1 * m.SB3 * xi0))
    D2 = b * xi0 * kE2 * m.k2 * m.Sj1 * (m.SE2 * kB1 - ze0 * m.SB3 * xi0)
    return A2, B2, C2, D2


def region_radius(P: NciParams) -> float:
    """Radius of the disk around the beam resonance whose roots define the growth:
    (wp2/gamma)^(1/3), the scale at which the cubic's leading and constant terms
    balance (the NCI roots lie well inside it)."""
    return (P.wp2 / P.gamma) ** (1.0 / 3.0)


class _OnBoundary(Exception):
    pass


def _winding(f, x0, x1, y0, y1):
    """Number of zeros of f inside the rectangle (argument principle): the change of
    arg f around the boundary, sampled until no step exceeds 0.5 rad."""
    n = 32
    while n <= 1 << 14:
        t = np.arange(n) / n
        z = np.concatenate([x0 + (x1 - x0) * t + 1j * y0, x1 + 1j * (y0 + (y1 - y0) * t),
                            x1 - (x1 - x0) * t + 1j * y1, x0 + 1j * (y1 - (y1 - y0) * t), [x0 + 1j * y0]])
        g = f(z)
        if np.all(g != 0):
            d = np.angle(g[1:] / g[:-1])
            if np.max(np.abs(d)) <= 0.5:
                return int(round(np.sum(d) / (2.0 * math.pi)))
        n *= 4
    raise _OnBoundary()


def _newton(f, w, tol=1e-14, maxit=100):
    """Newton's method with a central-difference derivative."""
    for _ in range(maxit):
        fw = f(w)
        h = 1e-7 * max(1.0, abs(w))
        d = (f(w + h) - f(w - h)) / (2.0 * h)
        if d == 0 or not np.isfinite(d):
            return None
        step = fw / d
        w = w - step
        if not np.isfinite(w):
            return None
        if abs(step) <= tol * max(1.0, abs(w)):
            return complex(w)
    return None


# split fractions of the subdivision, away from 1/2 so that the real axis (where the real
# roots lie) and the resonance do not fall on a split line; the next pair is tried when a
# zero lies too close to a split line for its count to be resolved
_SPLITS = ((0.4871, 0.5317), (0.4413, 0.5689), (0.5593, 0.4231), (0.3917, 0.6143))


def _zeros_in_rect(f, x0, x1, y0, y1, hmin, N, out):
    if N == 0:
        return
    if N == 1:
        w = _newton(f, complex(x0 + _SPLITS[0][0] * (x1 - x0), y0 + _SPLITS[0][1] * (y1 - y0)))
        if w is not None and x0 <= w.real <= x1 and y0 <= w.imag <= y1:
            out.append(w)
            return
    if max(x1 - x0, y1 - y0) < hmin:            # a cluster below resolution: its centre, N times
        out.extend([complex(0.5 * (x0 + x1), 0.5 * (y0 + y1))] * N)
        return
    for fx, fy in _SPLITS:
        xm, ym = x0 + fx * (x1 - x0), y0 + fy * (y1 - y0)
        kids = [(x0, xm, y0, ym), (xm, x1, y0, ym), (x0, xm, ym, y1), (xm, x1, ym, y1)]
        try:
            ns = [_winding(f, *k) for k in kids]
        except _OnBoundary:
            continue
        if sum(ns) != N:
            raise RuntimeError("argument principle: inconsistent zero counts")
        for k, nk in zip(kids, ns):
            _zeros_in_rect(f, *k, hmin, nk, out)
        return
    raise RuntimeError("argument principle: zeros on every split line tried")


def zeros_in_disk(f, c: complex, rho: float):
    """All zeros of the entire function f with |w - c| < rho: a rectangle enclosing the
    disk is split into four until each piece holds one zero (counted by the argument
    principle), which Newton's method then locates inside it."""
    if not rho > 0.0:
        return []
    for e in (1.0, 1.013, 1.029):
        x0, x1 = c.real - e * rho, c.real + 1.0007 * e * rho
        y0, y1 = c.imag - 1.0003 * e * rho, c.imag + 1.0011 * e * rho
        try:
            N = _winding(f, x0, x1, y0, y1)
        except _OnBoundary:
            continue
        out = []
        # resolution: zeros closer than this are returned as one point, N times (below it,
        # rounding in w and in f decides the phase of f)
        hmin = max(1e-12 * rho, 1e-9 * max(1.0, abs(c)))
        _zeros_in_rect(f, x0, x1, y0, y1, hmin, N, out)
        return [w for w in out if abs(w - c) < rho]
    raise RuntimeError("argument principle: zeros on the enclosing rectangle")


def resonance(P: NciParams, m: ModeSymbols) -> float:
    """w at the beam resonance w' = k1' v0."""
    return m.k1a * P.v0 - m.mu * 2.0 * math.pi / P.dt


def roots(P: NciParams, k1: float, k2: float, mu: int, nu1: int, rho: float | None = None):
    """All roots of the full relation within rho (default region_radius) of the beam resonance."""
    m = symbols(P, k1, k2, mu, nu1)
    r = region_radius(P) if rho is None else rho
    return zeros_in_disk(lambda w: G_of(P, m, w), complex(resonance(P, m)), r)


def growth(P: NciParams, k1: float, k2: float, mu: int, nu1: int) -> float:
    """NCI growth rate of alias (mu, nu1) at (k1, k2): the largest Im w over the roots in the
    region around the beam resonance, 0 if none grows."""
    rs = roots(P, k1, k2, mu, nu1)
    return max([r.imag for r in rs] + [0.0])


def growth_scan(P: NciParams, mu: int, nu1: int, n1: int = 64, n2: int = 64):
    """Growth over a (k1, k2) grid of the fundamental Brillouin zone (k1 > 0, k2 > 0)."""
    k1s = (np.arange(n1) + 0.5) * (math.pi / P.dx1) / n1
    k2s = (np.arange(n2) + 0.5) * (math.pi / P.dx2) / n2
    G = np.zeros((n1, n2))
    for i, k1 in enumerate(k1s):
        for j, k2 in enumerate(k2s):
            G[i, j] = growth(P, k1, k2, mu, nu1)
    return k1s, k2s, G
