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
  * S'_B3 in the cubic coefficients is S_B3;
  * the current filter F(k1) and the j1 correction multiply S_j1
    (S_j1 <- S_j1 F corr) and the filter multiplies S_j2;
  * momentum-conserving interpolation, shape order l = 2 unless given;
  * the growth rate is max Im(w) over the roots, 0 if all are real.

The cubic asym1 (expansion about w' = k1' v0 with v0 -> 1) gives seeds; each
seed is refined by Newton's method on F(w) = D(w) (w' - k1' v0), whose only
extra root, at the resonance itself, is rejected.

Pins (tests/test_oracle_nci_mlp.py, tests/test_golden_paper_values.py): the
vacuum limit factorises into the hybrid EM modes and the beam resonance; the
resonance roots scale with sqrt(wp2); the (0,0) modes grow far more slowly
than the (0,+-1) modes; the value Sec. 4 prints: zero (0,0) growth at the
Table 1 parameters with the printed k1 modification, positive growth without
it; and the root finding: the growth from the cubic seeds and Newton steps
equals the one from a brute-force scan of |F| around the resonance.  The
growth rates of other individual modes live in the paper's absent figures:
the coupled relation's values there rest on these properties only, so they
are parity unpinned.
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


def wbracket(P: NciParams, w: complex) -> complex:
    return np.sin(0.5 * w * P.dt) / (0.5 * P.dt)


def F_of(P: NciParams, m: ModeSymbols, w: complex) -> complex:
    """D(w) (w' - k1' v0): the dispersion function without the resonance pole."""
    v0 = P.v0
    wg = 2.0 * math.pi / P.dt
    wp = w + m.mu * wg
    Delta = wp - m.k1a * v0
    wb = wbracket(P, w)
    sgn = -1.0 if (m.mu % 2) else 1.0
    a = P.wp2 / P.gamma ** 3 * sgn
    b = P.wp2 / P.gamma * sgn
    K2 = m.kE1 * m.kE1 + m.kE2 * m.kE2
    first = Delta * Delta - a * m.Sj1 * m.SE1 * wp / wb
    second = (wb * wb - K2) * Delta - b * m.Sj2 * (m.SE2 * wb - m.SB3 * m.kE1 * v0)
    C = b / wb * (m.Sj1 * m.SE1 * wp * m.kE2 * m.kE2 * (v0 * v0 - 1.0)
                  + m.Sj2 * m.SE2 * m.kE2 * m.kE2 * Delta
                  + m.Sj1 * m.kE2 * (m.SE2 * m.kE1 * m.k2 * v0 - m.SB3 * m.k2 * v0 * v0 * wb))
    return first * second + C * Delta


def cubic_coeffs(P: NciParams, m: ModeSymbols):
    """A2, B2, C2, D2 of Eq. asym1 (v0 -> 1 in k~1, S'_B3 read as S_B3)."""
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


def newton(P: NciParams, m: ModeSymbols, w0: complex, tol: float = 1e-13, maxit: int = 60):
    """Newton's method on F with a central complex difference for F'."""
    w = complex(w0)
    for _ in range(maxit):
        f = F_of(P, m, w)
        h = 1e-7 * max(1.0, abs(w))
        d = (F_of(P, m, w + h) - F_of(P, m, w - h)) / (2.0 * h)
        if d == 0:
            return None
        step = f / d
        w -= step
        if abs(step) <= tol * max(1.0, abs(w)):
            return w
    return None


def roots(P: NciParams, k1: float, k2: float, mu: int, nu1: int):
    """Refined roots of the full relation near the beam resonance."""
    m = symbols(P, k1, k2, mu, nu1)
    wg = 2.0 * math.pi / P.dt
    w_res = m.k1a * P.v0 - mu * wg
    A2, B2, C2, D2 = cubic_coeffs(P, m)
    seeds = []
    if A2 != 0.0:
        seeds += [w_res + complex(r) for r in np.roots([A2, B2, C2, D2])]
    r0 = (P.wp2 / P.gamma) ** (1.0 / 3.0) * 0.05
    seeds += [w_res + r0 * complex(math.cos(t), math.sin(t)) for t in (math.pi / 6, math.pi / 2, 5 * math.pi / 6)]
    out = []
    for s in seeds:
        w = newton(P, m, s)
        if w is None:
            continue
        if abs(w + mu * wg - m.k1a * P.v0) < 1e-9 * max(1.0, abs(w)):
            continue                       # the removed pole
        if all(abs(w - u) > 1e-9 * max(1.0, abs(w)) for u in out):
            out.append(w)
    return out


def growth(P: NciParams, k1: float, k2: float, mu: int, nu1: int) -> float:
    rs = roots(P, k1, k2, mu, nu1)
    g = max([r.imag for r in rs], default=0.0)
    return max(g, 0.0)


def growth_scan(P: NciParams, mu: int, nu1: int, n1: int = 64, n2: int = 64):
    """Growth over a (k1, k2) grid of the fundamental Brillouin zone (k1 > 0, k2 > 0)."""
    k1s = (np.arange(n1) + 0.5) * (math.pi / P.dx1) / n1
    k2s = (np.arange(n2) + 0.5) * (math.pi / P.dx2) / n2
    G = np.zeros((n1, n2))
    for i, k1 in enumerate(k1s):
        for j, k2 in enumerate(k2s):
            G[i, j] = growth(P, k1, k2, mu, nu1)
    return k1s, k2s, G
