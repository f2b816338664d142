"""Pins of the NCI dispersion oracle and of the surrogate-network oracle.

NCI (Appendix):
  * the coupling term C and the placement of every symbol in the full relation
    (Eq. 2dmodesres) are pinned by the paper's own cubic (Eq. asym1): its
    constant and linear coefficients D2 and C2 are exactly the Taylor
    coefficients of xi0^2 D(dw') about the beam resonance in the v0 -> 1 limit
    (A2 and B2 drop higher-order coupling terms and agree to about 1e-3); this
    holds only with B time-centred (S_B3 carrying cos(w dt/2), whose expansion is
    the cubic's zeta0 + zeta1 dw');
  * the continuum limit (unit interpolation factors, exact derivatives, dt -> 0)
    against an independently written linearised cold relativistic beam (fluid
    momentum, continuity and Maxwell's equations): the relation's zeros are the
    fluid system's eigenfrequencies, which needs every group of C;
  * a planted sign error in any group of C, or the untimed S_B3, fails one of
    the two pins above;
  * vacuum factorisation, the sqrt(wp2) scaling of the resonance roots, the
    printed Sec. 4 statement (test_golden_paper_values.py), the qualitative
    (0,0) << (0,+-1) ordering and the smaller-time-step effect of Sec. 4;
  * the root finding: the number of roots equals the argument-principle count
    over the region's circle, and the growth equals the one from a brute-force
    scan of |F| (local minima refined by secant steps, no subdivision).

MLP: the FP64 backward pass equals central finite differences of the loss.
"""
import math

import numpy as np
import pytest

from oracle import mlp as omlp
from oracle import nci


def test_vacuum_limit_factorises():
    P = nci.NciParams(dt=0.08, dx1=0.2, dx2=0.2, gamma=50, wp2=0.0)
    k1, k2 = 7.0, 3.0
    m = nci.symbols(P, k1, k2, 0, 0)
    kb2 = math.sin(k2 * 0.1) / 0.1
    K = math.sqrt(k1 * k1 + kb2 * kb2)
    w_em = 2.0 / P.dt * math.asin(K * P.dt / 2.0)
    assert abs(nci.F_of(P, m, w_em)) < 1e-9 * abs(nci.F_of(P, m, w_em * 1.01))
    w_beam = k1 * P.v0
    assert abs(nci.F_of(P, m, w_beam)) < 1e-12
    assert nci.growth(P, k1, k2, 0, 0) == 0.0


def test_resonance_roots_scale_with_plasma_frequency():
    """The coupled roots next to w' = k1' v0 move away from it as sqrt(wp2)."""
    k1, k2, nu = 12.0, 8.0, 1
    sizes = []
    for wp2 in (1e-2, 1e-4):
        P = nci.NciParams(dt=0.08, dx1=0.2, dx2=0.2, gamma=50, wp2=wp2)
        m = nci.symbols(P, k1, k2, 0, nu)
        w_res = nci.resonance(P, m)
        sizes.append(max(abs(w - w_res) for w in nci.roots(P, k1, k2, 0, nu)))
    assert 0.07 < sizes[1] / sizes[0] < 0.14


# ---------------------------------------------------------------- the printed cubic
def _taylor_xi0sq_D(P, m, r=1e-2, n=64):
    """Taylor coefficients c0..c3 of xi0^2 D(dw') about the resonance (Cauchy integrals on
    a circle of radius r; D's pole at dw' = 0 only enters the coefficient of dw'^-1)."""
    wg = 2.0 * math.pi / P.dt
    kt = m.k1a - m.mu * wg
    xi0 = math.sin(0.5 * kt * P.dt) / (0.5 * P.dt)
    th = 2.0 * np.pi * np.arange(n) / n
    d = r * np.exp(1j * th)
    w = nci.resonance(P, m) + d
    D = nci.F_of(P, m, w) / d
    return [xi0 * xi0 * np.mean(D * np.exp(-1j * q * th)) / r ** q for q in range(4)]


def _cubic_cases():
    rng = np.random.default_rng(7)
    out = []
    for _ in range(12):
        gam = 1e5                                   # v0 -> 1 (the cubic sets v0 = 1 in k~1)
        b = rng.uniform(1.0, 5.0)                   # wp2 / gamma held finite
        P = nci.NciParams(dt=rng.uniform(0.02, 0.12), dx1=0.2, dx2=rng.uniform(0.1, 0.4), gamma=gam,
                          wp2=b * gam, order=int(rng.integers(1, 4)))
        k1 = rng.uniform(0.1, 0.9) * math.pi / P.dx1
        k2 = rng.uniform(0.1, 0.9) * math.pi / P.dx2
        out.append((P, k1, k2, 0, int(rng.integers(-1, 2))))
    return out


def _cubic_mismatch(P, k1, k2, mu, nu):
    m = nci.symbols(P, k1, k2, mu, nu)
    A2, B2, C2, D2 = nci.cubic_coeffs(P, m)
    c = _taylor_xi0sq_D(P, m)
    return (abs(c[0] / D2 - 1.0), abs(c[1] / C2 - 1.0), abs(c[2] / B2 - 1.0), abs(c[3] / A2 - 1.0))


@pytest.mark.parametrize("case", range(12))
def test_printed_cubic_is_the_expansion_of_the_full_relation(case):
    eD, eC, eB, eA = _cubic_mismatch(*_cubic_cases()[case])
    assert eD < 1e-6 and eC < 1e-6, (eD, eC)
    assert eB < 1e-2 and eA < 1e-2, (eB, eA)


# ---------------------------------------------------------------- the continuum limit
def _cold_beam_matrix(w, k1, k2, gamma, wp2):
    """Linearised cold relativistic beam (density n0 = 1, charge q = 1, mass m = 4 pi / wp2,
    velocity v0 along x1) with Maxwell's equations in Gaussian units, c = 1, for the
    perturbation (E1, E2, B3, u1, u2, n) ~ exp(i(k.x - w t)):
      Faraday        w B3 - k1 E2 + k2 E1 = 0
      Ampere         w E1 + k2 B3 + 4 pi i J1 = 0,  w E2 - k1 B3 + 4 pi i J2 = 0,
                     J1 = q (n0 u1 + v0 n), J2 = q n0 u2
      momentum       -i (w - k1 v0) gamma^3 m u1 = q E1,
                     -i (w - k1 v0) gamma m u2 = q (E2 - v0 B3)
      continuity     (w - k1 v0) n = n0 (k1 u1 + k2 u2)."""
    v0 = math.sqrt(1.0 - 1.0 / gamma ** 2)
    q, n0, ms = 1.0, 1.0, 4.0 * math.pi / wp2
    dw = w - k1 * v0
    M = np.zeros((6, 6), dtype=complex)
    M[0, [0, 1, 2]] = [k2, -k1, w]
    M[1, [0, 2, 3, 5]] = [w, k2, 4j * math.pi * q * n0, 4j * math.pi * q * v0]
    M[2, [1, 2, 4]] = [w, -k1, 4j * math.pi * q * n0]
    M[3, [0, 3]] = [-q, -1j * dw * gamma ** 3 * ms]
    M[4, [1, 2, 4]] = [-q, q * v0, -1j * dw * gamma * ms]
    M[5, [3, 4, 5]] = [n0 * k1, n0 * k2, -dw]
    return M


def _continuum_symbols(k1, k2):
    return nci.ModeSymbols(k1, k2, k1, k1, k2, 1.0, 1.0, 1.0, 1.0, 1.0, 0, 0)


def _continuum_check(G, k1, k2, gamma, wp2):
    """Largest |G| at the fluid eigenfrequencies, relative to |G| a little away from them,
    and the largest relative change of det(M)/G over random frequencies."""
    M0 = _cold_beam_matrix(0.0, k1, k2, gamma, wp2)
    A = _cold_beam_matrix(1.0, k1, k2, gamma, wp2) - M0          # M(w) = M0 + w A
    ev = np.linalg.eigvals(-np.linalg.solve(A, M0))
    worst = 0.0
    for w in ev:
        ref = abs(G(w + 1e-3 * max(1.0, abs(w))))
        worst = max(worst, abs(G(w)) / ref)
    rng = np.random.default_rng(3)
    ratios = []
    for _ in range(6):
        w = complex(rng.normal(0, 10), rng.normal(0, 10))
        ratios.append(np.linalg.det(_cold_beam_matrix(w, k1, k2, gamma, wp2)) / G(w))
    spread = max(abs(r / ratios[0] - 1.0) for r in ratios)
    return worst, spread


@pytest.mark.parametrize("k1,k2,gamma,wp2", [(3.0, 2.0, 5.0, 10.0), (7.0, 0.5, 50.0, 100.0), (1.0, 4.0, 2.0, 3.0),
                                             (12.0, 8.0, 20.0, 40.0)])
def test_continuum_limit_is_the_cold_beam_fluid(k1, k2, gamma, wp2):
    """With unit interpolation factors, exact derivatives and dt -> 0, [w] F equals the
    determinant of the fluid system up to a constant: the same six eigenfrequencies."""
    P = nci.NciParams(dt=1e-7, dx1=0.2, dx2=0.2, gamma=gamma, wp2=wp2)
    m = _continuum_symbols(k1, k2)
    worst, spread = _continuum_check(lambda w: nci.G_of(P, m, w), k1, k2, gamma, wp2)
    assert worst < 1e-8 and spread < 1e-8, (worst, spread)


# ---------------------------------------------------------------- planted mistakes
def _mutant_F(kind):
    """F_of with one deliberate error (test infrastructure: the pins must reject each)."""
    def F(P, m, w):
        v0 = P.v0
        wp = w + m.mu * 2.0 * math.pi / P.dt
        Delta = wp - m.k1a * v0
        wb = nci.wbracket(P, w)
        SB3 = m.SB3 if kind == "untimed_SB3" else nci.sb3_of(P, m, w)
        sgn = -1.0 if (m.mu % 2) else 1.0
        a, b = P.wp2 / P.gamma ** 3 * sgn, P.wp2 / P.gamma * sgn
        K2 = m.kE1 ** 2 + m.kE2 ** 2
        s = [1.0, 1.0, 1.0]
        if kind.startswith("flip_C"):
            s[int(kind[-1])] = -1.0
        first = Delta * Delta - a * m.Sj1 * m.SE1 * wp / wb
        second = (wb * wb - K2) * Delta - b * m.Sj2 * (m.SE2 * wb - SB3 * m.kE1 * v0)
        C = b / wb * (s[0] * m.Sj1 * m.SE1 * wp * m.kE2 ** 2 * (v0 * v0 - 1.0)
                      + s[1] * m.Sj2 * m.SE2 * m.kE2 ** 2 * Delta
                      + s[2] * m.Sj1 * m.kE2 * (m.SE2 * m.kE1 * m.k2 * v0 - SB3 * m.k2 * v0 * v0 * wb))
        return first * second + C * Delta
    return F


@pytest.mark.parametrize("kind", ["flip_C0", "flip_C1", "flip_C2", "untimed_SB3"])
def test_pins_reject_planted_mistakes(kind, monkeypatch):
    monkeypatch.setattr(nci, "F_of", _mutant_F(kind))
    cubic_bad = max(max(_cubic_mismatch(*c)[:2]) for c in _cubic_cases()[:4]) > 1e-3
    worst, spread = _continuum_check(lambda w: nci.G_of(nci.NciParams(dt=1e-7, gamma=5.0, wp2=10.0),
                                                        _continuum_symbols(3.0, 2.0), w), 3.0, 2.0, 5.0, 10.0)
    continuum_bad = worst > 1e-4 or spread > 1e-4
    assert cubic_bad or continuum_bad, kind


# ---------------------------------------------------------------- physics of Sec. 3 and Sec. 4
def test_zero_zero_modes_slower_than_pm1():
    P = nci.NciParams(dt=0.08, dx1=0.2, dx2=0.2, gamma=50, wp2=100.0)
    g00 = max(nci.growth_scan(P, 0, 0, 16, 16)[2].max(), 0.0)
    gpm = max(nci.growth_scan(P, 0, -1, 16, 16)[2].max(), nci.growth_scan(P, 0, 1, 16, 16)[2].max())
    assert gpm > 0.0
    assert g00 < 0.5 * gpm


def test_zero_zero_growth_falls_with_the_time_step():
    """Sec. 4: the (0,0) modes near the physical modes' harmonics are moved away, and their growth
    reduced, by reducing the time step.  Fastest (0,0) growth over a 32 x 32 (k1, k2) scan at the
    Table 1 plasma, dt = 0.06, 0.04, 0.02 (dx1 = dx2 = 0.2)."""
    g = [nci.growth_scan(nci.NciParams(dt=dt), 0, 0, 32, 32)[2].max() for dt in (0.06, 0.04, 0.02)]
    assert g[0] > g[1] > g[2] > 0.0
    assert g[2] < 0.5 * g[0]


# ---------------------------------------------------------------- root finding
def _circle_count(P, m, c, rho, n=1 << 14):
    """Zeros of [w] F inside |w - c| < rho by the argument principle on a dense circle."""
    th = 2.0 * np.pi * np.arange(n + 1) / n
    g = nci.G_of(P, m, c + rho * np.exp(1j * th))
    d = np.angle(g[1:] / g[:-1])
    assert np.max(np.abs(d)) < 0.5
    return int(round(np.sum(d) / (2.0 * math.pi)))


def _brute_roots(P, m, center, R, n=401):
    """Roots of F in the square |Re|, |Im| <= R around `center` found without subdivision or
    Newton iteration: every local minimum of |F| on grids of the square and of two smaller
    squares at its centre, refined by the secant method, kept if F vanishes there (relative
    to a point 1e-3 away); then the same inside a small square around each refined root, to
    split close pairs."""
    from numpy.lib.stride_tricks import sliding_window_view

    def scan(c0, half, npts):
        x = np.linspace(-half, half, npts)
        X, Y = np.meshgrid(x, x, indexing="ij")
        W = c0 + X + 1j * Y
        L = np.log(np.abs(nci.F_of(P, m, W)) + 1e-300)
        ismin = L[1:-1, 1:-1] <= sliding_window_view(L, (3, 3)).min(axis=(2, 3))
        h = x[1] - x[0]
        found = []
        for i, j in np.argwhere(ismin):
            a = complex(W[i + 1, j + 1])
            b = a + h * (0.3 + 0.2j)
            fa, fb = nci.F_of(P, m, a), nci.F_of(P, m, b)
            for _ in range(200):
                if fb == fa:
                    break
                c = b - fb * (b - a) / (fb - fa)
                a, fa, b, fb = b, fb, c, nci.F_of(P, m, c)
                if abs(b - a) < 1e-14 * max(1.0, abs(b)):
                    if abs(nci.F_of(P, m, b)) <= 1e-9 * abs(nci.F_of(P, m, b + 1e-3)):
                        found.append(b)
                    break
        return found
    out = []
    level1 = scan(center, R, n) + scan(center, 0.05 * R, 241) + scan(center, 0.002 * R, 241)
    for r in level1:
        for r2 in [r] + scan(r, 1e-3 * R, 61):
            if abs(r2.real - center.real) <= R and abs(r2.imag - center.imag) <= R and \
                    all(abs(r2 - u) > 1e-8 for u in out):
                out.append(r2)
    return out


# the fastest-growing (k1, k2) of a 16 x 16 scan of each alias at the Table 1 parameters, and
# modes of other aliases, stable and unstable
@pytest.mark.parametrize("mu,nu,k1,k2", [(0, 0, 6.381360077604267, 0.4908738521234052),
                                         (0, -1, 14.23534171157875, 10.30835089459151),
                                         (0, 1, 15.21708941582556, 9.326603190344699),
                                         (1, -1, 10.0, 8.0), (1, 0, 3.0, 5.0), (0, 0, 2.0, 12.0), (0, -1, 5.0, 3.0)])
def test_roots_are_complete_and_match_a_brute_force_scan(mu, nu, k1, k2):
    """The oracle's roots in the region are as many as the argument principle counts on its
    circle, and its growth rate equals the one from a brute-force scan of |F|."""
    P = nci.NciParams()
    m = nci.symbols(P, k1, k2, mu, nu)
    c = complex(nci.resonance(P, m))
    rho = nci.region_radius(P)
    rs = nci.roots(P, k1, k2, mu, nu)
    assert len(rs) == _circle_count(P, m, c, rho)
    for r in rs:
        assert abs(nci.G_of(P, m, r)) < 1e-9 * abs(nci.G_of(P, m, r + 1e-3)), r
    brute = [r for r in _brute_roots(P, m, c, rho) if abs(r - c) < rho]
    g_brute = max([r.imag for r in brute] + [0.0])
    assert abs(nci.growth(P, k1, k2, mu, nu) - g_brute) < 1e-9
    for r in brute:
        if r.imag > 1e-9:
            assert min(abs(r - u) for u in rs) < 1e-7, r


@pytest.mark.parametrize("width,depth", [(8, 2), (16, 3)])
def test_mlp_oracle_backprop_equals_finite_differences(width, depth):
    rng = np.random.default_rng(width)
    n_in, B = 6, 7
    npar = omlp.num_params(n_in, width, depth)
    p = rng.standard_normal(npar) * 0.3
    x = rng.standard_normal((B, n_in))
    t = rng.standard_normal(B)
    g, loss = omlp.gradients(p, x, t, n_in, width, depth, rnd=False)
    h = 1e-6
    for i in rng.choice(npar, 25, replace=False):
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        lp = np.mean((omlp.forward(pp, x, n_in, width, depth, rnd=False)[0] - t) ** 2)
        lm = np.mean((omlp.forward(pm, x, n_in, width, depth, rnd=False)[0] - t) ** 2)
        assert abs((lp - lm) / (2 * h) - g[i]) < 1e-7 * max(1.0, abs(g[i]))


def test_bf16_rounding_is_round_to_nearest_even():
    # 1 + 2^-8 lies halfway between two BF16 values: ties go to the even mantissa (1.0)
    assert omlp.bf16(np.array([1.0 + 2.0 ** -8]))[0] == 1.0
    assert omlp.bf16(np.array([1.0 + 3 * 2.0 ** -8]))[0] == 1.0 + 2.0 ** -6
    assert omlp.bf16(np.array([-3.0]))[0] == -3.0
