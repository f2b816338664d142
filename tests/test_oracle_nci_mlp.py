"""Pins of the NCI dispersion oracle and of the surrogate-network oracle.

NCI (Appendix): with the plasma frequency -> 0 the relation factorises into
the vacuum hybrid modes [w]^2 = k1^2 + [k]2^2 and the beam resonance; the
resonance roots move away as sqrt(wp2); the (0,0) modes grow far more slowly
than the fastest (0,+-1) modes (Sec. 3, Sec. 6).  Quantitative growth rates of
the paper live in absent figures, and the printed cubic (Eq. asym1) disagrees
with the full relation in character for some modes (garbled coefficients), so
the growth values of the coupled relation are pinned by the paper only through
the Sec. 4 statement; the cubic is used only to seed Newton's method on the
full relation, and the root finding itself is pinned by a brute-force scan of
|F| over the complex plane around the resonance.

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
    """The resonance roots of the full relation move away from w' = k1' v0 as
    sqrt(wp2) (two-stream-like coupling of the beam mode)."""
    k1, k2, nu = 12.0, 8.0, 1
    sizes = []
    for wp2 in (1e-2, 1e-4):
        P = nci.NciParams(dt=0.08, dx1=0.2, dx2=0.2, gamma=50, wp2=wp2)
        m = nci.symbols(P, k1, k2, 0, nu)
        w_res = m.k1a * P.v0
        near = [abs(w - w_res) for w in nci.roots(P, k1, k2, 0, nu) if abs(w - w_res) < 1.0]
        sizes.append(max(near))
    assert 0.07 < sizes[1] / sizes[0] < 0.14


def test_zero_zero_modes_slower_than_pm1():
    P = nci.NciParams(dt=0.08, dx1=0.2, dx2=0.2, gamma=50, wp2=100.0)
    g00 = max(nci.growth_scan(P, 0, 0, 16, 16)[2].max(), 0.0)
    gpm = max(nci.growth_scan(P, 0, -1, 16, 16)[2].max(), nci.growth_scan(P, 0, 1, 16, 16)[2].max())
    assert gpm > 0.0
    assert g00 < 0.5 * gpm


def test_zero_zero_growth_falls_with_the_time_step():
    """Sec. 4: the (0,0) modes near the physical modes' harmonics are moved away, and their growth
    reduced, by reducing the time step.  Fastest (0,0) growth over a 64 x 64 (k1, k2) scan at the
    Table 1 plasma, dt = 0.06, 0.04, 0.02 (dx1 = dx2 = 0.2)."""
    g = [nci.growth_scan(nci.NciParams(dt=dt), 0, 0, 64, 64)[2].max() for dt in (0.06, 0.04, 0.02)]
    assert g[0] > g[1] > g[2] > 0.0
    assert g[2] < 0.5 * g[0]


def _brute_roots(P, m, center, boxes=((2.0, 401), (0.06, 241))):
    """Roots of F in square boxes around `center` found without the oracle's seeds or Newton
    iteration: every local minimum of |F| on a grid of the box, refined by the secant method,
    kept if F vanishes there (relative to a point 1e-3 away) and it is not the resonance point."""
    from numpy.lib.stride_tricks import sliding_window_view
    out = []
    for R, n in boxes:
        x = np.linspace(-R, R, n)
        X, Y = np.meshgrid(x, x, indexing="ij")
        W = center + X + 1j * Y
        L = np.log(np.abs(nci.F_of(P, m, W)) + 1e-300)
        ismin = L[1:-1, 1:-1] <= sliding_window_view(L, (3, 3)).min(axis=(2, 3))
        h = x[1] - x[0]
        for i, j in np.argwhere(ismin):
            a = complex(W[i + 1, j + 1])
            b = a + h * (0.3 + 0.2j)
            fa, fb = nci.F_of(P, m, a), nci.F_of(P, m, b)
            r = None
            for _ in range(200):
                if fb == fa:
                    break
                c = b - fb * (b - a) / (fb - fa)
                a, fa, b, fb = b, fb, c, nci.F_of(P, m, c)
                if abs(b - a) < 1e-14 * max(1.0, abs(b)):
                    r = b
                    break
            if r is None or abs(r - center) > R or abs(r - center) < 1e-9:
                continue
            if abs(nci.F_of(P, m, r)) > 1e-9 * abs(nci.F_of(P, m, r + 1e-3)):
                continue
            if all(abs(r - u) > 1e-8 for u in out):
                out.append(r)
    return out


# the fastest-growing (k1, k2) of a 16 x 16 scan of each alias at the Table 1 parameters, and
# modes of other aliases, stable and unstable
@pytest.mark.parametrize("mu,nu,k1,k2", [(0, 0, 6.381360077604267, 0.4908738521234052),
                                         (0, -1, 14.23534171157875, 10.30835089459151),
                                         (0, 1, 15.21708941582556, 9.326603190344699),
                                         (1, -1, 10.0, 8.0), (1, 0, 3.0, 5.0), (0, 0, 2.0, 12.0), (0, -1, 5.0, 3.0)])
def test_growth_equals_brute_force_root_scan(mu, nu, k1, k2):
    """The growth rate (max Im w over the roots near the beam resonance) from the oracle's cubic
    seeds and Newton steps equals the one from a brute-force scan of |F| over the complex plane
    around the resonance, and every growing root the scan finds is among the oracle's roots."""
    P = nci.NciParams()
    m = nci.symbols(P, k1, k2, mu, nu)
    w_res = m.k1a * P.v0 - mu * 2.0 * math.pi / P.dt
    brute = _brute_roots(P, m, w_res)
    oracle_roots = nci.roots(P, k1, k2, mu, nu)
    g_brute = max([r.imag for r in brute] + [0.0])
    assert abs(nci.growth(P, k1, k2, mu, nu) - g_brute) < 1e-9
    for r in brute:
        if r.imag > 1e-9:
            assert min(abs(r - u) for u in oracle_roots) < 1e-7, r


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
