"""Batched GPU root solver of the NCI dispersion relation (Appendix) against
the FP64 oracle, for shape orders 1, 2 and 3, with and without the Sec. 4 k1
modification: per sample and alias the same set of roots in the region about
the beam resonance (the same count, every oracle root found by the GPU), and
so the same growth rate."""
import math

import numpy as np
import pytest

from gpu_util import hyb_module, need_gpu, torch

pytestmark = pytest.mark.gpu

ALIASES = ((0, -1), (0, 0), (0, 1))


def _samples(n, seed, bump_every=0):
    rng = np.random.default_rng(seed)
    dx1 = 0.2
    dx2 = dx1 * rng.uniform(0.5, 2.0, n)
    cour = 2.0 / np.sqrt(np.pi ** 2 / dx1 ** 2 + 4.0 / dx2 ** 2)
    dt = np.minimum(dx1 * rng.uniform(0.1, 0.9, n), 0.98 * cour)
    gamma = rng.uniform(5.0, 100.0, n)
    kc = rng.uniform(0.3, 1.0, n)
    k1 = rng.uniform(0.01, 1.0, n) * math.pi / dx1
    k2 = rng.uniform(0.01, 1.0, n) * math.pi / dx2
    kl, ku, km = np.zeros(n), np.zeros(n), np.zeros(n)
    if bump_every:
        sel = np.arange(n) % bump_every == 0
        kl[sel], ku[sel], km[sel] = 0.15, 0.26, 0.01      # the printed Sec. 4 modification
        k1[sel] = rng.uniform(0.1, 0.3, sel.sum()) * 2 * math.pi / dx1
    S = np.stack([dt, np.full(n, dx1), dx2, gamma, np.full(n, 100.0), kc, np.full(n, 0.2), k1, k2, kl, ku, km],
                 axis=1)
    return np.ascontiguousarray(S)


@pytest.mark.parametrize("order", [1, 2, 3])
def test_nci_roots_match_oracle(order):
    need_gpu()
    hyb = hyb_module()
    from oracle import nci
    S = _samples(90, 10 + order, bump_every=5)
    R, C, G, err = hyb.nci_roots(torch.from_numpy(S).cuda(), aliases=ALIASES, order=order)
    assert err == 0
    R, C, G = R.cpu().numpy(), C.cpu().numpy(), G.cpu().numpy()
    g_only = hyb.nci_growth(torch.from_numpy(S).cuda(), aliases=ALIASES, order=order).cpu().numpy()
    assert np.array_equal(g_only, G)          # both entry points run the same solve
    ambiguous = 0
    total = 0
    for i in range(S.shape[0]):
        dt, dx1, dx2, gam, wp2, kc, fw, k1, k2, kl, ku, km = S[i]
        P = nci.NciParams(dt=dt, dx1=dx1, dx2=dx2, gamma=gam, wp2=wp2, order=order, filt_kc=kc, filt_w=fw,
                          kmod_l=kl, kmod_u=ku, kmod_max=km)
        rho = nci.region_radius(P)
        for a, (mu, nu) in enumerate(ALIASES):
            total += 1
            m = nci.symbols(P, k1, k2, mu, nu)
            c = nci.resonance(P, m)
            ro = nci.roots(P, k1, k2, mu, nu)
            rg = list(R[i, a, :C[i, a]])
            # a root within 1e-6 rho of the region's circle may be counted on either side
            if any(abs(abs(w - c) - rho) < 1e-6 * rho for w in ro + rg):
                ambiguous += 1
                continue
            assert len(rg) == len(ro), (i, a, ro, rg)
            for w in ro:                              # every oracle root is found by the GPU
                assert min(abs(w - u) for u in rg) < 1e-7 * max(1.0, abs(w)), (i, a, w, rg)
            go = max([w.imag for w in ro] + [0.0])
            assert abs(G[i, a] - go) < 1e-8 * max(1.0, abs(c)), (i, a, G[i, a], go)
    assert ambiguous <= 0.01 * total, (ambiguous, total)


def test_nci_cold_limit_has_no_growth():
    """wp -> 0: the roots near the resonance are real (no growth)."""
    need_gpu()
    hyb = hyb_module()
    S = _samples(64, 5)
    S[:, 4] = 1e-12
    g = hyb.nci_growth(torch.from_numpy(S).cuda()).cpu().numpy()
    assert np.max(g) < 1e-5


def test_nci_printed_bump_statement_on_gpu():
    """Sec. 4 at the Table 1 parameters (dt = 0.08, dx = 0.2, gamma = 50, n/n_p = 100,
    quadratic shapes): the (0, 0) modes grow without the printed k1 modification and
    not with it (64 x 64 scan of the fundamental zone, as the oracle's golden test)."""
    need_gpu()
    hyb = hyb_module()
    n = 64
    k1 = (np.arange(n) + 0.5) * (math.pi / 0.2) / n
    k2 = (np.arange(n) + 0.5) * (math.pi / 0.2) / n
    K1, K2 = np.meshgrid(k1, k2, indexing="ij")
    base = np.stack([np.full(n * n, 0.08), np.full(n * n, 0.2), np.full(n * n, 0.2), np.full(n * n, 50.0),
                     np.full(n * n, 100.0), np.zeros(n * n), np.full(n * n, 0.2), K1.ravel(), K2.ravel(),
                     np.zeros(n * n), np.zeros(n * n), np.zeros(n * n)], axis=1)
    bump = base.copy()
    bump[:, 9:12] = (0.15, 0.26, 0.01)
    g0 = hyb.nci_growth(torch.from_numpy(np.ascontiguousarray(base)).cuda(), aliases=((0, 0),)).cpu().numpy()
    g1 = hyb.nci_growth(torch.from_numpy(np.ascontiguousarray(bump)).cuda(), aliases=((0, 0),)).cpu().numpy()
    assert g0.max() > 1e-2
    assert g1.max() < 1e-10
