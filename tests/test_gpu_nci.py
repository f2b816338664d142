"""Batched GPU root solver of the NCI dispersion relation (Appendix) against
the FP64 oracle: per sample and alias the same growth rate, and every GPU
root is a root of the oracle's dispersion function."""
import math

import numpy as np
import pytest

from gpu_util import hyb_module, need_gpu, torch

pytestmark = pytest.mark.gpu


def _samples(n, seed):
    rng = np.random.default_rng(seed)
    dx1 = 0.2
    dx2 = dx1 * rng.uniform(0.5, 2.0, n)
    cour = 2.0 / np.sqrt(np.pi ** 2 / dx1 ** 2 + 4.0 / dx2 ** 2)
    dt = np.minimum(dx1 * rng.uniform(0.1, 0.9, n), 0.98 * cour)
    gamma = rng.uniform(5.0, 100.0, n)
    kc = rng.uniform(0.3, 1.0, n)
    k1 = rng.uniform(0.02, 1.0, n) * math.pi / dx1
    k2 = rng.uniform(0.02, 1.0, n) * math.pi / dx2
    S = np.stack([dt, np.full(n, dx1), dx2, gamma, np.full(n, 100.0), kc, np.full(n, 0.2), k1, k2], axis=1)
    return np.ascontiguousarray(S)


def test_nci_growth_matches_oracle():
    need_gpu()
    hyb = hyb_module()
    from oracle import nci
    S = _samples(160, 3)
    aliases = ((0, -1), (0, 0), (0, 1))
    g, r = hyb.nci_growth(torch.from_numpy(S).cuda(), aliases=aliases, want_roots=True)
    g = g.cpu().numpy()
    r = r.cpu().numpy()
    agree = 0
    total = 0
    for i in range(S.shape[0]):
        dt, dx1, dx2, gam, wp2, kc, fw, k1, k2 = S[i]
        P = nci.NciParams(dt=dt, dx1=dx1, dx2=dx2, gamma=gam, wp2=wp2, order=2, filt_kc=kc, filt_w=fw)
        for a, (mu, nu) in enumerate(aliases):
            go = nci.growth(P, k1, k2, mu, nu)
            total += 1
            if abs(go - g[i, a]) <= 1e-7 * max(1.0, go):
                agree += 1
            if g[i, a] > 0:
                # the GPU root is a root of the oracle's dispersion function
                m = nci.symbols(P, k1, k2, mu, nu)
                w = complex(r[i, a])
                f = nci.F_of(P, m, w)
                h = 1e-7 * max(1.0, abs(w))
                d = (nci.F_of(P, m, w + h) - nci.F_of(P, m, w - h)) / (2 * h)
                assert abs(f / d) < 1e-8 * max(1.0, abs(w)), (i, a, w, f, d)
    assert agree >= 0.97 * total, (agree, total)


def test_nci_cold_limit_reduces_to_vacuum_and_resonance():
    """wp -> 0: the refined roots near the resonance are real (no growth)."""
    need_gpu()
    hyb = hyb_module()
    S = _samples(64, 5)
    S[:, 4] = 1e-12
    g = hyb.nci_growth(torch.from_numpy(S).cuda()).cpu().numpy()
    assert np.max(g) < 1e-5
