"""hyb_correct_current_noalloc: the allocation-free variant of the j1
correction, for callers whose device memory is owned by someone else (a
framework's pool) or who cannot afford cudaMalloc's synchronisation.  It must
give the same result as hyb_correct_current, also on a second call that finds
the first call's data still in the library's static working array, and the
same result as the oracle's correction."""
import numpy as np
import pytest

from gpu_util import hyb_module, need_gpu, rel_err, to_dev, to_np, torch

pytestmark = pytest.mark.gpu

TOL = {64: 1e-12, 32: 1e-5}


def _pair(hyb, desc, shape, prec, rng, stream):
    """One call of each entry point on the same random j1; returns (noalloc, regular)."""
    dt = torch.float64 if prec == 64 else torch.float32
    g = hyb.Grid(desc)
    try:
        j1 = to_dev(rng.standard_normal(shape), dt)
        ref = j1.clone()
        J = [ref, torch.zeros_like(ref), torch.zeros_like(ref)]
        E = [torch.zeros_like(ref) for _ in range(3)]
        B = [torch.zeros_like(ref) for _ in range(3)]
        g.bind(E, B, J)
        g.correct_current()                # the existing entry point (grid-owned scratch)
        hyb.hyb_correct_current_noalloc(desc, int(j1.data_ptr()), stream)
        torch.cuda.synchronize()
        return to_np(j1), to_np(ref)
    finally:
        g.close()


@pytest.mark.parametrize("n1,n2", [(4096, 600), (1024, 2100)])   # several row blocks of the static array,
@pytest.mark.parametrize("prec", [64, 32])                           # the last one ragged
def test_noalloc_correction_matches_regular_entry_point(prec, n1, n2):
    need_gpu()
    hyb = hyb_module()
    desc = hyb.make_desc(n1=n1, n2=n2, dx1=0.2, dx2=0.2, dt=0.1, precision=prec, path=1)
    rng = np.random.default_rng(prec)
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):                  # two calls in a row on different data
        a, b = _pair(hyb, desc, (n2, n1), prec, rng, stream)
        assert rel_err(a, b) < TOL[prec], call


# 3D rows, the Yee-recovery symbol and the Sec. 4 bump change the correction factor; the
# calls alternate between them so each one finds another call's tables in the array
CASES = [
    dict(dims=3, n1=256, n2=12, n3=10, dx1=0.2, dx2=0.2, dx3=0.2, dt=0.05),
    dict(dims=2, n1=512, n2=40, dx1=0.2, dx2=0.2, dt=0.05, yee_mode=True),
    dict(dims=2, n1=256, n2=33, dx1=0.2, dx2=0.2, dt=0.05, kmod_l=0.15, kmod_u=0.26, kmod_max=0.01),
    dict(dims=3, n1=64, n2=5, n3=7, dx1=0.1, dx2=0.2, dx3=0.3, dt=0.02, kmod_l=0.1, kmod_u=0.3, kmod_max=0.05),
]


@pytest.mark.parametrize("prec", [64, 32])
def test_noalloc_correction_mode_switches_and_oracle(prec, orc):
    need_gpu()
    hyb = hyb_module()
    rng = np.random.default_rng(100 + prec)
    stream = torch.cuda.current_stream().cuda_stream
    for rep in range(2):
        for c in CASES:
            desc = hyb.make_desc(precision=prec, path=1, **c)
            shape = (c["n3"], c["n2"], c["n1"]) if c["dims"] == 3 else (c["n2"], c["n1"])
            dt = torch.float64 if prec == 64 else torch.float32
            j1 = to_dev(rng.standard_normal(shape), dt)
            # the oracle's correction of the same (rounded) input
            g = orc.grid(**{k: v for k, v in c.items()})
            J = [to_np(j1).copy(), np.zeros(shape), np.zeros(shape)]
            orc.process_current(g, J, True, False)
            hyb.hyb_correct_current_noalloc(desc, int(j1.data_ptr()), stream)
            torch.cuda.synchronize()
            assert rel_err(to_np(j1), J[0]) < TOL[prec], (rep, c)
            a, b = _pair(hyb, desc, shape, prec, rng, stream)
            assert rel_err(a, b) < TOL[prec], (rep, c)
