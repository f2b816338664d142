"""hyb_correct_current_noalloc: the allocation-free variant of the j1
correction, for callers whose device memory is owned by someone else (a
framework's pool) or who cannot afford cudaMalloc's synchronisation.  It must
give the same result as hyb_correct_current, also on a second call that finds
the first call's data still in the library's static working array."""
import numpy as np
import pytest

from gpu_util import hyb_module, need_gpu, rel_err, to_dev, to_np, torch

pytestmark = pytest.mark.gpu

TOL = {64: 1e-12, 32: 1e-5}


@pytest.mark.parametrize("n1,n2", [(4096, 600), (1024, 2100)])   # several row blocks of the static array,
@pytest.mark.parametrize("prec", [64, 32])                           # the last one ragged
def test_noalloc_correction_matches_regular_entry_point(prec, n1, n2):
    need_gpu()
    hyb = hyb_module()
    dt = torch.float64 if prec == 64 else torch.float32
    desc = hyb.make_desc(n1=n1, n2=n2, dx1=0.2, dx2=0.2, dt=0.1, precision=prec, path=1)
    g = hyb.Grid(desc)
    rng = np.random.default_rng(prec)
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):                  # two calls in a row on different data
        j1 = to_dev(rng.standard_normal((n2, n1)), dt)
        ref = j1.clone()
        J = [ref, torch.zeros_like(ref), torch.zeros_like(ref)]
        E = [torch.zeros_like(ref) for _ in range(3)]
        B = [torch.zeros_like(ref) for _ in range(3)]
        g.bind(E, B, J)
        g.correct_current()                # the existing entry point (grid-owned scratch)
        hyb.hyb_correct_current_noalloc(desc, int(j1.data_ptr()), stream)
        torch.cuda.synchronize()
        assert rel_err(to_np(j1), to_np(ref)) < TOL[prec], call
    g.close()
