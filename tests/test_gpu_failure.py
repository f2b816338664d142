"""Failure detection without a GPU fault: the bounded device waits of the fused
advance (the halo-exchange flag and the row-staging mbarrier) and of the
single-launch batched step (the barrier between a role's CTAs) give up on a
condition nothing satisfies and report HYB_ETIMEOUT to the host; the context
stays usable (a parity-checked advance runs right after)."""
import numpy as np
import pytest

from paper_1502_01376_gb300 import workloads as wl

from gpu_util import hyb_module, need_gpu, orc_grid, rel_err, to_dev, to_np, torch

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("which", [0, 1, 2])
def test_bounded_wait_gives_up_and_reports(orc, which):
    need_gpu()
    hyb = hyb_module()
    st = hyb.hyb_wait_selftest(which, 0.2)
    assert st == hyb.HYB_ETIMEOUT, st
    assert "gave up" in hyb.lib().hyb_last_error().decode()
    # the context still works: a fused advance matches the oracle
    w = wl.Workload("t", 2, 1024, 12, dx1=0.2, dx2=0.2, dt=0.1, precision=32, filt_kc=0.5, filt_w=0.2, seed=4)
    g = hyb.Grid(hyb.desc_from_workload(w, path=2))
    E0, B0 = wl.band_limited_fields(w)
    f32 = lambda a: a.astype(np.float32).astype(np.float64)
    E = [to_dev(a, torch.float32) for a in E0]
    B = [to_dev(a, torch.float32) for a in B0]
    J = [torch.zeros(w.shape, device="cuda", dtype=torch.float32) for _ in range(3)]
    g.bind(E, B, J)
    g.advance(3)
    g.check()
    Eo, Bo = [f32(a) for a in E0], [f32(a) for a in B0]
    orc.step(orc_grid(orc, w), Eo, Bo, [np.zeros(w.shape) for _ in range(3)], nsteps=3)
    assert max(rel_err(to_np(a), b) for a, b in zip(E + B, Eo + Bo)) < 1e-5
    g.close()


def test_selftest_rejects_bad_arguments():
    need_gpu()
    hyb = hyb_module()
    assert hyb.hyb_wait_selftest(3, 0.1) == hyb.HYB_EINVAL
    assert hyb.hyb_wait_selftest(0, 0.0) == hyb.HYB_EINVAL
    assert hyb.hyb_wait_selftest(0, 60.0) == hyb.HYB_EINVAL
