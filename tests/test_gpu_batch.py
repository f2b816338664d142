"""Batched launch (hyb_batch_*): several independent grids advanced by one
CUDA-graph launch per step give exactly the single-grid results, before and
after the strip-height autotuner, and match the oracle."""
import numpy as np
import pytest

from paper_1502_01376_gb300 import workloads as wl

from gpu_util import hyb_module, need_gpu, orc_grid, rel_err, to_dev, to_np, torch

pytestmark = pytest.mark.gpu

SIZES = [(512, 128, 32), (1024, 37, 32), (2048, 64, 32), (4096, 24, 32), (1024, 256, 32), (256, 16, 64)]


def _inputs(w, seed):
    E0, B0 = wl.band_limited_fields(w)
    rng = np.random.default_rng(seed)
    J0 = [rng.standard_normal(w.shape) * 1e-3 for _ in range(3)]
    return E0, B0, J0


def test_batch_equals_single_grids_and_oracle(orc):
    need_gpu()
    hyb = hyb_module()
    ws = [wl.Workload(f"b{i}", 2, n1, n2, dx1=0.2, dx2=0.2, dt=0.08, precision=p, filt_kc=0.5, filt_w=0.2, seed=40 + i)
          for i, (n1, n2, p) in enumerate(SIZES)]
    descs = [hyb.desc_from_workload(w) for w in ws]
    batch = hyb.Batch(descs)
    singles, bt, st, ins = [], [], [], []
    for i, w in enumerate(ws):
        dt = torch.float32 if w.precision == 32 else torch.float64
        E0, B0, J0 = _inputs(w, i)
        ins.append((E0, B0, J0))
        mk = lambda arrs: [to_dev(a, dt) for a in arrs]
        tb = (mk(E0), mk(B0), mk(J0))
        ts = (mk(E0), mk(B0), mk(J0))
        batch.bind(i, *tb)
        g = hyb.Grid(descs[i])
        g.bind(*ts)
        singles.append(g)
        bt.append(tb)
        st.append(ts)
    assert batch.launches_per_step >= 2
    nst = 6
    batch.advance(nst)
    for g in singles:
        g.advance(nst)
    torch.cuda.synchronize()
    def same_as_singles(what):
        for i in range(len(ws)):
            for a, b in zip(bt[i][0] + bt[i][1], st[i][0] + st[i][1]):
                assert torch.equal(a, b), (SIZES[i], what)

    same_as_singles("first steps")
    # oracle on two of them
    for i in (1, 5):
        w = ws[i]
        E0, B0, J0 = ins[i]
        rnd = (lambda a: a.astype(np.float32).astype(np.float64)) if w.precision == 32 else (lambda a: a)
        Eo, Bo, Jo = [rnd(a) for a in E0], [rnd(a) for a in B0], [rnd(a) for a in J0]
        orc.step(orc_grid(orc, w), Eo, Bo, Jo, nsteps=nst)
        tol = 1e-5 if w.precision == 32 else 1e-12
        for a, b in zip(bt[i][0] + bt[i][1], Eo + Bo):
            assert rel_err(to_np(a), b) < tol
    # autotune, then the batch still reproduces the single grids exactly
    batch.tune(2)
    for n1 in (512, 1024, 2048, 4096):
        assert 2 <= batch.rows_per_strip(n1) <= 64
    batch.advance(3)
    for g in singles:
        g.advance(3)
    torch.cuda.synchronize()
    same_as_singles("after tune")
    # heights set by hand (odd ones, and one row, clamped to two-row strips) give the same results
    for n1, h in ((512, 7), (1024, 5), (2048, 17), (4096, 1)):
        batch.set_rows_per_strip(n1, h)
        assert batch.rows_per_strip(n1) == h
    for n1, h in ((8192, 4), (1024, 0)):
        with pytest.raises(hyb.HybError):
            batch.set_rows_per_strip(n1, h)
    batch.advance(2)
    for g in singles:
        g.advance(2)
    torch.cuda.synchronize()
    same_as_singles("after set_rows_per_strip")
    batch.close()
