"""Edge cases of the boundary: the smallest and largest row lengths, the
fewest rows, one-row-per-strip fused grids, ragged strips, the DFT-GEMM's
fewest rows and ragged tiles, k1-resident fields on the smallest grids, an
empty particle set (deposit and PIC step), a batch of one grid, and the sizes
the ABI rejects."""
import numpy as np
import pytest

from paper_1502_01376_gb300 import workloads as wl

from gpu_util import hyb_module, need_gpu, orc_grid, rel_err, to_dev, to_np, torch

pytestmark = pytest.mark.gpu

TOL = {64: 1e-12, 32: 1e-5}


def _run(orc, hyb, w, path, nst=3, seed=5):
    dt = torch.float64 if w.precision == 64 else torch.float32
    g = hyb.Grid(hyb.desc_from_workload(w, path=path))
    E0, B0 = wl.band_limited_fields(w)
    rng = np.random.default_rng(seed)
    J0 = [rng.standard_normal(w.shape) * 1e-3 for _ in range(3)]
    rnd = (lambda a: a) if w.precision == 64 else (lambda a: a.astype(np.float32).astype(np.float64))
    E = [to_dev(a, dt) for a in E0]
    B = [to_dev(a, dt) for a in B0]
    J = [to_dev(a, dt) for a in J0]
    g.bind(E, B, J)
    g.advance(nst)
    g.check()
    Eo, Bo, Jo = [rnd(a) for a in E0], [rnd(a) for a in B0], [rnd(a) for a in J0]
    orc.step(orc_grid(orc, w), Eo, Bo, Jo, nsteps=nst)
    errs = [rel_err(to_np(a), b) for a, b in zip(E + B, Eo + Bo)]
    g.close()
    return errs


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("n1,n2", [(8, 2), (8, 3), (16, 2), (8192, 3)])
def test_three_pass_extreme_row_lengths(orc, prec, n1, n2):
    need_gpu()
    hyb = hyb_module()
    w = wl.Workload("e", 2, n1, n2, dx1=0.2, dx2=0.25, dt=0.05, precision=prec, filt_kc=0.5, filt_w=0.2, seed=9)
    errs = _run(orc, hyb, w, path=1)
    assert max(errs) < TOL[prec], errs


def test_three_pass_3d_1024_rows_fp32(orc):
    """The 3D benchmark's row length (the register-resident 1024-point row FFT) with a ragged row count."""
    need_gpu()
    hyb = hyb_module()
    w = wl.Workload("e31", 3, 1024, 6, 5, dx1=0.2, dx2=0.2, dx3=0.2, dt=0.08, precision=32, filt_kc=0.5, filt_w=0.2,
                    seed=14)
    errs = _run(orc, hyb, w, path=1)
    assert max(errs) < TOL[32], errs


@pytest.mark.parametrize("prec", [64, 32])
def test_three_pass_3d_two_planes(orc, prec):
    need_gpu()
    hyb = hyb_module()
    w = wl.Workload("e3", 3, 32, 2, 2, dx1=0.2, dx2=0.25, dx3=0.3, dt=0.05, precision=prec, filt_kc=0.6, filt_w=0.2,
                    seed=10)
    errs = _run(orc, hyb, w, path=1)
    assert max(errs) < TOL[prec], errs


@pytest.mark.parametrize("n1,n2", [(4096, 4), (4096, 5), (512, 4), (2048, 7)])
def test_fused_fewest_rows(orc, n1, n2):
    """Strips of two or three rows (n2 / 2 strips), the smallest grids the fused path takes."""
    need_gpu()
    hyb = hyb_module()
    w = wl.Workload("ef", 2, n1, n2, dx1=0.2, dx2=0.2, dt=0.1, precision=32, filt_kc=0.5, filt_w=0.2, seed=11)
    errs = _run(orc, hyb, w, path=2)
    assert max(errs) < TOL[32], errs


@pytest.mark.parametrize("path", [3, 4])
@pytest.mark.parametrize("n1,n2", [(16, 2), (1024, 2), (32, 129)])
def test_dftgemm_fewest_rows_and_ragged_tiles(orc, n1, n2, path):
    """The tensor-core DFT-GEMM with the fewest rows a grid has (one 128-row tile mostly empty), the
    longest rows it takes (several passes over the output columns and K chunks) and a row count
    one past a tile boundary."""
    need_gpu()
    hyb = hyb_module()
    w = wl.Workload("ed", 2, n1, n2, dx1=0.2, dx2=0.25, dt=0.05, precision=32, filt_kc=0.5, filt_w=0.2, seed=19)
    errs = _run(orc, hyb, w, path=path)
    assert max(errs) < 6e-5, errs


@pytest.mark.parametrize("n1,n2", [(8, 2), (4096, 4)])
def test_resident_fewest_rows(orc, n1, n2):
    """k1-resident fields on the smallest grids: the step equals the oracle's."""
    need_gpu()
    hyb = hyb_module()
    w = wl.Workload("er", 2, n1, n2, dx1=0.2, dx2=0.25, dt=0.05, precision=64, filt_kc=0.5, filt_w=0.2, seed=23)
    g = hyb.Grid(hyb.desc_from_workload(w))
    E0, B0 = wl.band_limited_fields(w)
    rng = np.random.default_rng(24)
    J0 = [rng.standard_normal(w.shape) * 1e-3 for _ in range(3)]
    T = [to_dev(a, torch.float64) for a in list(E0) + list(B0) + J0]
    g.bind(T[0:3], T[3:6], T[6:9])
    g.set_resident(True)
    g.advance(0)                                 # no step: nothing imported or written
    g.advance(3)
    g.check()
    Eo, Bo, Jo = [a.copy() for a in E0], [a.copy() for a in B0], [a.copy() for a in J0]
    orc.step(orc_grid(orc, w), Eo, Bo, Jo, nsteps=3)
    errs = [rel_err(to_np(a), b) for a, b in zip(T[:6], Eo + Bo)]
    assert max(errs) < TOL[64], errs
    g.close()


def test_pic_step_without_particles(orc):
    """A PIC step with no particles (both modes): the fields advance as hyb_advance with zero current."""
    need_gpu()
    hyb = hyb_module()
    w = wl.Workload("ep", 2, 64, 8, dx1=0.2, dx2=0.2, dt=0.08, precision=64, seed=29)
    E0, B0 = wl.band_limited_fields(w)
    for resident in (False, True):
        g = hyb.Grid(hyb.desc_from_workload(w))
        T = [to_dev(a, torch.float64) for a in list(E0) + list(B0)] + [torch.zeros(w.shape, dtype=torch.float64,
                                                                                     device="cuda") for _ in range(3)]
        g.bind(T[0:3], T[3:6], T[6:9])
        if resident:
            g.set_resident(True)
        pic = hyb.Pic(g)
        e_i = torch.zeros((0, 2), dtype=torch.int32, device="cuda")
        e_f = torch.zeros((0, 2), dtype=torch.float64, device="cuda")
        e_1 = torch.zeros(0, dtype=torch.float64, device="cuda")
        e_3 = torch.zeros((0, 3), dtype=torch.float64, device="cuda")
        pic.step(e_i, e_f, e_3, e_1, e_1, e_f, e_1, order=2, nsteps=2)
        g.check()
        Eo, Bo = [a.copy() for a in E0], [a.copy() for a in B0]
        orc.step(orc_grid(orc, w), Eo, Bo, [np.zeros(w.shape) for _ in range(3)], nsteps=2)
        errs = [rel_err(to_np(a), b) for a, b in zip(T[:6], Eo + Bo)]
        assert max(errs) < TOL[64], (resident, errs)
        pic.close()
        g.close()


def test_deposit_without_particles_zeroes_j(orc):
    need_gpu()
    hyb = hyb_module()
    w = wl.Workload("ed", 2, 64, 8, dx1=0.2, dx2=0.2, dt=0.05, precision=64, seed=12)
    g = hyb.Grid(hyb.desc_from_workload(w, path=1))
    E = [torch.zeros(w.shape, dtype=torch.float64, device="cuda") for _ in range(3)]
    B = [torch.zeros(w.shape, dtype=torch.float64, device="cuda") for _ in range(3)]
    J = [torch.ones(w.shape, dtype=torch.float64, device="cuda") for _ in range(3)]
    g.bind(E, B, J)
    empty_i = torch.zeros((0, 2), dtype=torch.int32, device="cuda")
    empty_f = torch.zeros((0, 2), dtype=torch.float64, device="cuda")
    empty_v = torch.zeros((0, 3), dtype=torch.float64, device="cuda")
    empty_q = torch.zeros(0, dtype=torch.float64, device="cuda")
    g.deposit(empty_i, empty_f, empty_f, empty_v, empty_q, 1)
    g.check()
    torch.cuda.synchronize()
    assert all(float(j.abs().max()) == 0.0 for j in J)
    g.close()


def test_batch_of_one_grid_equals_single(orc):
    need_gpu()
    hyb = hyb_module()
    w = wl.Workload("eb", 2, 1024, 16, dx1=0.2, dx2=0.2, dt=0.1, precision=32, filt_kc=0.5, filt_w=0.2, seed=13)
    E0, B0 = wl.band_limited_fields(w)
    mk = lambda arrs: [to_dev(a, torch.float32) for a in arrs]
    Jz = [np.zeros(w.shape) for _ in range(3)]
    tb, ts = (mk(E0), mk(B0), mk(Jz)), (mk(E0), mk(B0), mk(Jz))
    b = hyb.Batch([hyb.desc_from_workload(w)])
    b.bind(0, *tb)
    g = hyb.Grid(hyb.desc_from_workload(w))
    g.bind(*ts)
    b.advance(2)
    g.advance(2)
    torch.cuda.synchronize()
    for x, y in zip(tb[0] + tb[1], ts[0] + ts[1]):
        assert torch.equal(x, y)
    b.close()
    g.close()


def test_sizes_the_abi_rejects():
    need_gpu()
    hyb = hyb_module()
    for bad in (dict(n1=4, n2=8), dict(n1=16384, n2=4), dict(n1=96, n2=8), dict(n1=64, n2=1)):
        w = wl.Workload("x", 2, bad["n1"], bad["n2"], dx1=0.2, dx2=0.2, dt=0.01, precision=64, seed=1)
        with pytest.raises(Exception):
            hyb.Grid(hyb.desc_from_workload(w))
