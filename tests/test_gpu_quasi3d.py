"""Quasi-3D azimuthal-mode path (Sec. 5) against the FP64 oracle: complex
fields of modes m = 0, 1, 2 (and 3) on a conducting cylinder, FP64 and FP32,
with the j_z correction and the k1 filter; also inside a batch."""
import numpy as np
import pytest

from oracle import quasi3d as q

from gpu_util import hyb_module, need_gpu, rel_err, torch

pytestmark = pytest.mark.gpu

TOL = {64: 1e-12, 32: 1e-5}


def _fields(nr, nz, seed, scale=1.0):
    rng = np.random.default_rng(seed)
    return [(rng.standard_normal((nr, nz)) + 1j * rng.standard_normal((nr, nz))) * scale for _ in range(3)]


def _run_pair(hyb, m, prec, nz=128, nr=37, nsteps=6, seed=0, filt=True):
    dz, dr = 0.2, 0.15
    dt = 0.9 * 2 / np.sqrt(np.pi ** 2 / dz ** 2 + (4 * m * m + 6) / dr ** 2)
    g = q.QGrid(nz=nz, nr=nr, dz=dz, dr=dr, dt=dt, m=m, filt_kc=0.5 if filt else 0.0, filt_w=0.2)
    E, B, J = _fields(nr, nz, seed), _fields(nr, nz, seed + 1), _fields(nr, nz, seed + 2, 1e-2)
    cdt = torch.complex128 if prec == 64 else torch.complex64
    rnd = (lambda a: a) if prec == 64 else (lambda a: a.astype(np.complex64).astype(np.complex128))
    Eo, Bo, Jo = [rnd(a) for a in E], [rnd(a) for a in B], [rnd(a) for a in J]
    desc = hyb.make_desc(dims=20, n1=nz, n2=nr, dx1=dz, dx2=dr, dt=dt, precision=prec, filt_kc=0.5 if filt else 0.0,
                         filt_w=0.2, azimuthal_m=m)
    grid = hyb.Grid(desc)
    Et = [torch.from_numpy(a).to("cuda", cdt) for a in E]
    Bt = [torch.from_numpy(a).to("cuda", cdt) for a in B]
    Jt = [torch.from_numpy(a).to("cuda", cdt) for a in J]
    grid.bind(Et, Bt, Jt)
    return g, grid, (Eo, Bo, Jo), (Et, Bt, Jt), desc


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("m", [0, 1, 2, 3])
def test_quasi3d_matches_oracle(m, prec):
    need_gpu()
    hyb = hyb_module()
    g, grid, (Eo, Bo, Jo), (Et, Bt, Jt), _ = _run_pair(hyb, m, prec, seed=10 * m + prec)
    q.step(g, Eo, Bo, Jo, 6)
    grid.advance(6)
    for a, b in zip(Et + Bt, Eo + Bo):
        assert rel_err(a.cpu().numpy().view(np.float64 if prec == 64 else np.float32).astype(np.float64),
                       b.view(np.float64)) < TOL[prec]
    grid.close()


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("nz,nr", [(16, 5), (2048, 2), (2048, 9), (4096, 3)])
def test_quasi3d_row_lengths(nz, nr, prec):
    """Short rows (many rows per block), the batched workload's z length (one row per block, next
    block prefetched) and rows longer than the prefetch holds (direct loads)."""
    need_gpu()
    hyb = hyb_module()
    g, grid, (Eo, Bo, Jo), (Et, Bt, Jt), _ = _run_pair(hyb, 1, prec, nz=nz, nr=nr, nsteps=3, seed=nz + nr)
    q.step(g, Eo, Bo, Jo, 3)
    grid.advance(3)
    for a, b in zip(Et + Bt, Eo + Bo):
        assert rel_err(a.cpu().numpy().view(np.float64 if prec == 64 else np.float32).astype(np.float64),
                       b.view(np.float64)) < TOL[prec]
    grid.close()


def test_quasi3d_in_batch_with_2d_grids():
    need_gpu()
    hyb = hyb_module()
    from paper_1502_01376_gb300 import workloads as wl
    g, grid, (Eo, Bo, Jo), (Et, Bt, Jt), qdesc = _run_pair(hyb, 1, 32, nz=256, nr=20, seed=77)
    w = wl.Workload("b", 2, 1024, 16, dx1=0.2, dx2=0.2, dt=0.08, precision=32, filt_kc=0.5, filt_w=0.2, seed=5)
    E0, B0 = wl.band_limited_fields(w)
    mk = lambda arrs: [torch.from_numpy(a.astype(np.float32)).cuda() for a in arrs]
    b = hyb.Batch([hyb.desc_from_workload(w), qdesc])
    E2, B2, J2 = mk(E0), mk(B0), [torch.zeros(w.shape, device="cuda") for _ in range(3)]
    b.bind(0, E2, B2, J2)
    Eq = [t.clone() for t in Et]
    Bq = [t.clone() for t in Bt]
    b.bind(1, Eq, Bq, Jt)
    b.advance(4)
    grid.advance(4)
    torch.cuda.synchronize()
    for a, c in zip(Eq + Bq, Et + Bt):
        assert torch.equal(a, c)
    b.close()
    grid.close()


def test_quasi3d_modes_advanced_together_in_a_batch():
    """Modes with nz = 2048 and a common radial grid run as one set of launches in a batch (their
    arrays in one z transform, all modes in one leapfrog launch): each mode's result equals its
    own grid's, and one mode against the oracle."""
    need_gpu()
    hyb = hyb_module()
    from paper_1502_01376_gb300 import workloads as wl
    runs = [_run_pair(hyb, m, 32, nz=2048, nr=24, seed=90 + m) for m in (0, 1, 2)]
    w = wl.Workload("b", 2, 1024, 16, dx1=0.2, dx2=0.2, dt=0.08, precision=32, filt_kc=0.5, filt_w=0.2, seed=5)
    E0, B0 = wl.band_limited_fields(w)
    mk = lambda arrs: [torch.from_numpy(a.astype(np.float32)).cuda() for a in arrs]
    b = hyb.Batch([r[4] for r in runs] + [hyb.desc_from_workload(w)])
    b.single_launch = False                    # the graph of launches (the single launch: test_gpu_batch_single.py)
    assert b.launches_per_step == 3 + 2        # modes: z transform, leapfrog, inverse; the 2D grid: halo, fused
    copies = []
    for i, (_, grid, _, (Et, Bt, Jt), _) in enumerate(runs):
        Eq, Bq = [t.clone() for t in Et], [t.clone() for t in Bt]
        b.bind(i, Eq, Bq, Jt)
        copies.append((Eq, Bq))
    b.bind(3, mk(E0), mk(B0), [torch.zeros(w.shape, device="cuda") for _ in range(3)])
    b.advance(3)
    for _, grid, _, _, _ in runs:
        grid.advance(3)
    torch.cuda.synchronize()
    for (Eq, Bq), (_, _, _, (Et, Bt, _), _) in zip(copies, runs):
        for a, c in zip(Eq + Bq, Et + Bt):
            assert torch.equal(a, c)
    g, _, (Eo, Bo, Jo), (Et, Bt, _), _ = runs[1]
    q.step(g, Eo, Bo, Jo, 3)
    for a, c in zip(Et + Bt, Eo + Bo):
        assert rel_err(a.cpu().numpy().view(np.float32).astype(np.float64), c.view(np.float64)) < TOL[32]
    b.close()
    for r in runs:
        r[1].close()


@pytest.mark.parametrize("m", [0, 1, 2])
def test_quasi3d_batched_workload_size(m):
    """The batched benchmark's quasi-3D modes at full size (nz x nr = 2048 x 512, FP32, dz = dr = 0.2,
    filtered): every output element against the oracle after two steps."""
    need_gpu()
    hyb = hyb_module()
    nz, nr, dz = 2048, 512, 0.2
    dt = min(0.08, 0.9 * 2 / np.sqrt(np.pi ** 2 / dz ** 2 + (4 * m * m + 6) / dz ** 2))
    g = q.QGrid(nz=nz, nr=nr, dz=dz, dr=dz, dt=dt, m=m, filt_kc=0.5, filt_w=0.2)
    E, B, J = _fields(nr, nz, 500 + m), _fields(nr, nz, 600 + m), _fields(nr, nz, 700 + m, 1e-2)
    rnd = lambda a: a.astype(np.complex64).astype(np.complex128)
    Eo, Bo, Jo = [rnd(a) for a in E], [rnd(a) for a in B], [rnd(a) for a in J]
    desc = hyb.make_desc(dims=20, n1=nz, n2=nr, dx1=dz, dx2=dz, dt=dt, precision=32, filt_kc=0.5, filt_w=0.2,
                         azimuthal_m=m)
    grid = hyb.Grid(desc)
    Et, Bt, Jt = ([torch.from_numpy(a).to("cuda", torch.complex64) for a in X] for X in (E, B, J))
    grid.bind(Et, Bt, Jt)
    q.step(g, Eo, Bo, Jo, 2)
    grid.advance(2)
    for a, b in zip(Et + Bt, Eo + Bo):
        assert rel_err(a.cpu().numpy().view(np.float32).astype(np.float64), b.view(np.float64)) < TOL[32]
    grid.close()
