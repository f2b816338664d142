"""Field gather + relativistic Boris push (hyb_push) against the FP64 oracle:
2D and 3D, FP32 and FP64, shape orders 1-3, particles that start outside their
cell, rejected particles, and the drifting-plasma benchmark (4096 x 1024, 8 + 8
particles per cell) on a sample of particles."""
import numpy as np
import pytest

from oracle import push as P
from paper_1502_01376_gb300 import workloads as wl

from gpu_util import hyb_module, need_gpu, torch

pytestmark = pytest.mark.gpu

TOL = {32: 1e-5, 64: 1e-12}


def _grid(hyb, dims, prec, shape, dt=0.08, dx=0.2):
    kw = dict(dims=dims, n1=shape[0], n2=shape[1], dx1=dx, dx2=dx, dt=dt, precision=prec)
    if dims == 3:
        kw.update(n3=shape[2], dx3=dx)
    return hyb.Grid(hyb.make_desc(**kw))


def _check(res, ref, prec, dims):
    cell, off, u, off_new, v3 = res
    c2, o2, un, on, v3o, ok = ref
    assert np.array_equal(cell, c2)
    assert np.array_equal(off.astype(np.float64), o2)           # same decision, same precision
    tol = TOL[prec]
    assert np.max(np.abs(u - un)) <= tol * max(1.0, np.max(np.abs(un)))
    assert np.max(np.abs(off_new - on)) <= tol
    if v3 is not None:
        assert np.max(np.abs(v3 - v3o)) <= tol


@pytest.mark.parametrize("sort", [False, True])
@pytest.mark.parametrize("prec", [32, 64])
@pytest.mark.parametrize("order", [1, 2, 3])
@pytest.mark.parametrize("dims", [2, 3])
def test_push_matches_oracle(dims, order, prec, sort):
    """Random particles (each block's cells spread over the grid: gathers from global memory) and
    the same particles sorted by cell (2D blocks stage their fields in a shared tile)."""
    need_gpu()
    hyb = hyb_module()
    shape = (128, 40) if dims == 2 else (32, 12, 10)
    rng = np.random.default_rng(100 * dims + 10 * order + prec)
    dt_np = np.float32 if prec == 32 else np.float64
    tdt = torch.float32 if prec == 32 else torch.float64
    g = _grid(hyb, dims, prec, shape)
    fields = [rng.standard_normal(shape[::-1]).astype(dt_np) for _ in range(6)]
    n = 40000 if sort else 6000          # sorted: about 8 particles per 2D cell, as in the workload
    cell = np.stack([rng.integers(0, s, n) for s in shape], axis=1).astype(np.int32)
    off = rng.uniform(0.0, 1.0, (n, dims))
    off[: n // 3] = rng.uniform(-1.0, 2.0, (n // 3, dims))      # a previous step's off_new
    off = off.astype(dt_np)
    u = (rng.standard_normal((n, 3)) * 20.0).astype(dt_np)
    qm = rng.choice([-1.0, 1.0], n).astype(dt_np)
    if sort:
        key = np.zeros(n, dtype=np.int64)
        for a in reversed(range(dims)):
            key = key * shape[a] + cell[:, a]
        o = np.argsort(key, kind="stable")
        cell, off, u, qm = cell[o], off[o], u[o], qm[o]
    E = [torch.from_numpy(f).cuda() for f in fields[:3]]
    B = [torch.from_numpy(f).cuda() for f in fields[3:]]
    J = [torch.zeros(shape[::-1], dtype=tdt, device="cuda") for _ in range(3)]
    g.bind(E, B, J)
    tc, to, tu, tq = (torch.from_numpy(a.copy()).cuda() for a in (cell, off, u, qm))
    on = torch.empty_like(to)
    v3 = torch.empty(n, dtype=tdt, device="cuda") if dims == 2 else None
    g.push(tc, to, tu, tq, on, v3, order=order)
    g.check()
    ref = P.push(fields, cell, off, u, qm, 0.08, np.array([0.2, 0.2, 0.2]), order)
    assert ref[5].all()
    _check((tc.cpu().numpy(), to.cpu().numpy(), tu.cpu().numpy().astype(np.float64),
            on.cpu().numpy().astype(np.float64), None if v3 is None else v3.cpu().numpy().astype(np.float64)),
           ref, prec, dims)
    g.close()


def test_push_rejects_out_of_range_particles():
    """Offsets outside [-1, 2) or cells out of range: left unchanged, off_new = off, flagged."""
    need_gpu()
    hyb = hyb_module()
    shape = (32, 16)
    g = _grid(hyb, 2, 32, shape)
    E = [torch.ones(shape[::-1], device="cuda") for _ in range(3)]
    B = [torch.ones(shape[::-1], device="cuda") for _ in range(3)]
    J = [torch.zeros(shape[::-1], device="cuda") for _ in range(3)]
    g.bind(E, B, J)
    cell = torch.tensor([[3, 4], [3, 4], [32, 0], [5, 5]], dtype=torch.int32, device="cuda")
    off = torch.tensor([[0.5, 0.5], [2.5, 0.5], [0.5, 0.5], [0.5, -1.5]], device="cuda")
    u = torch.ones(4, 3, device="cuda")
    qm = torch.ones(4, device="cuda")
    on = torch.empty_like(off)
    c0, o0, u0 = cell.clone(), off.clone(), u.clone()
    g.push(cell, off, u, qm, on, None, order=2)
    with pytest.raises(hyb.HybError):
        g.check()
    assert torch.equal(cell[1:], c0[1:]) and torch.equal(off[1:], o0[1:]) and torch.equal(u[1:], u0[1:])
    assert torch.equal(on[1:], o0[1:])
    assert not torch.equal(u[0], u0[0])          # the valid particle moved on
    g.close()


def test_push_drift_plasma_full_size_sampled():
    """The benchmark's workload: 4096 x 1024 FP32, 8 + 8 particles per cell (67 M), quadratic
    shapes, band-limited random E and B; 20 000 sampled particles against the oracle."""
    need_gpu()
    hyb = hyb_module()
    w = wl.DRIFT_PLASMA
    E0, B0 = wl.band_limited_fields(w)
    fields = [a.astype(np.float32) for a in list(E0) + list(B0)]
    g = hyb.Grid(hyb.desc_from_workload(w))
    E = [torch.from_numpy(f).cuda() for f in fields[:3]]
    B = [torch.from_numpy(f).cuda() for f in fields[3:]]
    J = [torch.zeros(w.shape, device="cuda") for _ in range(3)]
    g.bind(E, B, J)
    cell, off, u, qm = wl.plasma_push_particles_torch(w, "cuda")
    n = qm.numel()
    assert n == 2 * w.ppc * w.cells
    sel = torch.from_numpy(np.random.default_rng(7).choice(n, 20000, replace=False)).cuda()
    ins = [t[sel].cpu().numpy() for t in (cell, off, u, qm)]
    on = torch.empty_like(off)
    v3 = torch.empty_like(qm)
    g.push(cell, off, u, qm, on, v3, order=w.shape_order)
    g.check()
    ref = P.push(fields, ins[0], ins[1], ins[2], ins[3], w.dt, np.array([w.dx1, w.dx2]), w.shape_order)
    _check((cell[sel].cpu().numpy(), off[sel].cpu().numpy(), u[sel].cpu().numpy().astype(np.float64),
            on[sel].cpu().numpy().astype(np.float64), v3[sel].cpu().numpy().astype(np.float64)), ref, 32, 2)
    g.close()


def test_push_checks_pair_alignment():
    """2D offsets are read as one pair per particle: a pointer one real off the pair is refused
    on the host (HYB_EALIGN) before any launch."""
    need_gpu()
    hyb = hyb_module()
    shape = (32, 16)
    g = _grid(hyb, 2, 32, shape)
    E = [torch.zeros(shape[::-1], device="cuda") for _ in range(3)]
    g.bind(E, [t.clone() for t in E], [t.clone() for t in E])
    cell = torch.zeros(8, 2, dtype=torch.int32, device="cuda")
    buf = torch.zeros(17, device="cuda")
    off = buf[1:].view(8, 2)                     # 4-byte offset from the pair boundary
    u = torch.zeros(8, 3, device="cuda")
    qm = torch.ones(8, device="cuda")
    on = torch.zeros(8, 2, device="cuda")
    with pytest.raises(hyb.HybError, match="HYB_EALIGN"):
        g.push(cell, off, u, qm, on, None, order=1)
    g.close()
