"""The batched step as ONE persistent launch (hyb_batch_* single launch): fused 2D grids of every
row length the fused kernels take (n1 = 512, 1024, 2048, 4096; strips of uneven height) and
quasi-3D modes m = 0, 1, 2 (nz = 2048) advanced by a launch whose CTAs are split into roles give
exactly the bits of the graph of separate launches and of the single grids; the autotuner's split
and choice of form leave the bound fields as they were; the oracle checks one grid and one mode."""
import numpy as np
import pytest

from oracle import quasi3d as q
from paper_1502_01376_gb300 import workloads as wl

from gpu_util import hyb_module, need_gpu, orc_grid, rel_err, to_dev, to_np, torch

pytestmark = pytest.mark.gpu

SIZES_2D = [(512, 64), (512, 37), (1024, 96), (2048, 40), (2048, 128), (4096, 24), (4096, 70)]
NR_Q3 = 40


def _q3_desc(hyb, m):
    dz, dr = 0.2, 0.2
    dt = 0.9 * 2 / np.sqrt(np.pi ** 2 / dz ** 2 + (4 * m * m + 6) / dr ** 2)
    return hyb.make_desc(dims=20, n1=2048, n2=NR_Q3, dx1=dz, dx2=dr, dt=dt, precision=32, filt_kc=0.5,
                         filt_w=0.2, azimuthal_m=m), dt


def _q3_fields(seed):
    rng = np.random.default_rng(seed)
    mk = lambda s: [(rng.standard_normal((NR_Q3, 2048)) + 1j * rng.standard_normal((NR_Q3, 2048))) * s for _ in range(3)]
    return mk(1.0), mk(1.0), mk(1e-2)


def _setup(hyb, with_2d=True, with_q3=True):
    descs, inputs, ws = [], [], []
    if with_2d:
        for i, (n1, n2) in enumerate(SIZES_2D):
            w = wl.Workload(f"s{i}", 2, n1, n2, dx1=0.2, dx2=0.2, dt=0.08, precision=32, filt_kc=0.5, filt_w=0.2,
                            seed=60 + i)
            E0, B0 = wl.band_limited_fields(w)
            rng = np.random.default_rng(i)
            J0 = [rng.standard_normal(w.shape) * 1e-3 for _ in range(3)]
            descs.append(hyb.desc_from_workload(w))
            inputs.append(("2d", E0, B0, J0))
            ws.append(w)
    if with_q3:
        for m in (0, 1, 2):
            d, dt = _q3_desc(hyb, m)
            descs.append(d)
            inputs.append(("q3",) + _q3_fields(70 + m))
            ws.append((m, dt))
    return descs, inputs, ws


def _bind(batch, inputs):
    bufs = []
    for i, (kind, E, B, J) in enumerate(inputs):
        if kind == "2d":
            mk = lambda arrs: [to_dev(a, torch.float32) for a in arrs]
        else:
            mk = lambda arrs: [torch.from_numpy(a.astype(np.complex64)).cuda() for a in arrs]
        t = (mk(E), mk(B), mk(J))
        batch.bind(i, *t)
        bufs.append(t)
    return bufs


def _same(bufs_a, bufs_b, what):
    for i, (a, b) in enumerate(zip(bufs_a, bufs_b)):
        for x, y in zip(a[0] + a[1], b[0] + b[1]):
            assert torch.equal(x, y), (i, what)


@pytest.mark.parametrize("with_2d,with_q3", [(True, True), (True, False), (False, True)])
def test_single_launch_equals_graph_of_launches(with_2d, with_q3):
    need_gpu()
    hyb = hyb_module()
    descs, inputs, _ = _setup(hyb, with_2d, with_q3)
    one = hyb.Batch(descs)
    many = hyb.Batch(descs)
    assert one.single_launch and one.launches_per_step == 1
    many.single_launch = False
    assert not many.single_launch and many.launches_per_step >= 2
    ctas = one.role_ctas()
    present = ([with_2d] * 4) + [with_q3]
    assert all((c >= 1) == p for c, p in zip(ctas, present)), ctas
    ba, bb = _bind(one, inputs), _bind(many, inputs)
    one.advance(5)
    many.advance(5)
    one.check()
    many.check()
    _same(ba, bb, "5 steps")
    one.close()
    many.close()


def test_single_launch_tuned_singles_and_oracle(orc):
    """Autotuner (strips, split of the CTAs, form of the step) on the bound fields: they end as they
    were; then the batch equals the single grids step by step, and the oracle one 2D grid and one
    mode."""
    need_gpu()
    hyb = hyb_module()
    descs, inputs, ws = _setup(hyb)
    batch = hyb.Batch(descs)
    bufs = _bind(batch, inputs)
    singles, sbufs = [], []
    for i, d in enumerate(descs):
        g = hyb.Grid(d)
        kind, E, B, J = inputs[i]
        if kind == "2d":
            mk = lambda arrs: [to_dev(a, torch.float32) for a in arrs]
        else:
            mk = lambda arrs: [torch.from_numpy(a.astype(np.complex64)).cuda() for a in arrs]
        t = (mk(E), mk(B), mk(J))
        g.bind(*t)
        singles.append(g)
        sbufs.append(t)
    before = [[x.clone() for x in b[0] + b[1]] for b in bufs]
    batch.tune(2)
    torch.cuda.synchronize()
    for b, c in zip(bufs, before):
        for x, y in zip(b[0] + b[1], c):
            assert torch.equal(x, y)
    ctas = batch.role_ctas()
    assert all(c >= 1 for c in ctas) and sum(ctas) == torch.cuda.get_device_properties(0).multi_processor_count
    batch.single_launch = True
    nst = 4
    batch.advance(nst)
    for g in singles:
        g.advance(nst)
    torch.cuda.synchronize()
    _same(bufs, sbufs, "single launch vs single grids")
    # oracle: the 4096 x 70 grid and mode m = 1
    i2 = SIZES_2D.index((4096, 70))
    w = ws[i2]
    _, E0, B0, J0 = inputs[i2]
    rnd = lambda a: a.astype(np.float32).astype(np.float64)
    Eo, Bo, Jo = [rnd(a) for a in E0], [rnd(a) for a in B0], [rnd(a) for a in J0]
    orc.step(orc_grid(orc, w), Eo, Bo, Jo, nsteps=nst)
    for a, b in zip(bufs[i2][0] + bufs[i2][1], Eo + Bo):
        assert rel_err(to_np(a), b) < 1e-5
    iq = len(SIZES_2D) + 1
    m, dt = ws[iq]
    gq = q.QGrid(nz=2048, nr=NR_Q3, dz=0.2, dr=0.2, dt=dt, m=m, filt_kc=0.5, filt_w=0.2)
    _, E, B, J = inputs[iq]
    rq = lambda a: a.astype(np.complex64).astype(np.complex128)
    Eo, Bo, Jo = [rq(a) for a in E], [rq(a) for a in B], [rq(a) for a in J]
    q.step(gq, Eo, Bo, Jo, nst)
    for a, c in zip(bufs[iq][0] + bufs[iq][1], Eo + Bo):
        assert rel_err(a.cpu().numpy().view(np.float32).astype(np.float64), c.view(np.float64)) < 1e-5
    batch.close()
    for g in singles:
        g.close()


def test_single_launch_needs_every_grid_in_a_role():
    """An FP64 grid (three-pass path) has no role: the batch keeps the graph of launches and refuses
    the single launch."""
    need_gpu()
    hyb = hyb_module()
    w = wl.Workload("a", 2, 1024, 32, dx1=0.2, dx2=0.2, dt=0.08, precision=32, seed=1)
    w64 = wl.Workload("b", 2, 256, 16, dx1=0.2, dx2=0.2, dt=0.08, precision=64, seed=2)
    b = hyb.Batch([hyb.desc_from_workload(w), hyb.desc_from_workload(w64)])
    assert not b.single_launch and b.role_ctas() == [0] * 5
    with pytest.raises(hyb.HybError):
        b.single_launch = True
    b.close()


def test_role_split_set_by_hand():
    """A split set by hand (every role at least one CTA, at most one CTA per SM) gives the same bits;
    a split that leaves a role without CTAs, or gives one to an absent role, is refused."""
    need_gpu()
    hyb = hyb_module()
    descs, inputs, _ = _setup(hyb)
    one = hyb.Batch(descs)
    many = hyb.Batch(descs)
    many.single_launch = False
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    with pytest.raises(hyb.HybError):
        one.set_role_ctas([0, 10, 10, 10, 10])
    with pytest.raises(hyb.HybError):
        one.set_role_ctas([sms, 1, 1, 1, 1])
    one.set_role_ctas([1, 2, 3, 4, 5])                    # far from balanced, most CTAs idle
    ba, bb = _bind(one, inputs), _bind(many, inputs)
    one.advance(3)
    many.advance(3)
    torch.cuda.synchronize()
    _same(ba, bb, "split by hand")
    one.close()
    many.close()
    q3_only = hyb.Batch(_setup(hyb, with_2d=False)[0])
    with pytest.raises(hyb.HybError):
        q3_only.set_role_ctas([1, 0, 0, 0, 10])
    q3_only.set_role_ctas([0, 0, 0, 0, 3])
    q3_only.close()
