"""GPU parity of the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances: 1e-12 relative per field for the FP64 GPU path, 1e-5 for FP32
(relative L2 error ||gpu - oracle|| / ||oracle|| per field)."""
import numpy as np
import pytest

from paper_1502_01376_gb300 import workloads as wl

from gpu_util import hyb_module, need_gpu, orc_grid, rel_err, to_dev, to_np, torch

pytestmark = pytest.mark.gpu

TOL = {64: 1e-12, 32: 1e-5}


def _setup(hyb, w, path=0, **over):
    dt = torch.float64 if w.precision == 64 else torch.float32
    desc = hyb.desc_from_workload(w, path=path, **over)
    g = hyb.Grid(desc)
    E0, B0 = wl.band_limited_fields(w)
    E = [to_dev(a, dt) for a in E0]
    B = [to_dev(a, dt) for a in B0]
    J = [torch.zeros(w.shape, device="cuda", dtype=dt) for _ in range(3)]
    g.bind(E, B, J)
    return g, E0, B0, E, B, J


def _compare(E, B, Eo, Bo, tol, tag=""):
    errs = [rel_err(to_np(a), b) for a, b in zip(E + B, Eo + Bo)]
    assert max(errs) < tol, (tag, errs)
    return errs


@pytest.mark.parametrize("path", [1, 0])
def test_vacuum_beam_workload_fp64_100_steps(orc, path):
    """Config: 2D 128x64 FP64, beam of 4096 particles at 0.99c, deposit each step, 100 steps."""
    need_gpu()
    hyb = hyb_module()
    w = wl.VACUUM_BEAM
    g, E0, B0, E, B, J = _setup(hyb, w, path=path)
    go = orc_grid(orc, w)
    p = wl.make_particles(w)
    Eo = [a.copy() for a in E0]
    Bo = [a.copy() for a in B0]
    for n in range(w.steps):
        cell, off0, off1, v3 = wl.ballistic_move(w, p, n)
        Jo = orc.deposit(go, cell, off0, off1, v3, p.q, w.shape_order)
        orc.step(go, Eo, Bo, Jo)
        g.deposit(torch.from_numpy(cell).cuda(), to_dev(off0, torch.float64), to_dev(off1, torch.float64),
                  to_dev(v3, torch.float64), to_dev(p.q, torch.float64), w.shape_order)
        g.advance(1)
        if n in (0, 9):
            _compare(E, B, Eo, Bo, TOL[64], f"step {n}")
    g.check()
    _compare(E, B, Eo, Bo, TOL[64], "final")


@pytest.mark.parametrize("n1,n2", [(64, 37), (256, 12), (1024, 5)])
@pytest.mark.parametrize("prec", [64, 32])
def test_three_pass_random_fields(orc, n1, n2, prec):
    need_gpu()
    hyb = hyb_module()
    w = wl.Workload("t", 2, n1, n2, dx1=0.2, dx2=0.25, dt=0.08, precision=prec, filt_kc=0.5, filt_w=0.2, seed=3)
    g, E0, B0, E, B, J = _setup(hyb, w, path=1)
    rng = np.random.default_rng(4)
    J0 = [rng.standard_normal(w.shape) * 1e-3 for _ in range(3)]
    dt = torch.float64 if prec == 64 else torch.float32
    for c in range(3):
        J[c].copy_(to_dev(J0[c], dt))
    rnd = (lambda a: a) if prec == 64 else (lambda a: a.astype(np.float32).astype(np.float64))
    Jin = [rnd(a) for a in J0]               # inputs rounded on the host exactly as the GPU sees them
    Ein = [rnd(a) for a in E0]
    Bin = [rnd(a) for a in B0]
    go = orc_grid(orc, w)
    nst = 10
    orc.step(go, Ein, Bin, Jin, nsteps=nst)
    g.advance(nst)
    _compare(E, B, Ein, Bin, TOL[prec])


@pytest.mark.parametrize("prec", [64, 32])
def test_three_pass_3d(orc, prec):
    need_gpu()
    hyb = hyb_module()
    w = wl.Workload("t3", 3, 64, 12, 10, dx1=0.2, dx2=0.2, dx3=0.25, dt=0.06, precision=prec,
                    filt_kc=0.6, filt_w=0.2, seed=5)
    g, E0, B0, E, B, J = _setup(hyb, w, path=1)
    rng = np.random.default_rng(6)
    dt = torch.float64 if prec == 64 else torch.float32
    J0 = [rng.standard_normal(w.shape) * 1e-3 for _ in range(3)]
    for c in range(3):
        J[c].copy_(to_dev(J0[c], dt))
    rnd = (lambda a: a) if prec == 64 else (lambda a: a.astype(np.float32).astype(np.float64))
    Jin = [rnd(a) for a in J0]
    Ein = [rnd(a) for a in E0]
    Bin = [rnd(a) for a in B0]
    go = orc_grid(orc, w)
    orc.step(go, Ein, Bin, Jin, nsteps=5)
    g.advance(5)
    _compare(E, B, Ein, Bin, TOL[prec])


@pytest.mark.parametrize("yee", [True, False])
def test_yee_mode_and_bump(orc, yee):
    need_gpu()
    hyb = hyb_module()
    w = wl.Workload("ty", 2, 128, 16, dx1=0.2, dx2=0.2, dt=0.08, precision=64, seed=8)
    over = dict(yee_mode=True) if yee else dict(kmod_l=0.15, kmod_u=0.26, kmod_max=0.01)
    g, E0, B0, E, B, J = _setup(hyb, w, path=1, **over)
    go = orc_grid(orc, w, **over)
    Eo, Bo = [a.copy() for a in E0], [a.copy() for a in B0]
    Jo = [np.zeros(w.shape) for _ in range(3)]
    orc.step(go, Eo, Bo, Jo, nsteps=4)
    g.advance(4)
    _compare(E, B, Eo, Bo, TOL[64])


@pytest.mark.parametrize("sort", [False, True])
@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("order", [1, 2, 3])
@pytest.mark.parametrize("dims", [2, 3])
def test_deposit_matches_oracle(orc, prec, order, dims, sort):
    """Random particle order (contributions added to J directly) and cell order (2D blocks add
    into a shared tile first)."""
    need_gpu()
    hyb = hyb_module()
    if dims == 2:
        w = wl.Workload("td", 2, 64, 24, dx1=0.2, dx2=0.3, dt=0.07, precision=prec, kind="plasma", ppc=2,
                        gamma=3.0, u_th=0.3, shape_order=order, seed=9)
    else:
        w = wl.Workload("td3", 3, 16, 8, 6, dx1=0.2, dx2=0.3, dx3=0.25, dt=0.05, precision=prec, kind="plasma",
                        ppc=1, gamma=2.0, u_th=0.3, shape_order=order, seed=10)
    real = np.float64 if prec == 64 else np.float32
    dt = torch.float64 if prec == 64 else torch.float32
    g, E0, B0, E, B, J = _setup(hyb, w, path=1)
    p = wl.make_particles(w)
    cell, off0, off1, v3 = wl.ballistic_move(w, p, 2, real=real)
    q = p.q.astype(real)
    if sort:
        key = np.zeros(len(q), dtype=np.int64)
        for a in reversed(range(dims)):
            key = key * (w.n1, w.n2, w.n3)[a] + cell[:, a]
        o = np.argsort(key, kind="stable")
        cell, off0, off1, v3, q = cell[o], off0[o], off1[o], v3[o], q[o]
    g.deposit(torch.from_numpy(cell).cuda(), to_dev(off0, dt), to_dev(off1, dt),
              to_dev(v3, dt) if dims == 2 else None, to_dev(q, dt), order)
    g.check()
    go = orc_grid(orc, w)
    Jo = orc.deposit(go, cell, off0.astype(np.float64), off1.astype(np.float64),
                     v3.astype(np.float64), q.astype(np.float64), order)
    tol = 1e-12 if prec == 64 else 1e-5
    for a, b in zip(J, Jo):
        assert rel_err(to_np(a), b) < tol


def test_deposit_flags_bad_particles():
    need_gpu()
    hyb = hyb_module()
    w = wl.Workload("tb", 2, 16, 8, dx1=0.2, dx2=0.2, dt=0.05, precision=64)
    g, E0, B0, E, B, J = _setup(hyb, w, path=1)
    cell = torch.tensor([[2, 3], [4, 4]], dtype=torch.int32, device="cuda")
    off0 = torch.tensor([[0.5, 0.5], [0.5, 0.5]], dtype=torch.float64, device="cuda")
    off1 = torch.tensor([[0.6, 0.5], [1.7, 0.5]], dtype=torch.float64, device="cuda")   # second moves > 1 cell
    q = torch.ones(2, dtype=torch.float64, device="cuda")
    g.deposit(cell, off0, off1, None, q, 1)
    with pytest.raises(hyb.HybError) as e:
        g.check()
    assert e.value.status == hyb.HYB_EDATA
    g.check()        # flag cleared


@pytest.mark.parametrize("prec", [64, 32])
def test_standalone_correction_and_filter(orc, prec):
    need_gpu()
    hyb = hyb_module()
    w = wl.Workload("tc", 2, 256, 10, dx1=0.2, dx2=0.2, dt=0.08, precision=prec, filt_kc=0.45, filt_w=0.3, seed=11)
    g, E0, B0, E, B, J = _setup(hyb, w, path=1)
    dt = torch.float64 if prec == 64 else torch.float32
    rng = np.random.default_rng(12)
    J0 = [rng.standard_normal(w.shape) for _ in range(3)]
    for c in range(3):
        J[c].copy_(to_dev(J0[c], dt))
    rnd = (lambda a: a) if prec == 64 else (lambda a: a.astype(np.float32).astype(np.float64))
    Jo = [rnd(a) for a in J0]
    go = orc_grid(orc, w)
    g.correct_current()
    orc.process_current(go, Jo, True, False)
    g.filter()
    orc.process_current(go, Jo, False, True)
    for a, b in zip(J, Jo):
        assert rel_err(to_np(a), b) < (1e-13 if prec == 64 else 1e-6)


@pytest.mark.parametrize("prec", [64, 32])
def test_diag_matches_oracle(orc, prec):
    need_gpu()
    hyb = hyb_module()
    w = wl.VACUUM_BEAM.scaled(n1=64, n2=20, n_particles=32, precision=prec, filt_kc=0.5, filt_w=0.2)
    dt = torch.float64 if prec == 64 else torch.float32
    desc = hyb.desc_from_workload(w, path=1)
    g = hyb.Grid(desc)
    E0, B0 = wl.band_limited_fields(w)
    E = [to_dev(a, dt) for a in E0]
    B = [to_dev(a, dt) for a in B0]
    J = [torch.zeros(w.shape, device="cuda", dtype=dt) for _ in range(3)]
    p = wl.make_particles(w)
    go = orc_grid(orc, w)
    cell, off0 = wl.position_at(w, p, 0)
    rho_np = orc.charge(go, cell, off0, p.q, 1)
    rho = to_dev(rho_np, dt)
    g.bind(E, B, J, rho)
    got = g.diag()
    rnd = (lambda a: a) if prec == 64 else (lambda a: a.astype(np.float32).astype(np.float64))
    want = orc.diag(go, [rnd(a) for a in E0], [rnd(a) for a in B0], rnd(rho_np))
    tol = 1e-11 if prec == 64 else 1e-5
    assert np.allclose(got[:6], want[:6], rtol=tol, atol=0)
    assert got[6] == pytest.approx(want[6], rel=1e-6 if prec == 32 else 1e-9)
    assert got[7] == pytest.approx(want[7], rel=1e-6 if prec == 32 else 1e-9)
    assert got[8] == pytest.approx(want[8], rel=1e-6 if prec == 32 else 1e-9)


def test_gauss_invariant_on_gpu(orc):
    """Gauss residual from the GPU's own diagnostic stays constant with the correction (Sec. 2.3)."""
    need_gpu()
    hyb = hyb_module()
    w = wl.VACUUM_BEAM.scaled(n1=64, n2=32, n_particles=128)
    desc = hyb.desc_from_workload(w)
    g = hyb.Grid(desc)
    E0, B0 = wl.band_limited_fields(w)
    E = [to_dev(a, torch.float64) for a in E0]
    B = [to_dev(a, torch.float64) for a in B0]
    J = [torch.zeros(w.shape, device="cuda", dtype=torch.float64) for _ in range(3)]
    rho = torch.zeros(w.shape, device="cuda", dtype=torch.float64)
    g.bind(E, B, J, rho)
    p = wl.make_particles(w)
    go = orc_grid(orc, w)
    for n in range(20):
        cell, off0, off1, v3 = wl.ballistic_move(w, p, n)
        rho.copy_(to_dev(orc.charge(go, cell, off0, p.q, 1), torch.float64))
        g0 = g.diag()
        g.deposit(torch.from_numpy(cell).cuda(), to_dev(off0, torch.float64), to_dev(off1, torch.float64),
                  to_dev(v3, torch.float64), to_dev(p.q, torch.float64), 1)
        g.advance(1)
        rho.copy_(to_dev(orc.charge(go, cell, off1, p.q, 1), torch.float64))
        g1 = g.diag()
        assert abs(g1[8] - g0[8]) < 1e-11 * max(g0[8], 1.0)


def test_advance_host_matches_device(orc):
    need_gpu()
    hyb = hyb_module()
    w = wl.Workload("th", 2, 128, 16, dx1=0.2, dx2=0.2, dt=0.08, precision=64, seed=13)
    g, E0, B0, E, B, J = _setup(hyb, w, path=1)
    Eh = [torch.from_numpy(a.copy()).pin_memory() for a in E0]
    Bh = [torch.from_numpy(a.copy()).pin_memory() for a in B0]
    Jh = [torch.zeros(w.shape, dtype=torch.float64).pin_memory() for _ in range(3)]
    g.advance_host(Eh, Bh, Jh, 3)
    g.advance(0)
    Eo, Bo = [a.copy() for a in E0], [a.copy() for a in B0]
    orc.step(orc_grid(orc, w), Eo, Bo, [np.zeros(w.shape)] * 3, nsteps=3)
    for a, b in zip(Eh + Bh, Eo + Bo):
        assert rel_err(a.numpy(), b) < 1e-12


@pytest.mark.parametrize("n1,n2", [(4096, 1024), (1024, 37), (512, 4), (2048, 70)])
def test_fused_host_step_matches_device_step(n1, n2):
    """One fused step from and to host arrays (copies and compute pipelined over chunks of rows,
    halo rows taken before the rows they come from are updated) equals the device-array step."""
    need_gpu()
    hyb = hyb_module()
    w = wl.Workload("hp", 2, n1, n2, dx1=0.2, dx2=0.2, dt=0.1, precision=32, filt_kc=0.5, filt_w=0.2, seed=17)
    rng = np.random.default_rng(n1 + n2)
    F0 = [rng.standard_normal(w.shape).astype(np.float32) * np.float32(1e-3) for _ in range(9)]
    gd = hyb.Grid(hyb.desc_from_workload(w))
    assert gd.path == 2
    D = [torch.from_numpy(a.copy()).cuda() for a in F0]
    gd.bind(D[0:3], D[3:6], D[6:9])
    gd.advance(1)
    gh = hyb.Grid(hyb.desc_from_workload(w))
    Dh = [torch.zeros(w.shape, device="cuda") for _ in range(9)]
    gh.bind(Dh[0:3], Dh[3:6], Dh[6:9])
    H = [torch.from_numpy(a.copy()).pin_memory() for a in F0]
    for _ in range(2):                      # twice: the second call reuses the pipeline's plan
        for h, a in zip(H, F0):
            h.copy_(torch.from_numpy(a))
        gh.advance_host(H[0:3], H[3:6], H[6:9], 1)
    gh.check()
    torch.cuda.synchronize()
    for a, b, dev in zip(H[:6], D[:6], Dh[:6]):
        assert torch.equal(a, b.cpu()), float((a - b.cpu()).abs().max())
        assert torch.equal(dev.cpu(), a)
    gd.close()
    gh.close()


def test_courant_rejected_and_alignment():
    need_gpu()
    hyb = hyb_module()
    d = hyb.make_desc(n1=64, n2=16, dx1=0.2, dx2=0.2, dt=0.2)
    with pytest.raises(hyb.HybError) as e:
        hyb.Grid(d)
    assert e.value.status == hyb.HYB_ECOURANT
    d = hyb.make_desc(n1=64, n2=16, dx1=0.2, dx2=0.2, dt=0.05, precision=64)
    g = hyb.Grid(d)
    base = torch.zeros(64 * 16 + 1, dtype=torch.float64, device="cuda")
    ok = [torch.zeros(64 * 16, dtype=torch.float64, device="cuda") for _ in range(8)]
    ptrs = [int(t.data_ptr()) for t in ok]
    with pytest.raises(hyb.HybError) as e:
        hyb.hyb_bind_fields(g.h, [int(base.data_ptr()) + 8] + ptrs[:2], ptrs[2:5], ptrs[5:8])
    assert e.value.status == hyb.HYB_EALIGN
    with pytest.raises(hyb.HybError) as e:
        g.advance(1)
    assert e.value.status == hyb.HYB_ESTATE


# ------------------------------------------------------------------ fused FP32 path
def _fused_case(orc, hyb, n1, n2, nsteps, filt=True, seed=21, amp_j=1e-3):
    w = wl.Workload("tf", 2, n1, n2, dx1=0.2, dx2=0.2, dt=0.1, precision=32,
                    filt_kc=0.5 if filt else 0.0, filt_w=0.2, seed=seed)
    g, E0, B0, E, B, J = _setup(hyb, w, path=2)
    assert g.path == 2
    rng = np.random.default_rng(seed + 1)
    J0 = [rng.standard_normal(w.shape) * amp_j for _ in range(3)]
    for c in range(3):
        J[c].copy_(to_dev(J0[c], torch.float32))
    rnd = lambda a: a.astype(np.float32).astype(np.float64)
    Eo, Bo, Jo = [rnd(a) for a in E0], [rnd(a) for a in B0], [rnd(a) for a in J0]
    orc.step(orc_grid(orc, w), Eo, Bo, Jo, nsteps=nsteps)
    g.advance(nsteps)
    return _compare(E, B, Eo, Bo, TOL[32], f"fused {n1}x{n2}")


@pytest.mark.parametrize("n1,n2", [(512, 8), (512, 37), (1024, 21), (2048, 13), (4096, 9), (4096, 64)])
def test_fused_matches_oracle(orc, n1, n2):
    need_gpu()
    hyb = hyb_module()
    _fused_case(orc, hyb, n1, n2, 10)


@pytest.mark.parametrize("n1,n2,path", [(4096, 64, 2), (2048, 24, 2), (1024, 21, 2), (512, 16, 2), (1024, 12, 1),
                                       (256, 12, 1)])
def test_per_field_accuracy_with_components_of_unequal_size(orc, n1, n2, path):
    """Per-field relative error stays at FP32 level when the components differ by orders of
    magnitude, as in the drifting plasma, where the drive j1 is large and the TE fields
    (E3, B1, B2) are far weaker than E2, B3: a transform that mixed two fields would give the
    weak one an error on the scale of the strong one."""
    need_gpu()
    hyb = hyb_module()
    w = wl.Workload("mix", 2, n1, n2, dx1=0.2, dx2=0.2, dt=0.1, precision=32, filt_kc=0.5, filt_w=0.2, seed=41)
    g, E0, B0, E, B, J = _setup(hyb, w, path=path)
    scale_e, scale_b = (1.0, 1.0, 1e-5), (1e-5, 1e-5, 1.0)
    E0 = [a * s for a, s in zip(E0, scale_e)]
    B0 = [a * s for a, s in zip(B0, scale_b)]
    rng = np.random.default_rng(42)
    J0 = [rng.standard_normal(w.shape) * s for s in (1e-1, 1e-3, 1e-9)]
    for t, a in zip(E + B + J, E0 + B0 + J0):
        t.copy_(to_dev(a, torch.float32))
    rnd = lambda a: a.astype(np.float32).astype(np.float64)
    Eo, Bo, Jo = [rnd(a) for a in E0], [rnd(a) for a in B0], [rnd(a) for a in J0]
    orc.step(orc_grid(orc, w), Eo, Bo, Jo, nsteps=5)
    g.advance(5)
    _compare(E, B, Eo, Bo, TOL[32], f"unequal components {n1}x{n2} path {path}")


def test_fused_without_filter_and_correction(orc):
    need_gpu()
    hyb = hyb_module()
    w = wl.Workload("tf", 2, 1024, 16, dx1=0.2, dx2=0.2, dt=0.1, precision=32, correct_j1=False, seed=3)
    g, E0, B0, E, B, J = _setup(hyb, w, path=2)
    rng = np.random.default_rng(5)
    J0 = [rng.standard_normal(w.shape) * 1e-3 for _ in range(3)]
    for c in range(3):
        J[c].copy_(to_dev(J0[c], torch.float32))
    rnd = lambda a: a.astype(np.float32).astype(np.float64)
    Eo, Bo, Jo = [rnd(a) for a in E0], [rnd(a) for a in B0], [rnd(a) for a in J0]
    orc.step(orc_grid(orc, w), Eo, Bo, Jo, nsteps=5)
    g.advance(5)
    _compare(E, B, Eo, Bo, TOL[32])


def test_fused_matches_three_pass_fp32():
    """Same arithmetic problem through the two FP32 paths."""
    need_gpu()
    hyb = hyb_module()
    w = wl.Workload("tf", 2, 2048, 40, dx1=0.2, dx2=0.2, dt=0.1, precision=32, filt_kc=0.5, filt_w=0.2, seed=9)
    ga, E0, B0, Ea, Ba, Ja = _setup(hyb, w, path=2)
    gb, _, _, Eb, Bb, Jb = _setup(hyb, w, path=1)
    rng = np.random.default_rng(10)
    for c in range(3):
        j = to_dev(rng.standard_normal(w.shape) * 1e-3, torch.float32)
        Ja[c].copy_(j)
        Jb[c].copy_(j)
    ga.advance(20)
    gb.advance(20)
    for a, b in zip(Ea + Ba, Eb + Bb):
        assert rel_err(to_np(a), to_np(b)) < 1e-5


def test_fused_full_size_drift_plasma_grid(orc):
    """The 4096 x 1024 grid in the launch configuration the benchmark times, 3 steps."""
    need_gpu()
    hyb = hyb_module()
    errs = _fused_case(orc, hyb, 4096, 1024, 3, seed=31)
    assert max(errs) < 1e-5


@pytest.mark.parametrize("n1,n2", [(2048, 2048), (512, 8192)])
def test_fused_team_kernel_full_size_grid(orc, n1, n2):
    """The same 4.19 M cells with rows of 2048 and 512 points, in the launch configuration of
    `bench.py --n1`: the team kernel at two CTAs per SM (304 and 1216 strips of about 7 rows,
    halo rows copied before each step), 3 steps against the oracle on every element."""
    need_gpu()
    hyb = hyb_module()
    errs = _fused_case(orc, hyb, n1, n2, 3, seed=41)
    assert max(errs) < 1e-5


def test_three_pass_3d_full_size_sampled_rows(orc):
    """The 3D 1024 x 256 x 256 FP32 grid in the launch configuration the benchmark times, one step,
    checked on sampled x1 rows: after one step a row depends only on the rows of its 3 x 3 (x2, x3)
    neighbourhood (Faraday reads E one row ahead, Ampere reads B one row behind), so the oracle run on
    that periodic 1024 x 3 x 3 window gives the exact centre row."""
    need_gpu()
    hyb = hyb_module()
    w = wl.DRIFT_PLASMA_3D
    n3, n2, n1 = w.shape
    rng = np.random.default_rng(77)
    host = [rng.standard_normal(w.shape, dtype=np.float32) * np.float32(1e-3) for _ in range(9)]
    dev = [torch.from_numpy(a).cuda() for a in host]
    g = hyb.Grid(hyb.desc_from_workload(w, path=1))
    g.bind(dev[0:3], dev[3:6], dev[6:9])
    g.advance(1)
    g.check()
    torch.cuda.synchronize()
    ww = w.scaled(n2=3, n3=3)
    go = orc_grid(orc, ww)
    samples = [(0, 0), (0, n2 - 1), (n3 - 1, 0), (n3 - 1, n2 - 1), (1, 3), (128, 127), (255, 128)]
    samples += [tuple(int(v) for v in rng.integers(0, (n3, n2))) for _ in range(5)]
    for i3, i2 in samples:
        win = np.ix_([(i3 - 1) % n3, i3, (i3 + 1) % n3], [(i2 - 1) % n2, i2, (i2 + 1) % n2])
        fw = [a[win].astype(np.float64) for a in host]
        Eo, Bo = fw[0:3], fw[3:6]
        orc.step(go, Eo, Bo, fw[6:9], nsteps=1)
        for name, d, o in zip(("E1", "E2", "E3", "B1", "B2", "B3"), dev[0:6], Eo + Bo):
            got = d[i3, i2].double().cpu().numpy()
            ref = o[1, 1]
            err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
            assert err < TOL[32], (i3, i2, name, err)
    g.close()


@pytest.mark.parametrize("prec", [64, 32])
def test_three_pass_step_inside_a_caller_graph(prec):
    """hyb_advance on the three-pass path replays its own captured step graph; called while the
    caller captures a CUDA graph of its own it launches plainly into that capture, and replaying
    the caller's graph advances the fields exactly like direct calls."""
    need_gpu()
    hyb = hyb_module()
    w = wl.Workload("cg", 3, 64, 6, 5, dx1=0.2, dx2=0.2, dx3=0.25, dt=0.06, precision=prec, filt_kc=0.5,
                    filt_w=0.2, seed=23)
    dt = torch.float64 if prec == 64 else torch.float32
    rng = np.random.default_rng(5)
    F0 = [rng.standard_normal(w.shape) * 1e-3 for _ in range(9)]
    ga = hyb.Grid(hyb.desc_from_workload(w, path=1))
    A = [to_dev(a, dt) for a in F0]
    ga.bind(A[0:3], A[3:6], A[6:9])
    ga.advance(1)                           # warm: tables, launch attributes, the grid's own step graph
    gb = hyb.Grid(hyb.desc_from_workload(w, path=1))
    Bt = [to_dev(a, dt) for a in F0]
    gb.bind(Bt[0:3], Bt[3:6], Bt[6:9])
    gb.advance(1)
    s = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    hyb.hyb_set_stream(gb.h, s.cuda_stream)
    with torch.cuda.graph(graph, stream=s):
        gb.advance(1)
    torch.cuda.synchronize()
    for _ in range(3):
        graph.replay()
    ga.advance(3)
    torch.cuda.synchronize()
    for a, b in zip(A[:6], Bt[:6]):
        assert torch.equal(a, b)
    ga.close()
    gb.close()
