"""The particle-in-cell step (hyb_pic_step) against the oracle's composition of the
same steps: B^{n+1/2} from the oracle's advance of a copy with zero current, B^n the
mean of B^{n-1/2} and B^{n+1/2}, the oracle's gather and Boris push with E^n, B^n,
its charge-conserving deposit, its advance; particles and fields compared element
by element (FP64 over three steps, FP32 over one).  The same with k1-resident
fields, where the step forms B^n from the resident spectra instead."""
import numpy as np
import pytest

from oracle import push as P
from paper_1502_01376_gb300 import workloads as wl

from gpu_util import hyb_module, need_gpu, rel_err, torch

pytestmark = pytest.mark.gpu


def _oracle_pic(orc, g, E, B, cell, off, u, qm, q, order, dt, dx, steps):
    E = [a.copy() for a in E]
    B = [a.copy() for a in B]
    for _ in range(steps):
        Ec, Bc = [a.copy() for a in E], [a.copy() for a in B]
        orc.step(g, Ec, Bc, [np.zeros_like(a) for a in E], 1)          # B^{n+1/2}
        Bn = [0.5 * (a + b) for a, b in zip(B, Bc)]
        c2, o2, un, on, v3, ok = P.push(E + Bn, cell, off, u, qm, dt, dx, order)
        assert ok.all()
        c2 = np.ascontiguousarray(c2, dtype=np.int32)
        J = orc.deposit(g, c2, np.ascontiguousarray(o2), np.ascontiguousarray(on), np.ascontiguousarray(v3), q, order)
        orc.step(g, E, B, J, 1)
        cell, off, u = c2, on, un
    return E, B, cell, off, u


@pytest.mark.parametrize("resident", [False, True])
@pytest.mark.parametrize("prec,steps,order", [(64, 3, 2), (64, 2, 3), (64, 2, 1), (32, 1, 2)])
def test_pic_steps_match_oracle(prec, steps, order, resident, orc):
    need_gpu()
    hyb = hyb_module()
    # FP32: a warm, mildly relativistic plasma, so that the two species' currents do not cancel
    # to a small difference whose FP32 rounding the 1e-5 bound would measure instead
    gam, uth = (5.0, 0.05) if prec == 64 else (1.5, 0.5)
    w = wl.Workload("pic_small", 2, 64, 24, dx1=0.2, dx2=0.2, dt=0.08, precision=prec, filt_kc=0.5, filt_w=0.2,
                    shape_order=order, seed=21, kind="plasma", ppc=2, gamma=gam, u_th=uth, field_amp=0.05)
    tdt = torch.float64 if prec == 64 else torch.float32
    real = np.float64 if prec == 64 else np.float32
    E0, B0 = wl.band_limited_fields(w)
    E0 = [a.astype(real).astype(np.float64) for a in E0]
    B0 = [a.astype(real).astype(np.float64) for a in B0]
    g = hyb.Grid(hyb.desc_from_workload(w))
    E = [torch.from_numpy(a).to("cuda", tdt) for a in E0]
    B = [torch.from_numpy(a).to("cuda", tdt) for a in B0]
    J = [torch.zeros(w.shape, dtype=tdt, device="cuda") for _ in range(3)]
    g.bind(E, B, J)
    if resident:
        g.set_resident(True)
    cell, off, u, qm, q = wl.pic_plasma_torch(w, "cuda")
    ins = [t.cpu().numpy() for t in (cell, off, u, qm, q)]
    pic = hyb.Pic(g)
    pic.step(cell, off, u, qm, q, torch.empty_like(off), torch.empty_like(qm), order=order, nsteps=steps)
    g.check()
    go = orc.grid(n1=w.n1, n2=w.n2, dx1=w.dx1, dx2=w.dx2, dt=w.dt, filt_kc=w.filt_kc, filt_w=w.filt_w)
    Eo, Bo, co, oo, uo = _oracle_pic(orc, go, E0, B0, ins[0], ins[1], ins[2].astype(np.float64),
                                     ins[3].astype(np.float64), ins[4].astype(np.float64), order, w.dt,
                                     np.array([w.dx1, w.dx2]), steps)
    tol = 1e-12 if prec == 64 else 1e-5
    for a, b in zip(E + B, Eo + Bo):
        assert rel_err(a.cpu().numpy(), b) < tol
    assert np.array_equal(cell.cpu().numpy(), co)
    assert np.max(np.abs(off.cpu().numpy().astype(np.float64) - oo)) < tol
    assert np.max(np.abs(u.cpu().numpy().astype(np.float64) - uo)) < tol * np.max(np.abs(uo))
    pic.close()
    g.close()


@pytest.mark.parametrize("resident,prec,n1", [(False, 64, 64), (True, 64, 64), (False, 32, 64), (True, 32, 64),
                                               (False, 32, 512)])
def test_pic_graph_replay_matches_plain_steps(prec, resident, n1):
    """A call of several steps replays one captured step as a CUDA graph; the fields and
    particles it leaves are those of the same steps taken one call at a time (plain
    launches), also on a second call with the same arguments (the graph reused), on the
    three-pass path (n1 = 64) and on a fused grid whose halo rows are copied before each step
    (n1 = 512).  The deposit adds with atomics, so two runs agree to rounding, not bit for bit: cells
    exactly, fields and particle offsets and momenta to the parity bound."""
    need_gpu()
    hyb = hyb_module()
    w = wl.Workload("pic_graph", 2, n1, 32, dx1=0.2, dx2=0.2, dt=0.08, precision=prec, filt_kc=0.5, filt_w=0.2,
                    shape_order=2, seed=5, kind="plasma", ppc=2, gamma=3.0, u_th=0.2, field_amp=0.05)
    tdt = torch.float64 if prec == 64 else torch.float32
    E0, B0 = wl.band_limited_fields(w)
    runs = []
    for chunks in ([1] * 12, [6, 6]):
        g = hyb.Grid(hyb.desc_from_workload(w))
        E = [torch.from_numpy(a).to("cuda", tdt) for a in E0]
        B = [torch.from_numpy(a).to("cuda", tdt) for a in B0]
        J = [torch.zeros(w.shape, dtype=tdt, device="cuda") for _ in range(3)]
        g.bind(E, B, J)
        if resident:
            g.set_resident(True)
        cell, off, u, qm, q = wl.pic_plasma_torch(w, "cuda")
        off_new, v3 = torch.empty_like(off), torch.empty_like(qm)
        pic = hyb.Pic(g)
        for k in chunks:
            pic.step(cell, off, u, qm, q, off_new, v3, order=2, nsteps=k)
        g.check()
        torch.cuda.synchronize()
        runs.append([t.cpu().numpy().copy() for t in E + B + [cell, off, u]])
        pic.close()
        g.close()
    tol = 1e-12 if prec == 64 else 1e-5
    for a, b in zip(runs[0][:6], runs[1][:6]):
        assert rel_err(a, b.astype(np.float64)) < tol
    assert np.array_equal(runs[0][6], runs[1][6])
    for a, b in zip(runs[0][7:], runs[1][7:]):
        assert np.max(np.abs(a.astype(np.float64) - b)) < tol * max(1.0, float(np.max(np.abs(b))))
