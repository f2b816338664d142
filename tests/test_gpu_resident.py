"""k1-resident fields (hyb_set_resident): E and B stay in k1 space between
steps and only j is transformed, with the real-space arrays as the output the
particles gather from.  Checked against the FP64 oracle step by step with a new
current every step, on the fused-path grid size (which then runs the
three-pass kernels), the n1 = 1024 FP32 rows (Ampere fused into the inverse,
storing the E spectra back), 3D, FP64 and the DFT-GEMM transform; plus the
state semantics (the real arrays are an output; setting resident again
re-imports them) and the standalone current calls between resident steps."""
import numpy as np
import pytest

from paper_1502_01376_gb300 import workloads as wl

from gpu_util import hyb_module, need_gpu, orc_grid, rel_err, to_dev, to_np, torch

pytestmark = pytest.mark.gpu

CASES = [
    # (dims, n1, n2, n3, precision, path, tol)
    (2, 4096, 24, 1, 32, 0, 1e-5),
    (2, 1024, 32, 1, 32, 1, 1e-5),
    (3, 1024, 8, 6, 32, 1, 1e-5),
    (2, 256, 20, 1, 64, 1, 1e-12),
    (3, 64, 6, 5, 64, 1, 1e-12),
    (2, 64, 16, 1, 32, 3, 1e-4),     # DFT-GEMM transform: the split-BF16 error bound of its own tests
    (3, 32, 8, 6, 32, 4, 1e-5),      # DFT-GEMM with three BF16 parts
]


def _grid(hyb, dims, n1, n2, n3, prec, path, seed):
    w = wl.Workload("res", dims, n1, n2, n3, dx1=0.2, dx2=0.25, dx3=0.3, dt=0.06, precision=prec,
                    filt_kc=0.6, filt_w=0.2, seed=seed)
    dt = torch.float64 if prec == 64 else torch.float32
    g = hyb.Grid(hyb.desc_from_workload(w, path=path))
    E0, B0 = wl.band_limited_fields(w)
    rnd = (lambda a: a) if prec == 64 else (lambda a: a.astype(np.float32).astype(np.float64))
    E = [to_dev(a, dt) for a in E0]
    B = [to_dev(a, dt) for a in B0]
    J = [torch.zeros(w.shape, device="cuda", dtype=dt) for _ in range(3)]
    g.bind(E, B, J)
    return w, g, E, B, J, [rnd(a) for a in E0], [rnd(a) for a in B0], rnd, dt


@pytest.mark.parametrize("dims,n1,n2,n3,prec,path,tol", CASES)
def test_resident_steps_match_oracle(orc, dims, n1, n2, n3, prec, path, tol):
    need_gpu()
    hyb = hyb_module()
    w, g, E, B, J, Eo, Bo, rnd, dt = _grid(hyb, dims, n1, n2, n3, prec, path, seed=21)
    g.set_resident(True)
    assert g.step_kernel.startswith("k1-resident")
    go = orc_grid(orc, w)
    rng = np.random.default_rng(22)
    for n in range(6):                        # a new current every step, as a deposit gives
        Jn = [rnd(rng.standard_normal(w.shape) * 1e-3) for _ in range(3)]
        for c in range(3):
            J[c].copy_(to_dev(Jn[c], dt))
        g.advance(1)
        orc.step(go, Eo, Bo, Jn)
        errs = [rel_err(to_np(a), b) for a, b in zip(E + B, Eo + Bo)]
        assert max(errs) < tol, (n, errs)
    g.check()
    g.close()


@pytest.mark.parametrize("n1", [4096, 1024])
def test_resident_state_semantics(orc, n1):
    """The bound real arrays are the output of a resident step, not its input: overwriting
    them changes nothing until hyb_set_resident is called again, which re-imports them.
    hyb_correct_current and hyb_filter between steps leave the state alone."""
    need_gpu()
    hyb = hyb_module()
    w, g, E, B, J, Eo, Bo, rnd, dt = _grid(hyb, 2, n1, 16, 1, 32, 0, seed=31)
    g.set_resident(True)
    go = orc_grid(orc, w)
    rng = np.random.default_rng(32)
    Jn = [rnd(rng.standard_normal(w.shape) * 1e-3) for _ in range(3)]
    for c in range(3):
        J[c].copy_(to_dev(Jn[c], dt))
    g.advance(2)
    orc.step(go, Eo, Bo, Jn, nsteps=2)
    # overwrite the real-space view: the next steps continue from the k1-space state
    for t in E + B:
        t.zero_()
    g.advance(2)
    orc.step(go, Eo, Bo, Jn, nsteps=2)
    errs = [rel_err(to_np(a), b) for a, b in zip(E + B, Eo + Bo)]
    assert max(errs) < 1e-5, errs
    # the standalone current calls use the j part of the scratch only
    g.correct_current()
    g.filter()
    Jp = [a.copy() for a in Jn]
    orc.process_current(go, Jp, True, False)
    orc.process_current(go, Jp, False, True)
    assert max(rel_err(to_np(a), b) for a, b in zip(J, Jp)) < 1e-5
    Jp = [rnd(to_np(a)) for a in J]
    g.advance(1)
    orc.step(go, Eo, Bo, Jp)
    errs = [rel_err(to_np(a), b) for a, b in zip(E + B, Eo + Bo)]
    assert max(errs) < 1e-5, errs
    # new real-space fields, imported by setting the grid resident again
    E1, B1 = wl.band_limited_fields(wl.Workload("res2", 2, n1, 16, dx1=0.2, dx2=0.25, dt=0.06, precision=32,
                                                  filt_kc=0.6, filt_w=0.2, seed=33))
    for t, a in zip(E + B, E1 + B1):
        t.copy_(to_dev(a, dt))
    Eo, Bo = [rnd(a) for a in E1], [rnd(a) for a in B1]
    g.set_resident(True)
    g.advance(3)
    orc.step(go, Eo, Bo, Jp, nsteps=3)
    errs = [rel_err(to_np(a), b) for a, b in zip(E + B, Eo + Bo)]
    assert max(errs) < 1e-5, errs
    # and back to the normal path, which reads the real arrays again
    g.set_resident(False)
    assert not g.step_kernel.startswith("k1-resident")
    g.advance(1)
    orc.step(go, Eo, Bo, Jp)
    errs = [rel_err(to_np(a), b) for a, b in zip(E + B, Eo + Bo)]
    assert max(errs) < 1e-5, errs
    g.close()


def test_resident_host_step_imports_the_host_fields(orc):
    """hyb_advance_host on a resident grid takes E, B from the host arrays (an import step)."""
    need_gpu()
    hyb = hyb_module()
    w, g, E, B, J, Eo, Bo, rnd, dt = _grid(hyb, 2, 1024, 12, 1, 32, 0, seed=41)
    g.set_resident(True)
    g.advance(2)                              # some state that the host step must not reuse
    rng = np.random.default_rng(42)
    Jn = [rnd(rng.standard_normal(w.shape) * 1e-3) for _ in range(3)]
    H = [torch.from_numpy(a.astype(np.float32)).pin_memory() for a in Eo + Bo + Jn]
    g.advance_host(H[0:3], H[3:6], H[6:9], 2)
    go = orc_grid(orc, w)
    orc.step(go, Eo, Bo, Jn, nsteps=2)
    errs = [rel_err(a.numpy(), b) for a, b in zip(H[:6], Eo + Bo)]
    assert max(errs) < 1e-5, errs
    g.close()


def test_resident_rejects_quasi3d():
    need_gpu()
    hyb = hyb_module()
    g = hyb.Grid(hyb.make_desc(dims=20, n1=64, n2=16, dx1=0.2, dx2=0.2, dt=0.05, precision=32, azimuthal_m=1))
    with pytest.raises(hyb.HybError):
        g.set_resident(True)
    g.close()
