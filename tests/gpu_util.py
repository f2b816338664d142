"""Helpers shared by the GPU parity tests (inputs from workloads, expected
values from the oracle; nothing here computes the method)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def hyb_module():
    from paper_1502_01376_gb300 import build, hyb
    build.build()
    return hyb


def to_dev(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype).contiguous()


def to_np(t):
    return t.detach().to("cpu", torch.float64).numpy()


def rel_err(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b.ravel())
    return np.linalg.norm((a - b).ravel()) / max(nb, 1e-30 * b.size)


def orc_grid(orc, w, **over):
    kw = dict(dims=w.dims, n1=w.n1, n2=w.n2, n3=w.n3, dx1=w.dx1, dx2=w.dx2, dx3=w.dx3, dt=w.dt,
              correct_j1=w.correct_j1, filt_kc=w.filt_kc, filt_w=w.filt_w)
    kw.update(over)
    return orc.grid(**kw)
