"""Thin ctypes binding of libhyb.so (C ABI: include/hyb.h).

Argument marshalling only: every step of the hybrid advance, the deposit and
the diagnostics runs in the library's CUDA kernels.  PyTorch supplies device
memory and the current stream.  There is no CPU fallback: if the library is
missing or cannot load, ``lib()`` raises.

Module-level functions carry the C names (``hyb_create_grid``, ...); ``Grid``
wraps them for tensors.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhyb.so")

HYB_OK, HYB_EINVAL, HYB_ECOURANT, HYB_EALIGN, HYB_ECUDA, HYB_ETIMEOUT, HYB_ESTATE, HYB_ENOMEM, HYB_EDATA = range(9)
STATUS_NAMES = ["HYB_OK", "HYB_EINVAL", "HYB_ECOURANT", "HYB_EALIGN", "HYB_ECUDA", "HYB_ETIMEOUT",
                "HYB_ESTATE", "HYB_ENOMEM", "HYB_EDATA"]


class HybError(RuntimeError):
    def __init__(self, status: int, msg: str):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{name}: {msg}")


class GridDesc(ctypes.Structure):
    _fields_ = [
        ("dims", ctypes.c_int),
        ("n1", ctypes.c_int), ("n2", ctypes.c_int), ("n3", ctypes.c_int),
        ("dx1", ctypes.c_double), ("dx2", ctypes.c_double), ("dx3", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("precision", ctypes.c_int),
        ("correct_j1", ctypes.c_int),
        ("filt_kc", ctypes.c_double), ("filt_w", ctypes.c_double),
        ("kmod_l", ctypes.c_double), ("kmod_u", ctypes.c_double), ("kmod_max", ctypes.c_double),
        ("yee_mode", ctypes.c_int),
        ("ampere", ctypes.c_double),
        ("path", ctypes.c_int),
        ("azimuthal_m", ctypes.c_int),
    ]


_lib = None
_lock = threading.Lock()
_V = ctypes.c_void_p
_P3 = ctypes.c_void_p * 3


def lib():
    """Load libhyb.so (build it first with paper_1502_01376_gb300.build)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError(f"{LIB_PATH} is missing: run paper_1502_01376_gb300/build.py "
                                  "(there is no CPU fallback)")
            L = ctypes.CDLL(LIB_PATH)
            S = ctypes.c_int
            D = ctypes.POINTER(GridDesc)
            L.hyb_courant_limit.argtypes = [D]
            L.hyb_courant_limit.restype = ctypes.c_double
            L.hyb_create_grid.argtypes = [D, _V, ctypes.POINTER(_V)]
            L.hyb_create_grid.restype = S
            L.hyb_set_stream.argtypes = [_V, _V]
            L.hyb_set_stream.restype = S
            L.hyb_bind_fields.argtypes = [_V, _P3, _P3, _P3, _V]
            L.hyb_bind_fields.restype = S
            L.hyb_deposit.argtypes = [_V, _V, _V, _V, _V, _V, ctypes.c_int64, ctypes.c_int]
            L.hyb_deposit.restype = S
            L.hyb_push.argtypes = [_V, _V, _V, _V, _V, _V, _V, ctypes.c_int64, ctypes.c_int]
            L.hyb_push.restype = S
            for fn in ("hyb_correct_current", "hyb_filter", "hyb_check", "hyb_destroy_grid"):
                getattr(L, fn).argtypes = [_V]
                getattr(L, fn).restype = S
            L.hyb_advance.argtypes = [_V, ctypes.c_int]
            L.hyb_advance.restype = S
            L.hyb_advance_host.argtypes = [_V, _P3, _P3, _P3, ctypes.c_int]
            L.hyb_advance_host.restype = S
            L.hyb_diag.argtypes = [_V, ctypes.POINTER(ctypes.c_double)]
            L.hyb_diag.restype = S
            L.hyb_last_error.argtypes = []
            L.hyb_last_error.restype = ctypes.c_char_p
            L.hyb_grid_path.argtypes = [_V]
            L.hyb_grid_path.restype = ctypes.c_int
            L.hyb_set_kernel_events.argtypes = [_V, _V, _V]
            L.hyb_set_kernel_events.restype = S
            L.hyb_batch_create.argtypes = [D, ctypes.c_int, _V, ctypes.POINTER(_V)]
            L.hyb_batch_create.restype = S
            L.hyb_batch_bind.argtypes = [_V, ctypes.c_int, _P3, _P3, _P3]
            L.hyb_batch_bind.restype = S
            L.hyb_batch_tune.argtypes = [_V, ctypes.c_int]
            L.hyb_batch_tune.restype = S
            L.hyb_batch_advance.argtypes = [_V, ctypes.c_int]
            L.hyb_batch_advance.restype = S
            L.hyb_batch_rows_per_strip.argtypes = [_V, ctypes.c_int]
            L.hyb_batch_rows_per_strip.restype = ctypes.c_int
            L.hyb_batch_set_rows_per_strip.argtypes = [_V, ctypes.c_int, ctypes.c_int]
            L.hyb_batch_set_rows_per_strip.restype = ctypes.c_int
            L.hyb_batch_launches_per_step.argtypes = [_V]
            L.hyb_batch_launches_per_step.restype = ctypes.c_int
            L.hyb_batch_set_single_launch.argtypes = [_V, ctypes.c_int]
            L.hyb_batch_set_single_launch.restype = S
            L.hyb_batch_check.argtypes = [_V]
            L.hyb_batch_check.restype = S
            L.hyb_batch_single_launch.argtypes = [_V]
            L.hyb_batch_single_launch.restype = ctypes.c_int
            L.hyb_batch_role_ctas.argtypes = [_V, ctypes.c_int]
            L.hyb_batch_role_ctas.restype = ctypes.c_int
            L.hyb_batch_set_role_ctas.argtypes = [_V, ctypes.POINTER(ctypes.c_int)]
            L.hyb_batch_set_role_ctas.restype = S
            L.hyb_batch_role_ms.argtypes = [_V, ctypes.c_int]
            L.hyb_batch_role_ms.restype = ctypes.c_double
            L.hyb_batch_destroy.argtypes = [_V]
            L.hyb_batch_destroy.restype = S
            L.hyb_correct_current_noalloc.argtypes = [D, _V, _V]
            L.hyb_correct_current_noalloc.restype = S
            L.hyb_nci_growth.argtypes = [_V, ctypes.c_int64, ctypes.c_int, ctypes.c_int, _V, ctypes.c_int, _V, _V, _V]
            L.hyb_nci_growth.restype = S
            L.hyb_nci_roots.argtypes = [_V, ctypes.c_int64, ctypes.c_int, ctypes.c_int, _V, ctypes.c_int, ctypes.c_int,
                                        _V, _V, _V, _V, _V]
            L.hyb_nci_roots.restype = S
            L.hyb_pic_create.argtypes = [_V, ctypes.POINTER(_V)]
            L.hyb_pic_create.restype = S
            L.hyb_pic_step.argtypes = [_V, _V, _V, _V, _V, _V, _V, _V, ctypes.c_int64, ctypes.c_int, ctypes.c_int]
            L.hyb_pic_step.restype = S
            L.hyb_pic_destroy.argtypes = [_V]
            L.hyb_pic_destroy.restype = S
            L.hyb_mlp_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _V, ctypes.POINTER(_V)]
            L.hyb_mlp_create.restype = S
            L.hyb_mlp_num_params.argtypes = [_V]
            L.hyb_mlp_num_params.restype = ctypes.c_int64
            for fn in ("hyb_mlp_set_params", "hyb_mlp_get_params"):
                getattr(L, fn).argtypes = [_V, _V]
                getattr(L, fn).restype = S
            L.hyb_mlp_forward.argtypes = [_V, _V, ctypes.c_int64, _V, _V]
            L.hyb_mlp_forward.restype = S
            L.hyb_mlp_gradients.argtypes = [_V, _V, _V, ctypes.c_int64, _V, _V, _V]
            L.hyb_mlp_gradients.restype = S
            L.hyb_mlp_train_step.argtypes = [_V, _V, _V, ctypes.c_int64, ctypes.c_float, _V, _V]
            L.hyb_mlp_train_step.restype = S
            L.hyb_mlp_destroy.argtypes = [_V]
            L.hyb_mlp_destroy.restype = S
            L.hyb_mlp_launch_count.argtypes = [_V]
            L.hyb_mlp_launch_count.restype = ctypes.c_int64
            L.hyb_set_resident.argtypes = [_V, ctypes.c_int]
            L.hyb_set_resident.restype = ctypes.c_int
            L.hyb_step_kernel.argtypes = [_V]
            L.hyb_step_kernel.restype = ctypes.c_char_p
            L.hyb_launches_per_step.argtypes = [_V]
            L.hyb_launches_per_step.restype = ctypes.c_int
            L.hyb_wait_selftest.argtypes = [ctypes.c_int, ctypes.c_double, _V]
            L.hyb_wait_selftest.restype = S
            _lib = L
    return _lib


def _check(st: int):
    if st != HYB_OK:
        raise HybError(st, lib().hyb_last_error().decode())


def make_desc(dims=2, n1=128, n2=64, n3=1, dx1=0.1, dx2=0.1, dx3=0.1, dt=0.05, precision=64,
              correct_j1=True, filt_kc=0.0, filt_w=0.0, kmod_l=0.0, kmod_u=0.0, kmod_max=0.0,
              yee_mode=False, ampere=0.0, path=0, azimuthal_m=0) -> GridDesc:
    return GridDesc(dims, n1, n2, n3, dx1, dx2, dx3, dt, precision, int(bool(correct_j1)), filt_kc, filt_w,
                    kmod_l, kmod_u, kmod_max, int(bool(yee_mode)), ampere, path, azimuthal_m)


def desc_from_workload(w, **over) -> GridDesc:
    kw = dict(dims=w.dims, n1=w.n1, n2=w.n2, n3=w.n3, dx1=w.dx1, dx2=w.dx2, dx3=w.dx3, dt=w.dt,
              precision=w.precision, correct_j1=w.correct_j1, filt_kc=w.filt_kc, filt_w=w.filt_w)
    kw.update(over)
    return make_desc(**kw)


# ---- C-named thin wrappers ---------------------------------------------------
def hyb_courant_limit(desc: GridDesc) -> float:
    return lib().hyb_courant_limit(ctypes.byref(desc))


def hyb_create_grid(desc: GridDesc, stream: int = 0) -> int:
    h = _V()
    _check(lib().hyb_create_grid(ctypes.byref(desc), _V(stream), ctypes.byref(h)))
    return h.value


def hyb_set_stream(g: int, stream: int):
    _check(lib().hyb_set_stream(_V(g), _V(stream)))


def hyb_bind_fields(g: int, E, B, J, rho=0):
    _check(lib().hyb_bind_fields(_V(g), _P3(*E), _P3(*B), _P3(*J), _V(rho or 0)))


def hyb_deposit(g: int, cell: int, off_old: int, off_new: int, v3: int, q: int, np_: int, order: int):
    _check(lib().hyb_deposit(_V(g), _V(cell), _V(off_old), _V(off_new), _V(v3 or 0), _V(q), np_, order))


def hyb_push(g: int, cell: int, off: int, u: int, qm: int, off_new: int, v3: int, np_: int, order: int):
    _check(lib().hyb_push(_V(g), _V(cell), _V(off), _V(u), _V(qm), _V(off_new), _V(v3 or 0), np_, order))


def hyb_correct_current(g: int):
    _check(lib().hyb_correct_current(_V(g)))


def hyb_correct_current_noalloc(desc: GridDesc, j1: int, stream: int = 0):
    """j1 correction without any device allocation (working memory is a
    static array of the library); for callers that cannot allocate."""
    _check(lib().hyb_correct_current_noalloc(ctypes.byref(desc), _V(j1), _V(stream)))


def hyb_filter(g: int):
    _check(lib().hyb_filter(_V(g)))


def hyb_advance(g: int, nsteps: int):
    _check(lib().hyb_advance(_V(g), nsteps))


def hyb_advance_host(g: int, E, B, J, nsteps: int):
    _check(lib().hyb_advance_host(_V(g), _P3(*E), _P3(*B), _P3(*J), nsteps))


def hyb_diag(g: int) -> np.ndarray:
    out = (ctypes.c_double * 9)()
    _check(lib().hyb_diag(_V(g), out))
    return np.array(list(out))


def hyb_check(g: int):
    _check(lib().hyb_check(_V(g)))


def hyb_wait_selftest(which: int, seconds: float, stream: int = 0) -> int:
    """Status of the bounded-wait self-test (HYB_ETIMEOUT is the designed outcome)."""
    return lib().hyb_wait_selftest(int(which), float(seconds), _V(stream))


def hyb_destroy_grid(g: int):
    _check(lib().hyb_destroy_grid(_V(g)))


def hyb_last_error() -> str:
    return lib().hyb_last_error().decode()


def hyb_set_kernel_events(g: int, start: int, stop: int):
    _check(lib().hyb_set_kernel_events(_V(g), _V(start), _V(stop)))


def hyb_grid_path(g: int) -> int:
    return lib().hyb_grid_path(_V(g))


def hyb_step_kernel(g: int) -> str:
    return lib().hyb_step_kernel(_V(g)).decode()


def hyb_launches_per_step(g: int) -> int:
    return lib().hyb_launches_per_step(_V(g))


def hyb_batch_create(descs, stream: int = 0) -> int:
    arr = (GridDesc * len(descs))(*descs)
    h = _V()
    _check(lib().hyb_batch_create(arr, len(descs), _V(stream), ctypes.byref(h)))
    return h.value


def hyb_batch_bind(b: int, i: int, E, B, J):
    _check(lib().hyb_batch_bind(_V(b), i, _P3(*E), _P3(*B), _P3(*J)))


def hyb_batch_tune(b: int, trials: int = 3):
    _check(lib().hyb_batch_tune(_V(b), trials))


def hyb_batch_advance(b: int, nsteps: int):
    _check(lib().hyb_batch_advance(_V(b), nsteps))


def hyb_batch_rows_per_strip(b: int, n1: int) -> int:
    return lib().hyb_batch_rows_per_strip(_V(b), n1)


def hyb_batch_set_rows_per_strip(b: int, n1: int, h: int) -> None:
    _check(lib().hyb_batch_set_rows_per_strip(_V(b), n1, h))


def hyb_batch_launches_per_step(b: int) -> int:
    return lib().hyb_batch_launches_per_step(_V(b))


def hyb_batch_set_single_launch(b: int, on: bool) -> None:
    _check(lib().hyb_batch_set_single_launch(_V(b), 1 if on else 0))


def hyb_batch_check(b: int) -> None:
    _check(lib().hyb_batch_check(_V(b)))


def hyb_batch_single_launch(b: int) -> bool:
    return lib().hyb_batch_single_launch(_V(b)) != 0


def hyb_batch_role_ctas(b: int, r: int) -> int:
    return lib().hyb_batch_role_ctas(_V(b), r)


def hyb_batch_set_role_ctas(b: int, ctas) -> None:
    arr = (ctypes.c_int * 5)(*[int(c) for c in ctas])
    _check(lib().hyb_batch_set_role_ctas(_V(b), arr))


def hyb_batch_role_ms(b: int, r: int) -> float:
    return lib().hyb_batch_role_ms(_V(b), r)


def hyb_batch_destroy(b: int):
    _check(lib().hyb_batch_destroy(_V(b)))


def hyb_nci_growth(samples: int, n: int, order: int, correct_j1: bool, alias: int, n_alias: int,
                   growth: int, root: int = 0, stream: int = 0):
    _check(lib().hyb_nci_growth(_V(samples), n, order, int(bool(correct_j1)), _V(alias), n_alias,
                                _V(growth), _V(root or 0), _V(stream)))


NCI_ROW = 12     # dt, dx1, dx2, gamma, wp2, filt_kc, filt_w, k1, k2, kmod_l, kmod_u, kmod_max


def hyb_nci_roots(samples: int, n: int, order: int, correct_j1: bool, alias: int, n_alias: int, max_roots: int,
                  roots: int, count: int, growth: int, err: int = 0, stream: int = 0):
    _check(lib().hyb_nci_roots(_V(samples), n, order, int(bool(correct_j1)), _V(alias), n_alias, max_roots,
                               _V(roots), _V(count), _V(growth), _V(err or 0), _V(stream)))


def nci_rows(samples):
    """[n, 9] (no k1 modification) or [n, 12] float64 CUDA rows -> contiguous [n, 12]."""
    import torch
    assert samples.is_cuda and samples.dtype == torch.float64 and samples.shape[1] in (9, NCI_ROW)
    if samples.shape[1] == 9:
        samples = torch.cat([samples, torch.zeros((samples.shape[0], 3), dtype=samples.dtype,
                                                  device=samples.device)], dim=1)
    return samples.contiguous()


def nci_growth(samples, aliases=((0, -1), (0, 0), (0, 1)), order=2, correct_j1=True, want_roots=False):
    """samples: CUDA float64 tensor [n, 9] or [n, 12]; returns growth [n, n_alias]
    (and the growing roots [n, n_alias] complex)."""
    import torch
    samples = nci_rows(samples)
    n = samples.shape[0]
    al = torch.tensor(list(aliases), dtype=torch.int32, device=samples.device).contiguous()
    g = torch.empty((n, len(aliases)), dtype=torch.float64, device=samples.device)
    r = torch.empty((n, len(aliases), 2), dtype=torch.float64, device=samples.device) if want_roots else None
    hyb_nci_growth(int(samples.data_ptr()), n, order, correct_j1, int(al.data_ptr()), len(aliases),
                   int(g.data_ptr()), int(r.data_ptr()) if r is not None else 0,
                   torch.cuda.current_stream().cuda_stream)
    if want_roots:
        return g, torch.view_as_complex(r)
    return g


def nci_roots(samples, aliases=((0, -1), (0, 0), (0, 1)), order=2, correct_j1=True, max_roots=16):
    """All roots in each alias's disk: (roots [n, n_alias, max_roots] complex, count [n, n_alias],
    growth [n, n_alias], err flags)."""
    import torch
    samples = nci_rows(samples)
    n = samples.shape[0]
    dev = samples.device
    al = torch.tensor(list(aliases), dtype=torch.int32, device=dev).contiguous()
    r = torch.zeros((n, len(aliases), max_roots, 2), dtype=torch.float64, device=dev)
    c = torch.zeros((n, len(aliases)), dtype=torch.int32, device=dev)
    g = torch.empty((n, len(aliases)), dtype=torch.float64, device=dev)
    e = torch.zeros(1, dtype=torch.int32, device=dev)
    hyb_nci_roots(int(samples.data_ptr()), n, order, correct_j1, int(al.data_ptr()), len(aliases), max_roots,
                  int(r.data_ptr()), int(c.data_ptr()), int(g.data_ptr()), int(e.data_ptr()),
                  torch.cuda.current_stream().cuda_stream)
    return torch.view_as_complex(r), c, g, int(e.item())


# ---- tensor convenience ----------------------------------------------------------
def _ptr(t):
    return 0 if t is None else int(t.data_ptr())


class Grid:
    """A grid bound to torch CUDA tensors E, B, J (lists of 3) and optional rho."""

    def __init__(self, desc: GridDesc, stream=None):
        import torch
        self.desc = desc
        self.torch = torch
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.h = hyb_create_grid(desc, self.stream.cuda_stream)
        if desc.dims == 20:
            self.dtype = torch.complex64 if desc.precision == 32 else torch.complex128
        else:
            self.dtype = torch.float32 if desc.precision == 32 else torch.float64
        self.tensors = None

    @property
    def shape(self):
        d = self.desc
        return (d.n3, d.n2, d.n1) if d.dims == 3 else (d.n2, d.n1)

    def _chk(self, t):
        assert t.is_cuda and t.dtype == self.dtype and t.is_contiguous() and tuple(t.shape) == self.shape, \
            (t.device, t.dtype, tuple(t.shape), self.shape)

    def bind(self, E, B, J, rho=None):
        for t in list(E) + list(B) + list(J) + ([rho] if rho is not None else []):
            self._chk(t)
        self.tensors = (list(E), list(B), list(J), rho)
        hyb_bind_fields(self.h, [_ptr(t) for t in E], [_ptr(t) for t in B], [_ptr(t) for t in J], _ptr(rho))
        return self

    def deposit(self, cell, off_old, off_new, v3, q, order):
        n = q.numel()
        hyb_deposit(self.h, _ptr(cell), _ptr(off_old), _ptr(off_new), _ptr(v3), _ptr(q), n, order)

    def push(self, cell, off, u, qm, off_new, v3=None, order=2):
        """Gather and Boris push (hyb_push): cell, off, u updated in place; off_new (and v3) written."""
        hyb_push(self.h, _ptr(cell), _ptr(off), _ptr(u), _ptr(qm), _ptr(off_new), _ptr(v3), qm.numel(), order)

    def correct_current(self):
        hyb_correct_current(self.h)

    def filter(self):
        hyb_filter(self.h)

    def advance(self, nsteps=1):
        hyb_advance(self.h, nsteps)

    def advance_host(self, E, B, J, nsteps=1):
        """E, B, J: pinned CPU tensors of the grid's dtype (E, B updated in place)."""
        hyb_advance_host(self.h, [_ptr(t) for t in E], [_ptr(t) for t in B], [_ptr(t) for t in J], nsteps)

    def diag(self):
        return hyb_diag(self.h)

    def check(self):
        hyb_check(self.h)

    def set_kernel_events(self, start=None, stop=None):
        """torch.cuda.Event pair (created with enable_timing=True and recorded
        once, so that the CUDA event exists) or None."""
        hyb_set_kernel_events(self.h, start.cuda_event if start is not None else 0,
                              stop.cuda_event if stop is not None else 0)

    @property
    def path(self):
        return hyb_grid_path(self.h)

    @property
    def launches_per_step(self):
        return hyb_launches_per_step(self.h)

    @property
    def step_kernel(self):
        return hyb_step_kernel(self.h)

    def set_resident(self, on=True):
        """k1-resident E, B between steps (hyb_set_resident); calling it again with on=True
        re-imports the bound real-space fields at the next step."""
        _check(lib().hyb_set_resident(_V(self.h), 1 if on else 0))

    def close(self):
        if self.h:
            hyb_destroy_grid(self.h)
            self.h = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Pic:
    """The particle-in-cell loop around a bound Grid (hyb_pic_*): push, deposit and
    advance per step, B time-centred for the push."""

    def __init__(self, grid: Grid):
        h = _V()
        _check(lib().hyb_pic_create(_V(grid.h), ctypes.byref(h)))
        self.h = h.value
        self.grid = grid

    def step(self, cell, off, u, qm, q, off_new, v3, order=2, nsteps=1):
        _check(lib().hyb_pic_step(_V(self.h), _V(_ptr(cell)), _V(_ptr(off)), _V(_ptr(u)), _V(_ptr(qm)), _V(_ptr(q)),
                                  _V(_ptr(off_new)), _V(_ptr(v3)), qm.numel(), order, nsteps))

    def close(self):
        if self.h:
            lib().hyb_pic_destroy(_V(self.h))
            self.h = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Several grids advanced together (one CUDA-graph launch per step)."""

    def __init__(self, descs, stream=None):
        import torch
        self.descs = list(descs)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.h = hyb_batch_create(self.descs, self.stream.cuda_stream)
        self.bound = {}

    def bind(self, i, E, B, J):
        self.bound[i] = (list(E), list(B), list(J))
        hyb_batch_bind(self.h, i, [_ptr(t) for t in E], [_ptr(t) for t in B], [_ptr(t) for t in J])

    def tune(self, trials=3):
        hyb_batch_tune(self.h, trials)

    def advance(self, nsteps=1):
        hyb_batch_advance(self.h, nsteps)

    def set_rows_per_strip(self, n1, h):
        hyb_batch_set_rows_per_strip(self.h, n1, h)

    def rows_per_strip(self, n1):
        return hyb_batch_rows_per_strip(self.h, n1)

    @property
    def launches_per_step(self):
        return hyb_batch_launches_per_step(self.h)

    def check(self):
        """Raises if a device-side wait of a step gave up (or a deposit skipped particles)."""
        hyb_batch_check(self.h)

    @property
    def single_launch(self):
        """True if a step is one persistent launch (False: a graph of launches)."""
        return hyb_batch_single_launch(self.h)

    @single_launch.setter
    def single_launch(self, on):
        hyb_batch_set_single_launch(self.h, on)

    def role_ctas(self):
        """CTAs of the single launch's roles: n1 = 4096, 512, 1024, 2048, quasi-3D."""
        return [hyb_batch_role_ctas(self.h, r) for r in range(5)]

    def set_role_ctas(self, ctas):
        """Sets the CTAs of the single launch's roles (as role_ctas() lists them)."""
        hyb_batch_set_role_ctas(self.h, ctas)

    def role_ms(self):
        """Each role's duration in the tuner's fastest single launch (ms)."""
        return [hyb_batch_role_ms(self.h, r) for r in range(5)]

    def close(self):
        if self.h:
            hyb_batch_destroy(self.h)
            self.h = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mlp_init_params(n_in: int, width: int, depth: int, seed: int = 0) -> np.ndarray:
    """Seeded Xavier-uniform weights, zero biases, in the library's layout."""
    rng = np.random.default_rng(seed)
    dims = [n_in] + [width] * depth + [1]
    parts = []
    for i in range(depth + 1):
        fi, fo = dims[i], dims[i + 1]
        lim = np.sqrt(6.0 / (fi + fo))
        parts.append(rng.uniform(-lim, lim, (fo, fi)).ravel())
        parts.append(np.zeros(fo))
    return np.concatenate(parts).astype(np.float32)


class MLP:
    """The NCI surrogate network (forward, backward and Adam in libhyb.so)."""

    def __init__(self, n_in=6, width=256, depth=4, params=None, seed=0):
        self.n_in, self.width, self.depth = n_in, width, depth
        p = mlp_init_params(n_in, width, depth, seed) if params is None else np.ascontiguousarray(params, dtype=np.float32)
        h = _V()
        _check(lib().hyb_mlp_create(n_in, width, depth, p.ctypes.data_as(_V), ctypes.byref(h)))
        self.h = h.value
        self.n_params = lib().hyb_mlp_num_params(_V(self.h))
        assert self.n_params == p.size

    def get_params(self) -> np.ndarray:
        out = np.zeros(self.n_params, dtype=np.float32)
        _check(lib().hyb_mlp_get_params(_V(self.h), out.ctypes.data_as(_V)))
        return out

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        _check(lib().hyb_mlp_set_params(_V(self.h), p.ctypes.data_as(_V)))

    def forward(self, x):
        import torch
        x = x.contiguous()
        y = torch.empty(x.shape[0], dtype=torch.float32, device=x.device)
        _check(lib().hyb_mlp_forward(_V(self.h), _V(int(x.data_ptr())), x.shape[0], _V(int(y.data_ptr())),
                                     _V(torch.cuda.current_stream().cuda_stream)))
        return y

    def gradients(self, x, t):
        import torch
        g = np.zeros(self.n_params, dtype=np.float32)
        loss = np.zeros(1, dtype=np.float32)
        _check(lib().hyb_mlp_gradients(_V(self.h), _V(int(x.data_ptr())), _V(int(t.data_ptr())), x.shape[0],
                                       g.ctypes.data_as(_V), loss.ctypes.data_as(_V),
                                       _V(torch.cuda.current_stream().cuda_stream)))
        return g, float(loss[0])

    def launch_count(self) -> int:
        return int(lib().hyb_mlp_launch_count(_V(self.h)))

    def train_step(self, x, t, lr, loss_out=None):
        import torch
        _check(lib().hyb_mlp_train_step(_V(self.h), _V(int(x.data_ptr())), _V(int(t.data_ptr())), x.shape[0],
                                        lr, _V(int(loss_out.data_ptr()) if loss_out is not None else 0),
                                        _V(torch.cuda.current_stream().cuda_stream)))

    def close(self):
        if self.h:
            _check(lib().hyb_mlp_destroy(_V(self.h)))
            self.h = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
