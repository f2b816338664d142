"""FP64 CPU oracle of the hybrid Yee-FFT field advance (arXiv:1502.01376).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py``.  The
product path (``paper_1502_01376_gb300``) never imports it and shares no code
with it.  The arithmetic lives in ``hyb_oracle.c`` (plain C, FP64, its own
textbook FFT); this module only marshals numpy arrays through ctypes.

Parity status per function (pins in ``tests/test_oracle_*.py``):
  fft / rfft / irfft   pinned: brute-force DFT, numpy.fft, round trip
  step (2D, 3D)        pinned: exact calculus of single modes (sigma+/-),
                       vacuum dispersion of Sec. 2.2, Yee recovery of Sec. 2.1,
                       Courant limit, div B and Gauss invariants of Sec. 2.3
  deposit / charge     pinned: continuity equation of Sec. 2.3, B-spline
                       moments, total current q v
  mode tables          pinned: special values of the correction and filter
  diag                 pinned through the invariants above
The sibling modules carry their own status: ``quasi3d`` (Bessel modes of a
conducting cylinder), ``nci`` (the printed cubic as the relation's expansion,
the cold-beam continuum limit, Sec. 4's printed zero growth, a brute-force root
scan), ``mlp`` (finite differences), ``push`` (B-spline
identities, exact uniform-field solutions, second-order convergence).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "liborc.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile hyb_oracle.c into liborc.so (gcc, OpenMP over independent rows)."""
    src = os.path.join(_HERE, "hyb_oracle.c")
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(src):
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", src, "-o", _LIB_PATH, "-lm"]
        subprocess.run(cmd, check=True)
    return _LIB_PATH


class OrcGrid(ctypes.Structure):
    _fields_ = [
        ("dims", ctypes.c_int),
        ("n1", ctypes.c_int), ("n2", ctypes.c_int), ("n3", ctypes.c_int),
        ("dx1", ctypes.c_double), ("dx2", ctypes.c_double), ("dx3", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("correct_j1", ctypes.c_int),
        ("filt_kc", ctypes.c_double), ("filt_w", ctypes.c_double),
        ("kmod_l", ctypes.c_double), ("kmod_u", ctypes.c_double), ("kmod_max", ctypes.c_double),
        ("yee_mode", ctypes.c_int),
        ("ampere", ctypes.c_double),
    ]


_DP = ctypes.POINTER(ctypes.c_double)
_IP = ctypes.POINTER(ctypes.c_int32)


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        G = ctypes.POINTER(OrcGrid)
        L.orc_fft.argtypes = [_DP, ctypes.c_int, ctypes.c_int]
        L.orc_rfft.argtypes = [_DP, ctypes.c_int, _DP]
        L.orc_irfft.argtypes = [_DP, ctypes.c_int, _DP]
        L.orc_mode_tables.argtypes = [G, _DP, _DP, _DP]
        L.orc_courant.argtypes = [G]
        L.orc_courant.restype = ctypes.c_double
        L.orc_step.argtypes = [G] + [_DP] * 9 + [ctypes.c_int]
        L.orc_process_current.argtypes = [G, _DP, _DP, _DP, ctypes.c_int, ctypes.c_int]
        L.orc_shape.argtypes = [ctypes.c_int, ctypes.c_double]
        L.orc_shape.restype = ctypes.c_double
        L.orc_deposit.argtypes = [G, _IP, _DP, _DP, _DP, _DP, ctypes.c_int64, ctypes.c_int, _DP, _DP, _DP]
        L.orc_charge.argtypes = [G, _IP, _DP, _DP, ctypes.c_int64, ctypes.c_int, _DP]
        L.orc_divb.argtypes = [G, _DP, _DP, _DP, _DP]
        L.orc_gauss.argtypes = [G, _DP, _DP, _DP, _DP, _DP]
        L.orc_diag.argtypes = [G] + [_DP] * 7 + [_DP]
        L.orc_num_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def _p(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_DP)


def _ip(a):
    assert a.dtype == np.int32 and a.flags.c_contiguous
    return a.ctypes.data_as(_IP)


def grid(dims=2, n1=128, n2=64, n3=1, dx1=0.1, dx2=0.1, dx3=0.1, dt=0.05, correct_j1=True,
         filt_kc=0.0, filt_w=0.0, kmod_l=0.0, kmod_u=0.0, kmod_max=0.0, yee_mode=False,
         ampere=4.0 * np.pi) -> OrcGrid:
    return OrcGrid(dims, n1, n2, n3 if dims == 3 else 1, dx1, dx2, dx3, dt, int(bool(correct_j1)),
                   filt_kc, filt_w, kmod_l, kmod_u, kmod_max, int(bool(yee_mode)), ampere)


def field_shape(g: OrcGrid):
    return (g.n3, g.n2, g.n1) if g.dims == 3 else (g.n2, g.n1)


# ---------------------------------------------------------------------------
def fft(z: np.ndarray, inverse: bool = False) -> np.ndarray:
    """Complex DFT (unnormalised, sign -1 forward / +1 inverse)."""
    z = np.ascontiguousarray(z, dtype=np.complex128).copy()
    lib().orc_fft(z.view(np.float64).ctypes.data_as(_DP), z.size, +1 if inverse else -1)
    return z


def rfft(x: np.ndarray) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = np.zeros(x.size // 2 + 1, dtype=np.complex128)
    lib().orc_rfft(_p(x), x.size, out.view(np.float64).ctypes.data_as(_DP))
    return out


def irfft(X: np.ndarray, n: int) -> np.ndarray:
    X = np.ascontiguousarray(X, dtype=np.complex128)
    out = np.zeros(n, dtype=np.float64)
    lib().orc_irfft(X.view(np.float64).ctypes.data_as(_DP), n, _p(out))
    return out


def mode_tables(g: OrcGrid):
    nk = g.n1 // 2 + 1
    keff, corr, filt = (np.zeros(nk) for _ in range(3))
    lib().orc_mode_tables(ctypes.byref(g), _p(keff), _p(corr), _p(filt))
    return keff, corr, filt


def courant(g: OrcGrid) -> float:
    return lib().orc_courant(ctypes.byref(g))


def step(g: OrcGrid, E, B, J, nsteps: int = 1):
    """Advance (E^n, B^{n-1/2}) by nsteps with current J (in place)."""
    rc = lib().orc_step(ctypes.byref(g), *[_p(a) for a in E], *[_p(a) for a in B], *[_p(a) for a in J], nsteps)
    if rc != 0:
        raise RuntimeError(f"orc_step failed ({rc})")


def process_current(g: OrcGrid, J, correct: bool, filt: bool):
    lib().orc_process_current(ctypes.byref(g), *[_p(a) for a in J], int(correct), int(filt))


def shape(order: int, d: float) -> float:
    return lib().orc_shape(order, d)


def deposit(g: OrcGrid, cell, off_old, off_new, v3, q, order: int):
    shp = field_shape(g)
    J = [np.zeros(shp) for _ in range(3)]
    np_ = q.size
    lib().orc_deposit(ctypes.byref(g), _ip(cell), _p(off_old), _p(off_new), _p(v3), _p(q), np_, order,
                      *[_p(a) for a in J])
    return J


def charge(g: OrcGrid, cell, off, q, order: int):
    rho = np.zeros(field_shape(g))
    lib().orc_charge(ctypes.byref(g), _ip(cell), _p(off), _p(q), q.size, order, _p(rho))
    return rho


def divb(g: OrcGrid, B):
    out = np.zeros(field_shape(g))
    lib().orc_divb(ctypes.byref(g), *[_p(a) for a in B], _p(out))
    return out


def gauss(g: OrcGrid, E, rho=None):
    out = np.zeros(field_shape(g))
    lib().orc_gauss(ctypes.byref(g), *[_p(a) for a in E], _p(rho), _p(out))
    return out


def diag(g: OrcGrid, E, B, rho=None):
    out = np.zeros(9)
    lib().orc_diag(ctypes.byref(g), *[_p(a) for a in E], *[_p(a) for a in B], _p(rho), _p(out))
    return out


def num_threads() -> int:
    return lib().orc_num_threads()
