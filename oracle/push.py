"""FP64 oracle of the particle step that feeds the deposit: field gather and
relativistic Boris push.  TEST INFRASTRUCTURE ONLY (imported by ``tests/`` and
the ``cpu_baseline`` leg of ``bench.py``; the product path never imports it).

Gather: the momentum-conserving interpolation of the Appendix (Eqs. for S_E and
S_B): every field component is interpolated with the order-l B-spline s_l along
each axis, taken at the component's own staggered grid points.  Positions are in
cell units, integer grid points at integers, a half point i + 1/2 stored at i:
  2D  E1 (1/2, 0)  E2 (0, 1/2)  E3 (0, 0)  B1 (0, 1/2)  B2 (1/2, 0)  B3 (1/2, 1/2)
  3D  E1 (1/2,0,0) E2 (0,1/2,0) E3 (0,0,1/2) B1 (0,1/2,1/2) B2 (1/2,0,1/2) B3 (1/2,1/2,0)
  F_c(x) = sum over grid points i of F_c[i] prod_a s_l(x_a - i_a - sigma_{c,a}),
with periodic wrap.  The sum runs over a fixed window of six points per axis;
the spline is zero outside its support.

Push (c = 1, Gaussian units, u = gamma v, h = (q/m) dt / 2), Boris's rotation:
  u- = u + h E;  t = h B / gamma(u-);  s = 2 t / (1 + |t|^2);
  u' = u- + u- x t;  u+ = u- + u' x s;  u_new = u+ + h E;
  x_new = x + dt u_new / gamma(u_new).
Before the gather each particle is moved to the cell that holds it (offsets in
[-1, 2) on entry); that integer decision and the new offset are taken in the
precision of the input offsets, as the GPU takes them.

Parity status (pins in ``tests/test_oracle_push.py``): gather pinned by the
B-spline partition of unity, exact reproduction of linear fields, and the
closed-form node weights; push pinned by the exact pure-E kick, the exact
|u|-preserving rotation angle 2 atan(h |B| / gamma) in a pure B field, the E x B
drift, and second-order convergence to the exact hyperbolic trajectory in a
uniform E field.
"""
from __future__ import annotations

import numpy as np

# staggering (1 = half point) of E1, E2, E3, B1, B2, B3 along x1, x2 (, x3)
STAGGER = {
    2: [(1, 0), (0, 1), (0, 0), (0, 1), (1, 0), (1, 1)],
    3: [(1, 0, 0), (0, 1, 0), (0, 0, 1), (0, 1, 1), (1, 0, 1), (1, 1, 0)],
}
WINDOW = np.arange(-2, 4)   # grid points relative to the cell, wide enough for l <= 3


def bspline(order: int, d):
    """Centred B-spline of order l (l + 1 points of support) in cell units."""
    a = np.abs(np.asarray(d, dtype=np.float64))
    if order == 1:
        return np.where(a < 1.0, 1.0 - a, 0.0)
    if order == 2:
        return np.where(a <= 0.5, 0.75 - a * a, np.where(a < 1.5, 0.5 * (1.5 - a) ** 2, 0.0))
    if order == 3:
        return np.where(a <= 1.0, (4.0 - 6.0 * a * a + 3.0 * a ** 3) / 6.0,
                        np.where(a < 2.0, (2.0 - a) ** 3 / 6.0, 0.0))
    raise ValueError("order must be 1, 2 or 3")


def renormalise(cell, off, shape):
    """Moves each particle to the cell that holds it, in the offsets' own precision.
    Returns (cell, off, ok); rejected particles (off outside [-1, 2) or cell out of
    range) keep their input values."""
    cell = np.array(cell, dtype=np.int64)
    off = np.array(off)
    one = off.dtype.type(1)
    n = np.asarray(shape, dtype=np.int64)
    ok = np.all((off >= -one) & (off < 2 * one) & (cell >= 0) & (cell < n), axis=1)
    c2, o2 = cell.copy(), off.copy()
    lo, hi = off < 0, off >= one
    o2[lo] = off[lo] + one
    c2[lo] -= 1
    o2[hi] = off[hi] - one
    c2[hi] += 1
    up = o2 >= one                   # -tiny + 1 rounded to 1
    o2[up] = 0
    c2[up] += 1
    c2 = np.mod(c2, n)
    c2[~ok], o2[~ok] = cell[~ok], off[~ok]
    return c2, o2, ok


def gather(fields, cell, off, order: int):
    """E, B at the particles: fields = [E1, E2, E3, B1, B2, B3], each [n2][n1]
    (2D) or [n3][n2][n1] (3D); cell int [np][dims]; off float [np][dims].
    Returns an array [np][6] in FP64."""
    dims = cell.shape[1]
    shape = fields[0].shape[::-1]          # (n1, n2[, n3])
    off = np.asarray(off, dtype=np.float64)
    out = np.zeros((cell.shape[0], 6))
    for c, st in enumerate(STAGGER[dims]):
        F = np.asarray(fields[c], dtype=np.float64)
        # weights along each axis for the window points
        w = [bspline(order, off[:, a:a + 1] - WINDOW[None, :] - 0.5 * st[a]) for a in range(dims)]
        idx = [np.mod(cell[:, a:a + 1] + WINDOW[None, :], shape[a]) for a in range(dims)]
        acc = np.zeros(cell.shape[0])
        if dims == 2:
            for j in range(len(WINDOW)):
                for i in range(len(WINDOW)):
                    acc += w[0][:, i] * w[1][:, j] * F[idx[1][:, j], idx[0][:, i]]
        else:
            for k in range(len(WINDOW)):
                for j in range(len(WINDOW)):
                    for i in range(len(WINDOW)):
                        acc += w[0][:, i] * w[1][:, j] * w[2][:, k] * F[idx[2][:, k], idx[1][:, j], idx[0][:, i]]
        out[:, c] = acc
    return out


def boris(u, E, B, qm, dt):
    """Relativistic Boris step u^{n-1/2} -> u^{n+1/2}; arrays [np][3], qm [np]."""
    u = np.asarray(u, dtype=np.float64)
    h = (0.5 * dt * np.asarray(qm, dtype=np.float64))[:, None]
    um = u + h * E
    g = np.sqrt(1.0 + np.sum(um * um, axis=1))[:, None]
    t = h * B / g
    s = 2.0 * t / (1.0 + np.sum(t * t, axis=1))[:, None]
    up = um + np.cross(um, t)
    return um + np.cross(up, s) + h * E


def push(fields, cell, off, u, qm, dt: float, dx, order: int):
    """One particle step.  Returns (cell, off, u_new, off_new, v3, ok): cell/off
    renormalised, u^{n+1/2}, x^{n+1} - cell in cell units, u3 / gamma.  Rejected
    particles keep u and get off_new = off, v3 = 0."""
    dims = np.asarray(cell).shape[1]
    shape = fields[0].shape[::-1]
    c2, o2, ok = renormalise(cell, off, shape)
    EB = gather(fields, c2, o2, order)
    un = boris(u, EB[:, :3], EB[:, 3:], qm, dt)
    un[~ok] = np.asarray(u, dtype=np.float64)[~ok]
    gi = 1.0 / np.sqrt(1.0 + np.sum(un * un, axis=1))
    o64 = o2.astype(np.float64)
    off_new = o64 + (dt / np.asarray(dx, dtype=np.float64)[None, :dims]) * un[:, :dims] * gi[:, None]
    off_new[~ok] = o64[~ok]
    v3 = np.where(ok, un[:, 2] * gi, 0.0)
    return c2, o64, un, off_new, v3, ok
