"""Seeded synthetic inputs for the hybrid Yee-FFT field advance.

This module holds none of the method's arithmetic: it draws random
band-limited fields and particle positions/velocities, and moves particles
ballistically (x^{n+1} = x^n + v dt) to give the deposit its start and end
points.  Both the CUDA path's tests and the oracle's tests take their inputs
from here, so the two sides see bit-identical inputs.

Workloads (shapes and distributions follow Table 1 and the drifting-plasma
setup of Sec. 3; c = 1, k_p = omega_p = 1):

  vacuum_beam      2D 128 x 64, dx = 0.1, dt = 0.05, FP64 state, 100 steps;
                   band-limited random E, B (|k| < 0.5 pi/dx, rms 1e-3 per
                   component); 4096 beam particles of charge -0.01 at
                   v1 = 0.99, uniform in the box, linear shapes, no filter.
  drift_plasma     2D 4096 x 1024, dx = 0.2, dt = 0.1, FP32 state; electrons
                   and positive particles (q/m = -1, +1), 8 per cell each,
                   uniform positions, u1 = gamma beta with gamma = 50 and a
                   Gaussian spread 1e-4 in u; density n/n_p = 100; quadratic
                   shapes; J1 correction + k1 low-pass filter at kc = 0.5 of
                   Nyquist, width 0.2 of Nyquist.
  drift_plasma_3d  3D 1024 x 256 x 256, dx = 0.2, dt = 0.08, gamma = 30,
                   2 particles per cell per species.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace

import numpy as np


@dataclass(frozen=True)
class Workload:
    name: str
    dims: int
    n1: int
    n2: int
    n3: int = 1
    dx1: float = 0.1
    dx2: float = 0.1
    dx3: float = 0.1
    dt: float = 0.05
    precision: int = 64
    steps: int = 100
    correct_j1: bool = True
    filt_kc: float = 0.0
    filt_w: float = 0.0
    shape_order: int = 1
    seed: int = 1
    # particles
    kind: str = "beam"            # "beam" | "plasma"
    n_particles: int = 4096       # beam only
    beam_q: float = -0.01
    beam_v1: float = 0.99
    ppc: int = 8                  # plasma: particles per cell per species
    gamma: float = 50.0
    u_th: float = 1e-4
    density: float = 100.0        # n / n_p
    field_amp: float = 1e-3
    field_kfrac: float = 0.5

    @property
    def shape(self):
        return (self.n3, self.n2, self.n1) if self.dims == 3 else (self.n2, self.n1)

    @property
    def cells(self) -> int:
        return self.n1 * self.n2 * (self.n3 if self.dims == 3 else 1)

    def scaled(self, **kw) -> "Workload":
        return replace(self, **kw)


VACUUM_BEAM = Workload("vacuum_beam_2d_128x64_f64", 2, 128, 64, dx1=0.1, dx2=0.1, dt=0.05,
                       precision=64, steps=100, seed=1, kind="beam", n_particles=4096,
                       shape_order=1)
DRIFT_PLASMA = Workload("drift_plasma_2d_4096x1024_f32", 2, 4096, 1024, dx1=0.2, dx2=0.2, dt=0.1,
                        precision=32, steps=1000, filt_kc=0.5, filt_w=0.2, shape_order=2, seed=2,
                        kind="plasma", ppc=8, gamma=50.0)
DRIFT_PLASMA_3D = Workload("drift_plasma_3d_1024x256x256_f32", 3, 1024, 256, 256, dx1=0.2, dx2=0.2,
                           dx3=0.2, dt=0.08, precision=32, steps=100, filt_kc=0.5, filt_w=0.2,
                           shape_order=2, seed=4, kind="plasma", ppc=2, gamma=30.0)

WORKLOADS = {w.name: w for w in (VACUUM_BEAM, DRIFT_PLASMA, DRIFT_PLASMA_3D)}


# ---------------------------------------------------------------------------
def band_limited_fields(w: Workload, rng: np.random.Generator | None = None):
    """Six real random fields (E1,E2,E3,B1,B2,B3) whose Fourier content is
    confined to |k| < kfrac * pi/dx (radially, in grid wavenumbers), with
    uniform random phases, each scaled to rms field_amp.  FP64."""
    rng = rng or np.random.default_rng(w.seed)
    shp = w.shape
    out = []
    # normalised wavenumbers in units of the Nyquist number of each axis
    axes = [np.fft.fftfreq(n) * 2.0 for n in shp[:-1]] + [np.fft.rfftfreq(shp[-1]) * 2.0]
    grids = np.meshgrid(*axes, indexing="ij")
    kr = np.sqrt(sum(g * g for g in grids))
    mask = (kr < w.field_kfrac)
    for _ in range(6):
        amp = rng.standard_normal(mask.shape)
        ph = rng.uniform(0.0, 2.0 * np.pi, mask.shape)
        spec = np.where(mask, amp * np.exp(1j * ph), 0.0)
        f = np.fft.irfftn(spec, s=shp, axes=tuple(range(len(shp))))
        rms = np.sqrt(np.mean(f * f))
        out.append(np.ascontiguousarray(f * (w.field_amp / rms if rms > 0 else 0.0)))
    return out[:3], out[3:]


@dataclass
class Particles:
    """Positions in cell units (x / dx per axis, FP64), velocities, charges."""
    x: np.ndarray          # [np, dims]
    v: np.ndarray          # [np, 3]  (v1, v2, v3)
    q: np.ndarray          # [np]

    @property
    def count(self) -> int:
        return self.q.size


def make_particles(w: Workload, rng: np.random.Generator | None = None) -> Particles:
    rng = rng or np.random.default_rng(w.seed + 1000)
    d = w.dims
    ext = np.array([w.n1, w.n2, w.n3][:d], dtype=np.float64)
    if w.kind == "beam":
        n = w.n_particles
        x = rng.uniform(0.0, 1.0, (n, d)) * ext
        v = np.zeros((n, 3))
        v[:, 0] = w.beam_v1
        q = np.full(n, w.beam_q)
        return Particles(x, v, q)
    # drifting plasma: two species, ppc each, q/m = -1 and +1
    ncell = w.cells
    n = ncell * w.ppc
    dV = w.dx1 * w.dx2 * (w.dx3 if d == 3 else 1.0)
    rho0 = w.density / (4.0 * np.pi)            # 4 pi rho0 = omega_p^2 = n/n_p
    xs, vs, qs = [], [], []
    for sign in (-1.0, +1.0):
        x = rng.uniform(0.0, 1.0, (n, d)) * ext
        u = rng.standard_normal((n, 3)) * w.u_th
        u[:, 0] += np.sqrt(w.gamma ** 2 - 1.0)
        gam = np.sqrt(1.0 + np.sum(u * u, axis=1))
        xs.append(x)
        vs.append(u / gam[:, None])
        qs.append(np.full(n, sign * rho0 * dV / w.ppc))
    return Particles(np.concatenate(xs), np.concatenate(vs), np.concatenate(qs))


def ballistic_move(w: Workload, p: Particles, step: int, real=np.float64):
    """Start/end points of step `step` (x^n -> x^{n+1}, ballistic), as the
    deposit interface takes them: integer cell of x^n per axis (periodic),
    offset of x^n and of x^{n+1} from that cell, in cell units, rounded to
    `real`.  Also returns v3 (the out-of-plane velocity in 2D)."""
    d = w.dims
    dxs = np.array([w.dx1, w.dx2, w.dx3][:d])
    ext = np.array([w.n1, w.n2, w.n3][:d], dtype=np.float64)
    x0 = np.mod(p.x + step * p.v[:, :d] * w.dt / dxs, ext)
    cell = np.floor(x0)
    off0 = x0 - cell
    off1 = off0 + p.v[:, :d] * w.dt / dxs
    off0r = off0.astype(real)
    off1r = off1.astype(real)
    # an offset just below 1 can round to 1 in the target precision: move it
    # to the next cell so that the rounded offset stays in [0, 1)
    up = off0r >= 1
    cell = np.where(up, cell + 1, cell)
    off0r = np.where(up, real(0), off0r).astype(real)
    off1r = np.where(up, (off1 - 1.0).astype(real), off1r).astype(real)
    cell = np.mod(cell, ext).astype(np.int32)
    off0 = np.ascontiguousarray(off0r)
    off1 = np.ascontiguousarray(off1r)
    v3 = np.ascontiguousarray(p.v[:, 2].astype(real))
    return np.ascontiguousarray(cell), off0, off1, v3


def position_at(w: Workload, p: Particles, step: int, real=np.float64):
    """Integer cell and offset of x^step (for charge densities)."""
    cell, off0, _, _ = ballistic_move(w, p, step, real)
    return cell, off0


def plasma_move_torch(w: Workload, device, seed: int | None = None, step: int = 0):
    """Drifting-plasma particles drawn directly on a CUDA device (seeded
    torch generator; same distributions as make_particles), each species
    stored in cell order, returned as the
    deposit interface takes them for step `step`: int32 cell [np, dims],
    float32 offsets of x^n and x^{n+1}, float32 v3 and q."""
    import torch
    gen = torch.Generator(device=device)
    gen.manual_seed(w.seed + 2000 if seed is None else seed)
    d = w.dims
    ext = torch.tensor([w.n1, w.n2, w.n3][:d], dtype=torch.float64, device=device)
    dxs = torch.tensor([w.dx1, w.dx2, w.dx3][:d], dtype=torch.float64, device=device)
    n = w.cells * w.ppc
    dV = w.dx1 * w.dx2 * (w.dx3 if d == 3 else 1.0)
    rho0 = w.density / (4.0 * np.pi)
    cells, off0s, off1s, v3s, qs = [], [], [], [], []
    for sign in (-1.0, +1.0):
        x = torch.rand(n, d, generator=gen, device=device, dtype=torch.float64) * ext
        u = torch.randn(n, 3, generator=gen, device=device, dtype=torch.float64) * w.u_th
        u[:, 0] += np.sqrt(w.gamma ** 2 - 1.0)
        v = u / torch.sqrt(1.0 + (u * u).sum(1, keepdim=True))
        del u
        x = torch.remainder(x + step * v[:, :d] * w.dt / dxs, ext)
        c = torch.floor(x)
        o0 = x - c
        o1 = o0 + v[:, :d] * w.dt / dxs
        o0f = o0.to(torch.float32)
        up = o0f >= 1                      # rounding to FP32 reached 1: move to the next cell
        c = torch.where(up, c + 1, c)
        o1 = torch.where(up, o1 - 1.0, o1)
        o0f = torch.where(up, torch.zeros_like(o0f), o0f)
        c = torch.remainder(c, ext)
        # stored in cell order, as a PIC code keeps its particles
        key = c[:, d - 1].to(torch.int64)
        for a in range(d - 2, -1, -1):
            key = key * int(ext[a].item()) + c[:, a].to(torch.int64)
        order = torch.argsort(key, stable=True)
        del key
        cells.append(c[order].to(torch.int32))
        off0s.append(o0f[order])
        off1s.append(o1[order].to(torch.float32))
        v3s.append(v[order, 2].to(torch.float32))
        del order
        qs.append(torch.full((n,), sign * rho0 * dV / w.ppc, device=device, dtype=torch.float32))
        del x, v, c, o0, o1
    return (torch.cat(cells).contiguous(), torch.cat(off0s).contiguous(), torch.cat(off1s).contiguous(),
            torch.cat(v3s).contiguous(), torch.cat(qs).contiguous())


def plasma_push_particles_torch(w: Workload, device, seed: int | None = None):
    """Both species of the drifting plasma for the particle push, drawn on a CUDA
    device (seeded torch generator), w.ppc per cell per species, stored in cell
    order (as a PIC code keeps them sorted): int32 cell [np, dims], float32
    offsets in [0, 1) [np, dims], float32 u = gamma v [np, 3] (drift gamma along
    x1 plus a Gaussian spread u_th), float32 q/m = -1 (electrons) or +1 [np]."""
    import torch
    gen = torch.Generator(device=device)
    gen.manual_seed(w.seed + 3000 if seed is None else seed)
    d = w.dims
    n = w.cells * w.ppc
    idx = torch.arange(w.cells, device=device, dtype=torch.int64).repeat_interleave(w.ppc)
    if d == 2:
        cell = torch.stack([idx % w.n1, idx // w.n1], dim=1)
    else:
        cell = torch.stack([idx % w.n1, (idx // w.n1) % w.n2, idx // (w.n1 * w.n2)], dim=1)
    cell = cell.to(torch.int32)
    del idx
    cells, offs, us, qms = [], [], [], []
    for sign in (-1.0, +1.0):
        cells.append(cell)
        offs.append(torch.rand(n, d, generator=gen, device=device, dtype=torch.float32))
        u = torch.randn(n, 3, generator=gen, device=device, dtype=torch.float32) * w.u_th
        u[:, 0] += float(np.sqrt(w.gamma ** 2 - 1.0))
        us.append(u)
        qms.append(torch.full((n,), sign, device=device, dtype=torch.float32))
    return (torch.cat(cells).contiguous(), torch.cat(offs).contiguous(), torch.cat(us).contiguous(),
            torch.cat(qms).contiguous())


def pic_plasma_torch(w: Workload, device, seed: int | None = None, real=None):
    """Both species of the drifting plasma for a particle-in-cell run, drawn on a CUDA
    device (seeded torch generator), w.ppc per cell per species, in cell order: a quiet
    start (the positive species at the electrons' positions, so the plasma starts
    neutral in every cell and E = B = 0 is consistent), independent Gaussian spreads
    u_th in u.  Returns int32 cell [np, dims], offsets in [0, 1) [np, dims],
    u = gamma v [np, 3], q/m = -1 or +1 [np] and the macro-particle charge
    q = +-rho0 dV / ppc [np] (rho0 = n/n_p / (4 pi), so omega_p^2 = n/n_p)."""
    import torch
    dt = real or (torch.float32 if w.precision == 32 else torch.float64)
    gen = torch.Generator(device=device)
    gen.manual_seed(w.seed + 4000 if seed is None else seed)
    d = w.dims
    n = w.cells * w.ppc
    idx = torch.arange(w.cells, device=device, dtype=torch.int64).repeat_interleave(w.ppc)
    if d == 2:
        cell = torch.stack([idx % w.n1, idx // w.n1], dim=1)
    else:
        cell = torch.stack([idx % w.n1, (idx // w.n1) % w.n2, idx // (w.n1 * w.n2)], dim=1)
    cell = cell.to(torch.int32)
    del idx
    off = torch.rand(n, d, generator=gen, device=device, dtype=torch.float64).to(dt)
    dV = w.dx1 * w.dx2 * (w.dx3 if d == 3 else 1.0)
    rho0 = w.density / (4.0 * np.pi)
    us, qms, qs = [], [], []
    for sign in (-1.0, +1.0):
        u = torch.randn(n, 3, generator=gen, device=device, dtype=torch.float64) * w.u_th
        u[:, 0] += float(np.sqrt(w.gamma ** 2 - 1.0))
        us.append(u.to(dt))
        qms.append(torch.full((n,), sign, device=device, dtype=dt))
        qs.append(torch.full((n,), sign * rho0 * dV / w.ppc, device=device, dtype=dt))
    return (torch.cat([cell, cell]).contiguous(), torch.cat([off, off]).contiguous(), torch.cat(us).contiguous(),
            torch.cat(qms).contiguous(), torch.cat(qs).contiguous())
