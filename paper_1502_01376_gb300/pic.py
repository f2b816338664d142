"""Drifting-plasma particle-in-cell runs on the GPU and the NCI growth they show
(Sec. 4: the E2 energy of the Table 1 plasma with and without the k1
modification, the low-pass filter of the current, and the choice of time step).

run() advances the Table 1 setup (256 x 256 cells of 0.2, periodic, gamma = 50,
n/n_p = 100, 8 + 8 particles per cell, quiet start) with the library's PIC step
(hyb_pic_step: gather and Boris push with B time-centred, charge-conserving
deposit, hybrid advance) and records the field energies from hyb_diag.
growth_rate() fits the exponential growth of an energy history; predicted()
gives the root solver's fastest growth over the run's own (k1, k2) modes.  All
arithmetic of the method runs in libhyb.so; this module chooses parameters,
loops and fits.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import hyb, workloads as wl

TABLE1 = wl.Workload("pic_table1_256x256", 2, 256, 256, dx1=0.2, dx2=0.2, dt=0.08, precision=32, filt_kc=0.0,
                     filt_w=0.2, shape_order=2, seed=11, kind="plasma", ppc=8, gamma=50.0, u_th=1e-4)
BUMP = (0.15, 0.26, 0.01)       # Sec. 4: k1l/kg1, k1u/kg1, dk_max/kg1


@dataclass
class History:
    t: np.ndarray          # times of the samples (units of 1/omega_0)
    energy: np.ndarray     # [samples, 6]: E1, E2, E3, B1, B2, B3 field energies
    seconds: float         # wall time of the run (GPU work included)
    steps: int


def run(w: wl.Workload = TABLE1, steps: int = 4000, every: int = 20, kmod=None, device="cuda",
        resident: bool = False) -> History:
    """A PIC run of workload w (its dt, filter, shape order) with an optional Sec. 4 k1
    modification kmod = (k1l, k1u, dk_max) in units of kg1; energies every `every` steps.
    resident: keep E, B in k1 space between steps (hyb_set_resident)."""
    import time

    import torch
    kl, ku, km = kmod if kmod else (0.0, 0.0, 0.0)
    desc = hyb.desc_from_workload(w, kmod_l=kl, kmod_u=ku, kmod_max=km)
    g = hyb.Grid(desc)
    dt_ = torch.float32 if w.precision == 32 else torch.float64
    E = [torch.zeros(w.shape, dtype=dt_, device=device) for _ in range(3)]
    B = [torch.zeros(w.shape, dtype=dt_, device=device) for _ in range(3)]
    J = [torch.zeros(w.shape, dtype=dt_, device=device) for _ in range(3)]
    g.bind(E, B, J)
    if resident:
        g.set_resident(True)
    cell, off, u, qm, q = wl.pic_plasma_torch(w, device)
    off_new = torch.empty_like(off)
    v3 = torch.empty_like(qm)
    pic = hyb.Pic(g)
    ts, es = [0.0], [g.diag()[:6]]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    done = 0
    while done < steps:
        k = min(every, steps - done)
        pic.step(cell, off, u, qm, q, off_new, v3, order=w.shape_order, nsteps=k)
        done += k
        ts.append(done * w.dt)
        es.append(g.diag()[:6])             # synchronous
    seconds = time.perf_counter() - t0
    g.check()
    pic.close()
    g.close()
    return History(np.array(ts), np.array(es), seconds, steps)


def growth_rate(t, W, windows=(16.0, 32.0, 64.0, 128.0), t_min: float = 20.0, r2_min: float = 0.98,
                min_rise: float = 1.0):
    """Exponential growth rate Gamma of a field amplitude whose energy is W(t) ~ exp(2 Gamma t):
    half the largest least-squares slope of log W over the windows of the longest length
    (of `windows`, after t_min, past the start-up where the noise builds up from E = B = 0)
    in which log W is a clean exponential (coefficient of determination >= r2_min) that
    rises by at least `min_rise` (e-folds of the energy), so that windows of noise, and
    short stretches steeper than the exponential phase as a whole, do not count.  With no such
    window, half the least-squares slope of log W over the whole run after t_min (about 0
    for a run that does not grow)."""
    t = np.asarray(t, float)
    L = np.log(np.maximum(np.asarray(W, float), 1e-300))
    sel = t >= t_min
    ts, Ls = t[sel], L[sel]
    best = None
    for win in sorted(windows, reverse=True):          # the longest window length that qualifies
        if best is not None:
            break
        for i in range(len(ts)):
            j = np.searchsorted(ts, ts[i] + win)
            if j > len(ts) or j - i < 6:
                break
            x, y = ts[i:j] - ts[i], Ls[i:j]
            xm, ym = x.mean(), y.mean()
            sxx = np.sum((x - xm) ** 2)
            sxy = np.sum((x - xm) * (y - ym))
            syy = np.sum((y - ym) ** 2)
            if sxx <= 0 or syy <= 0:
                continue
            slope = sxy / sxx
            r2 = sxy * sxy / (sxx * syy)
            if r2 >= r2_min and slope * (x[-1] - x[0]) >= min_rise and (best is None or slope > best):
                best = slope
    if best is None:
        best = np.polyfit(ts, Ls, 1)[0] if len(ts) >= 2 else 0.0
    return 0.5 * float(best)


ALL_ALIASES = tuple((mu, nu) for mu in (-1, 0, 1) for nu in (-2, -1, 0, 1, 2))


def predicted(w: wl.Workload = TABLE1, kmod=None, aliases=((0, -1), (0, 0), (0, 1)), order=None):
    """Fastest growth the root solver finds over the run's own modes (k1, k2 > 0 of the
    grid's fundamental zone) and the given aliases; returns (growth, k1, k2, alias)."""
    import torch
    kl, ku, km = kmod if kmod else (0.0, 0.0, 0.0)
    k1 = 2 * math.pi * np.arange(1, w.n1 // 2 + 1) / (w.n1 * w.dx1)
    k2 = 2 * math.pi * np.arange(1, w.n2 // 2 + 1) / (w.n2 * w.dx2)
    K1, K2 = np.meshgrid(k1, k2, indexing="ij")
    n = K1.size
    kc = w.filt_kc if 0.0 < w.filt_kc < 1.0 else 0.0
    rows = np.stack([np.full(n, w.dt), np.full(n, w.dx1), np.full(n, w.dx2), np.full(n, w.gamma),
                     np.full(n, w.density), np.full(n, kc), np.full(n, w.filt_w), K1.ravel(), K2.ravel(),
                     np.full(n, kl), np.full(n, ku), np.full(n, km)], axis=1)
    g = hyb.nci_growth(torch.from_numpy(np.ascontiguousarray(rows)).cuda(), aliases=aliases,
                       order=order or w.shape_order, correct_j1=w.correct_j1).cpu().numpy()
    i, a = np.unravel_index(np.argmax(g), g.shape)
    return float(g[i, a]), float(K1.ravel()[i]), float(K2.ravel()[i]), aliases[a]
