"""NCI surrogate: training data from the GPU root solver of the dispersion
relation (Appendix), a small MLP trained by the library's own kernels, and the
pick of the current-filter cutoff and the time step (Sec. 4 strategies: a
low-pass filter in k1 against the fastest (0, +-1) modes, a smaller time step
against the (0, 0) modes).

Inputs of the network, each scaled to [-1, 1]:
  dt/dx1 in [0.1, 0.9], dx2/dx1 in [0.5, 2], gamma in [5, 100],
  filter cutoff kc in [0.3, 1.0] (fraction of pi/dx1), k1 dx1/pi, k2 dx2/pi in (0, 1].
Target: the largest growth rate over the aliases (mu, nu1) = (0, -1), (0, 0),
(0, 1), times 20.  dx1 = 0.2 and n/n_p = 100 are held fixed (Table 1); samples
above the Courant limit of Sec. 2.2 are flagged and left out of training.
All host logic here is sampling, batching and selection; the root solve,
the network's forward/backward and Adam run in libhyb.so.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass

import numpy as np

from . import hyb

DX1 = 0.2
WP2 = 100.0
FILT_W = 0.2
ALIASES = ((0, -1), (0, 0), (0, 1))
RANGES = {"dt_dx1": (0.1, 0.9), "dx2_dx1": (0.5, 2.0), "gamma": (5.0, 100.0), "kc": (0.3, 1.0)}
TARGET_SCALE = 20.0


def courant_dt(dx1, dx2):
    return 2.0 / np.sqrt(np.pi ** 2 / dx1 ** 2 + 4.0 / dx2 ** 2)


@dataclass
class Params:
    dt_dx1: np.ndarray
    dx2_dx1: np.ndarray
    gamma: np.ndarray
    kc: np.ndarray
    kap1: np.ndarray      # k1 dx1 / pi
    kap2: np.ndarray      # k2 dx2 / pi

    def __len__(self):
        return self.dt_dx1.size

    @property
    def stable(self):
        return self.dt_dx1 * DX1 <= courant_dt(DX1, self.dx2_dx1 * DX1)


def sample(n: int, seed: int) -> Params:
    rng = np.random.default_rng(seed)
    u = lambda k: rng.uniform(*RANGES[k], n)
    return Params(u("dt_dx1"), u("dx2_dx1"), u("gamma"), u("kc"),
                  rng.uniform(0.01, 1.0, n), rng.uniform(0.01, 1.0, n))


def solver_rows(P: Params) -> np.ndarray:
    """[n, 9] rows for hyb_nci_growth: dt, dx1, dx2, gamma, wp2, kc, w, k1, k2."""
    dx2 = P.dx2_dx1 * DX1
    return np.ascontiguousarray(np.stack([P.dt_dx1 * DX1, np.full(len(P), DX1), dx2, P.gamma, np.full(len(P), WP2),
                                          P.kc, np.full(len(P), FILT_W), P.kap1 * np.pi / DX1, P.kap2 * np.pi / dx2],
                                         axis=1))


def features(P: Params) -> np.ndarray:
    def s(v, lo, hi):
        return 2.0 * (v - lo) / (hi - lo) - 1.0
    f = [s(P.dt_dx1, *RANGES["dt_dx1"]), s(P.dx2_dx1, *RANGES["dx2_dx1"]), s(P.gamma, *RANGES["gamma"]),
         s(P.kc, *RANGES["kc"]), 2.0 * P.kap1 - 1.0, 2.0 * P.kap2 - 1.0]
    return np.ascontiguousarray(np.stack(f, axis=1).astype(np.float32))


def growth_gpu(P: Params, chunk: int = 1 << 18):
    """Max growth over the aliases from the GPU root solver (torch float64, on the device)."""
    import torch
    rows = solver_rows(P)
    out = []
    for i in range(0, len(P), chunk):
        g = hyb.nci_growth(torch.from_numpy(rows[i:i + chunk]).cuda(), aliases=ALIASES)
        out.append(g.max(dim=1).values)
    return torch.cat(out)


def dataset(n: int, seed: int):
    """(features [m, 6] float32 cuda, targets [m] float32 cuda) for the Courant-stable samples."""
    import torch
    P = sample(n, seed)
    keep = P.stable
    Pk = Params(*(getattr(P, f)[keep] for f in ("dt_dx1", "dx2_dx1", "gamma", "kc", "kap1", "kap2")))
    g = growth_gpu(Pk)
    X = torch.from_numpy(features(Pk)).cuda()
    y = (g * TARGET_SCALE).float().contiguous()
    return X, y, int(keep.sum()), n


def train(mlp: "hyb.MLP", X, y, steps: int = 3000, batch: int = 8192, lr: float = 1e-3, seed: int = 0,
          lr_final: float = 1e-4):
    """Adam on minibatches drawn with a seeded generator; returns the loss history (host)."""
    import torch
    gen = torch.Generator(device=X.device)
    gen.manual_seed(seed)
    losses = torch.zeros(steps, dtype=torch.float32, device=X.device)
    n = X.shape[0]
    for s in range(steps):
        idx = torch.randint(0, n, (batch,), generator=gen, device=X.device)
        xb = X.index_select(0, idx).contiguous()
        yb = y.index_select(0, idx).contiguous()
        # cosine decay from lr to lr_final
        a = lr_final + 0.5 * (lr - lr_final) * (1 + math.cos(math.pi * s / max(1, steps - 1)))
        mlp.train_step(xb, yb, a, losses[s:s + 1])
    return losses.cpu().numpy()


def kgrid(nk: int):
    k = (np.arange(nk) + 0.5) / nk
    return np.repeat(k, nk), np.tile(k, nk)


def max_growth_surrogate(mlp, dt_dx1, dx2_dx1, gamma, kc, nk: int = 48) -> np.ndarray:
    """Predicted max growth over an nk x nk (k1, k2) grid for each candidate setting."""
    import torch
    k1, k2 = kgrid(nk)
    cands = len(dt_dx1)
    rep = lambda v: np.repeat(np.asarray(v, dtype=np.float64), nk * nk)
    P = Params(rep(dt_dx1), rep(dx2_dx1), rep(gamma), rep(kc), np.tile(k1, cands), np.tile(k2, cands))
    y = mlp.forward(torch.from_numpy(features(P)).cuda())
    return (y.view(cands, nk * nk).max(dim=1).values / TARGET_SCALE).cpu().numpy()


def max_growth_solver(dt_dx1, dx2_dx1, gamma, kc, nk: int = 48) -> np.ndarray:
    """The same maximum from the root solver."""
    k1, k2 = kgrid(nk)
    cands = len(dt_dx1)
    rep = lambda v: np.repeat(np.asarray(v, dtype=np.float64), nk * nk)
    P = Params(rep(dt_dx1), rep(dx2_dx1), rep(gamma), rep(kc), np.tile(k1, cands), np.tile(k2, cands))
    g = growth_gpu(P)
    return g.view(cands, nk * nk).max(dim=1).values.cpu().numpy()


def candidates(dx2_dx1: float, dt_grid, kc_grid):
    """The (dt/dx1, kc) candidates of a grid of settings that satisfy the Courant limit."""
    dts, kcs = np.meshgrid(np.asarray(dt_grid, float), np.asarray(kc_grid, float), indexing="ij")
    dts, kcs = dts.ravel(), kcs.ravel()
    ok = dts * DX1 <= courant_dt(DX1, dx2_dx1 * DX1)
    return dts[ok], kcs[ok]


def select(dts, kcs, score, idx=None, tol: float = 0.002) -> int:
    """Index of the candidate with the lowest score, preferring the largest cutoff and then
    the largest time step among those within tol of the lowest (keep the most physics
    bandwidth); only the candidates in idx (default all) compete."""
    idx = np.arange(len(dts)) if idx is None else np.asarray(idx)
    best = score[idx].min()
    good = idx[score[idx] <= best + tol]
    return int(good[np.lexsort((dts[good], kcs[good]))[-1]])


def pick_solver(gamma: float, dx2_dx1: float, dt_grid, kc_grid, tol: float = 0.002, nk: int = 48):
    """The method without the network: the root solver scores every candidate."""
    dts, kcs = candidates(dx2_dx1, dt_grid, kc_grid)
    t0 = time.perf_counter()
    score = max_growth_solver(dts, np.full(dts.size, dx2_dx1), np.full(dts.size, gamma), kcs, nk)
    secs = time.perf_counter() - t0
    i = select(dts, kcs, score, tol=tol)
    return {"dt_dx1": float(dts[i]), "kc": float(kcs[i]), "growth": float(score[i]), "candidates": int(dts.size),
            "seconds": secs, "all_dt": dts, "all_kc": kcs, "all_growth": score}


def pick(mlp, gamma: float, dx2_dx1: float, dt_grid, kc_grid, tol: float = 0.002, nk: int = 48, verify: int = 0):
    """Candidate (dt/dx1, kc) with the lowest predicted max growth (select()).  With
    verify = k > 0 the root solver, the surrogate's judge, re-scores the k candidates with
    the lowest predicted growth and the pick is made among them on its values."""
    dts, kcs = candidates(dx2_dx1, dt_grid, kc_grid)
    t0 = time.perf_counter()
    pred = max_growth_surrogate(mlp, dts, np.full(dts.size, dx2_dx1), np.full(dts.size, gamma), kcs, nk)
    t_pred = time.perf_counter() - t0
    score = pred
    idx = np.arange(dts.size)
    t_ver = 0.0
    if verify > 0:
        idx = np.argsort(pred)[:verify]
        t1 = time.perf_counter()
        score = np.full(dts.size, np.inf)
        score[idx] = max_growth_solver(dts[idx], np.full(idx.size, dx2_dx1), np.full(idx.size, gamma), kcs[idx], nk)
        t_ver = time.perf_counter() - t1
    i = select(dts, kcs, score, idx, tol)
    return {"dt_dx1": float(dts[i]), "kc": float(kcs[i]), "predicted": float(pred[i]), "candidates": int(dts.size),
            "seconds": t_pred, "verify_seconds": t_ver, "verified": int(verify),
            "all_dt": dts, "all_kc": kcs, "all_pred": pred}
