#!/usr/bin/env python
"""Benchmark of the hybrid Yee-FFT field advance on GB300.

Workload: the 2D drifting-plasma grid, 4096 x 1024 cells, FP32 fields,
dx = 0.2, dt = 0.1, J1 correction + k1 low-pass filter (kc = 0.5 of Nyquist);
J deposited once (charge-conserving, quadratic shapes) from 8 + 8 particles
per cell drifting at gamma = 50, before timing.  A step is one hyb_advance
(FFT of E, B, J along x1, J1 correction, filter, Faraday + Ampere per k1 mode,
inverse FFT).  Metric: cell-steps/s.  L2 is flushed (256 MB write) between
timed steps; each step is timed with CUDA events on the grid's stream.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

--impl reference times the FP64 CPU oracle (test infrastructure) on the
host cores on bounded samples of the same workload.  With torchrun (N > 1)
every rank runs an independent replica (the path does not shard across
GPUs here); value = N * cells / max-over-ranks step time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "hybrid-solver cell-steps/s on 1 GB300 at <=1e-5 rel err vs FP64; % HBM roofline"
UNIT = "cell-steps/s"
BYTES_PER_CELL_STEP = 60          # read E, B, J (9 words) + write E, B (6 words), FP32


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-extras", action="store_true", help="skip e2e, cpu baseline and fp64 comparison")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the short batched, 3D and surrogate measurements of the default run")
    ap.add_argument("--quick", action="store_true",
                    help="profiling mode: random band-limited J instead of the particle deposit, no extras")
    ap.add_argument("--n1", type=int, default=4096,
                    help="drift_plasma with another row length at the same 4096 x 1024 cells (4096 is the "
                         "benchmark; others show the n1 = 512 .. 2048 kernels and the three-pass path)")
    ap.add_argument("--batch-strips", default="",
                    help="batched workload: rows per strip per n1 as '512:3,1024:2,...' instead of the autotuner")
    ap.add_argument("--batch-split", default="",
                    help="batched workload with --batch-strips: CTAs of the single launch's roles (n1 = 4096, 512, "
                         "1024, 2048, quasi-3D) as '64,6,7,18,57'")
    ap.add_argument("--ppc", type=int, default=8,
                    help="push workload: particles per cell per species (8 is the benchmark; fewer for profiling)")
    ap.add_argument("--sweep-n1", default="16,32,64,128,256,512,1024",
                    help="x1_sweep workload: the row lengths to run (comma-separated)")
    ap.add_argument("--sweep-cells", type=int, default=1 << 25,
                    help="x1_sweep workload: cells per grid (2^25 is the sweep; smaller sizes are for profiling)")
    ap.add_argument("--rows3d", type=int, default=256,
                    help="3d workload: n2 = n3 = this (256 is the benchmark; smaller sizes are for profiling)")
    ap.add_argument("--workload", default="drift_plasma",
                    choices=["drift_plasma", "batched", "3d", "vacuum_beam", "x1_sweep", "surrogate", "push"],
                    help="drift_plasma (default, the headline): 2D 4096 x 1024 FP32; batched: 16 uneven 2D grids "
                         "+ quasi-3D modes m = 0, 1, 2 (2048 x 512 complex) in one CUDA-graph step; 3d: 1024 x 256 x 256 "
                         "FP32, radix FFT vs DFT-GEMM x1 transform; vacuum_beam: 2D 128 x 64 FP64; x1_sweep: both x1 "
                         "transforms for n1 = 16 .. 1024 at 2^25 cells; surrogate: NCI surrogate trained on 200k "
                         "root-solver samples, then the pick of cutoff and dt judged by the solver; push: field gather "
                         "and Boris push of the drifting plasma's 67 M particles")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


KERNEL_SOURCES = {
    "k_fused_tm": ("fused_tm.cu", "tm_body.cuh", "tm_sched.cuh", "tm_dev.cuh", "fused_dev.cuh", "fused_api.cuh",
                   "packed_dev.cuh"),
}
KERNEL_PROFILES = {
    "k_fused_tm": "fused_tm_drift_plasma_4096x1024.md",
}


def kernel_source_hash(kernel="k_fused_tm"):
    """Hash of the kernel's sources with line comments and blank lines dropped, so that the
    profile summary stays matched to the code through comment-only edits."""
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, "paper_1502_01376_gb300", "csrc", f)) as fh:
            for line in fh:
                code = line.split("//", 1)[0].rstrip()
                if code:
                    h.update(code.encode() + b"\n")
    return h.hexdigest()[:16]


# FP32 additions, multiplications and fused multiply-adds per cell-step of the n1 = 4096 fused
# kernel, counted from its factorization: a 2048-point complex FFT of 8 x 8 x 8 x 4 costs about
# 35.5 per complex point (an 8-point DFT 56 per 8 points, its seven twiddle products 28, three such
# stages, then 4 per point for the radix-4 stage), the even/odd split of the real transform about 4
# per real point, so a 4096-point real transform about 21.8 per point; 15 transforms per cell-step
# and about 36 for the per-mode Faraday and Ampere updates.
FP32_OPS_PER_CELL_STEP_N4096 = 15 * 21.8 + 36.0
FP32_LANES_PER_SM = 128


def fp32_view(cells, kernel_ms, sampler=None):
    """The fused kernel's FP32 operation rate against the FP32 lanes' peak (SMs x 128 lanes x the
    maximum SM clock seen by the clock sampler, else 2070 MHz): the kernel sits at the ridge point
    between this peak and the HBM bandwidth, so both fractions describe it."""
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    mhz = 2070.0
    if sampler is not None:
        summ = sampler.summary() or {}
        mhz = float(summ.get("sm_max_mhz") or mhz)
    peak = sms * FP32_LANES_PER_SM * mhz * 1e6
    ops = FP32_OPS_PER_CELL_STEP_N4096 * cells
    achieved = ops / (kernel_ms / 1e3)
    return {"ops_per_cell_step": FP32_OPS_PER_CELL_STEP_N4096, "ops_per_launch": ops, "achieved_ops_per_s": achieved,
            "peak_ops_per_s": peak, "frac": achieved / peak,
            "peak_from": f"{sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x {mhz:.0f} MHz"}


def profiled_traffic(cells, kernel):
    """DRAM bytes per launch of the fused kernel from the committed ncu summary, if it
    was taken on the current kernel source: the measured reads plus the writes, where
    the writes are the larger of the measured ones and the algorithmic 24 B per cell
    (E and B written once): output lines still dirty in L2 when the kernel ends are
    written back during the next kernel, outside the captured launch."""
    if kernel not in KERNEL_PROFILES:
        return None
    path = os.path.join(ROOT, "profiles", KERNEL_PROFILES[kernel])
    if not os.path.exists(path):
        return None
    src_hash, rd, wr = None, None, None
    for line in open(path):
        if line.startswith("kernel_source_hash:"):
            src_hash = line.split(":", 1)[1].strip()
        if line.startswith("dram_read_bytes_per_cell:"):
            rd = float(line.split(":", 1)[1].strip())
        if line.startswith("dram_write_bytes_per_cell:"):
            wr = float(line.split(":", 1)[1].strip())
    if src_hash != kernel_source_hash(kernel) or rd is None or wr is None:
        return None
    return {"bytes": (rd + max(wr, 24.0)) * cells, "read_bytes": rd * cells, "write_bytes_in_kernel": wr * cells,
            "read_over_algorithmic": rd / 36.0,
            "note": "writes counted at max(measured, algorithmic 24 B/cell): lines still dirty at kernel end "
                    "are written back after it"}


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None
        self.t0 = self.t1 = None
        self.spans = []                 # every marked (begin, end) interval

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append((time.time(), [c.strip() for c in line.split(",")]))

    def mark(self, begin):
        if begin:
            self.t0 = time.time()
        else:
            self.t1 = time.time()
            if self.t0:
                self.spans.append((self.t0, self.t1))

    def stop(self):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        inside = [r for t, r in self.rows if any(a <= t <= b for a, b in self.spans)]
        use = inside if inside else [r for _, r in self.rows]
        sm = [float(r[0]) for r in use if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in use if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in use for i in range(4) if len(r) > 4 + i and r[4 + i] == "Active"})
        pw = [float(r[2]) for r in use if r[2].replace(".", "").isdigit()]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(use), "in_timed_region": bool(inside),
                "power_w_max": max(pw) if pw else None}


def replica_aggregate(ms, kms, cells, world, device):
    """Max-over-ranks step and kernel times of independent replicas, and the
    whole-job value world * cells / max step time (cell-steps/s)."""
    import torch
    if world > 1:
        t = torch.tensor([ms, kms], device=device, dtype=torch.float64)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms, kms = float(t[0]), float(t[1])
    return ms, kms, world * cells / (ms / 1e3)


def cpu_baseline_sample(workload, budget_s=12.0):
    """The oracle as it stands on a bounded sample of the workload: the full
    4096-point x1 rows on a 4096 x R periodic strip, timed on the host cores."""
    import numpy as np
    import oracle
    from paper_1502_01376_gb300 import workloads as wl
    rows = 64
    w = workload.scaled(n2=rows)
    g = oracle.grid(n1=w.n1, n2=w.n2, dx1=w.dx1, dx2=w.dx2, dt=w.dt, filt_kc=w.filt_kc, filt_w=w.filt_w)
    E, B = wl.band_limited_fields(w)
    rng = np.random.default_rng(0)
    J = [rng.standard_normal(w.shape) * 1e-3 for _ in range(3)]
    oracle.step(g, E, B, J, 1)                 # warm
    t0 = time.perf_counter()
    n = 0
    while True:
        oracle.step(g, E, B, J, 1)
        n += 1
        if time.perf_counter() - t0 > budget_s or n >= 5000:
            break
    dt = time.perf_counter() - t0
    return {"value": w.cells * n / dt, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"{n} oracle steps of a {w.n1} x {rows} periodic strip of the workload ({dt:.1f} s)"}


def run_reference(args):
    ws, rank, _ = dist_env()
    from paper_1502_01376_gb300 import workloads as wl
    w = wl.DRIFT_PLASMA
    if rank != 0:
        return
    import numpy as np
    import oracle
    oracle.build()
    rows = 64                       # the same 4096 x 64 strip as the cpu_baseline sample
    ws_ = w.scaled(n2=rows)
    g = oracle.grid(n1=ws_.n1, n2=ws_.n2, dx1=ws_.dx1, dx2=ws_.dx2, dt=ws_.dt, filt_kc=ws_.filt_kc, filt_w=ws_.filt_w)
    E, B = wl.band_limited_fields(ws_)
    rng = np.random.default_rng(0)
    J = [rng.standard_normal(ws_.shape) * 1e-3 for _ in range(3)]
    for _ in range(args.warmup):
        oracle.step(g, E, B, J, 1)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.step(g, E, B, J, 1)
        times.append(time.perf_counter() - t0)
    ms = 1e3 * statistics.mean(times)
    value = ws_.cells / (ms / 1e3)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "sample_rows": rows, "n1": w.n1, "n2_full": w.n2},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": f"each step: one oracle step of a {ws_.n1} x {rows} periodic strip of the workload"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def time_steps(step_fn, K, W, stream, flush, sampler):
    """W untimed steps, then K steps each bracketed by CUDA events on `stream`,
    with an L2 flush (256 MB write) before every timed step."""
    import torch
    for _ in range(W):
        step_fn()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    if sampler:
        sampler.mark(True)
    for i in range(K):
        flush.zero_()
        ev[i][0].record(stream)
        step_fn()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    if sampler:
        sampler.mark(False)
    return statistics.mean(a.elapsed_time(b) for a, b in ev)


def x1_compare(hyb, w, arrs, stream, flush, sampler, steps_, warmup, dev):
    """Time the three-pass advance with the radix x1 FFT (path 1) and with the
    DFT-GEMM (path 3) on the same inputs; per-field relative L2 error of each
    after 3 steps against the FP64 GPU path (parity-tested against the oracle)."""
    import torch
    out = {}
    fin = {}
    for path in (64, 1, 3, 4):
        prec = 64 if path == 64 else 32
        dt = torch.float64 if prec == 64 else torch.float32
        g = hyb.Grid(hyb.desc_from_workload(w, path=1 if path == 64 else path, precision=prec), stream)
        F = [torch.from_numpy(a).to(device=dev, dtype=dt) for a in arrs]
        g.bind(F[0:3], F[3:6], F[6:9])
        g.advance(3)
        torch.cuda.synchronize()
        fin[path] = [f.double() if path != 64 else f for f in F[:6]]
        if path != 64:
            steps = steps_ if path == 1 else max(3, min(steps_, 20))      # the DFT-GEMM paths are slower
            out[f"ms_path{path}"] = time_steps(lambda: g.advance(1), steps, warmup, stream, flush, sampler)
            out[f"launches_path{path}"] = g.launches_per_step
        g.close()
        del F
    names = ("E1", "E2", "E3", "B1", "B2", "B3")
    for path in (1, 3, 4):
        out[f"err_path{path}"] = {n: float((a - b).norm() / b.norm()) for n, a, b in zip(names, fin[path], fin[64])}
    return out


def measure_surrogate(hyb, sg, steps, warmup, sampler=None, n_samples=200000):
    """The learned part: n_samples (dt/dx1, dx2/dx1, gamma, kc, k1, k2) samples labelled by
    the FP64 GPU root solver of the NCI dispersion relation, the MLP 6 -> 256 x 4 -> 1
    trained by the library's own kernels, then the pick of filter cutoff and dt for
    the drifting-plasma run (gamma 50, square cells), judged by the root solver."""
    import numpy as np
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    X, y, kept, n = sg.dataset(n_samples, seed=21)
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    Xv, yv, _, _ = sg.dataset(20000, seed=22)
    net = hyb.MLP(6, 256, 4, seed=5)
    batch = 8192
    sg.train(net, X, y, steps=warmup, batch=batch, lr=2e-3, seed=0)       # warm-up steps (not timed)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if sampler:
        sampler.mark(True)
    n_launch0 = net.launch_count()
    ev0.record()
    hist = sg.train(net, X, y, steps=steps, batch=batch, lr=2e-3, seed=1)
    ev1.record()
    n_launches = net.launch_count() - n_launch0
    torch.cuda.synchronize()
    if sampler:
        sampler.mark(False)
    train_ms = ev0.elapsed_time(ev1)
    pred = net.forward(Xv)
    mse = float(torch.mean((pred - yv) ** 2))
    var = float(torch.var(yv))
    dts = np.arange(0.2, 0.51, 0.05)
    kcs = np.arange(0.3, 1.01, 0.1)
    sg.pick(net, 50.0, 1.0, dts, kcs)                   # first call sizes the activation buffers
    res = sg.pick(net, 50.0, 1.0, dts, kcs)
    confirmed = float(sg.max_growth_solver([res["dt_dx1"]], [1.0], [50.0], [res["kc"]])[0])
    # the surrogate prunes, the root solver judges the 16 most promising candidates
    resv = sg.pick(net, 50.0, 1.0, dts, kcs, verify=16)
    confirmed_v = float(sg.max_growth_solver([resv["dt_dx1"]], [1.0], [50.0], [resv["kc"]])[0])
    unfiltered = float(sg.max_growth_solver([0.5], [1.0], [50.0], [1.0])[0])
    ex = sg.pick_solver(50.0, 1.0, dts[:1], kcs[:1])    # warm
    ex = sg.pick_solver(50.0, 1.0, dts, kcs)
    net.close()
    return {"value": steps * batch / (train_ms / 1e3), "unit": "samples/s", "steps": steps,
            "ms_per_step": train_ms / steps, "gpu_launches": n_launches,
            "config": {"workload": f"nci_surrogate_{n_samples // 1000}k", "samples": n, "kept_below_courant": kept,
                       "label_seconds": t_data, "batch": batch, "loss_first": float(hist[:10].mean()),
                       "loss_last": float(hist[-50:].mean()), "val_r2": 1.0 - mse / var,
                       "pick": {"dt_dx1": res["dt_dx1"], "kc": res["kc"], "predicted": res["predicted"],
                                "solver_at_pick": confirmed, "solver_unfiltered_dt0.5": unfiltered,
                                "candidates": res["candidates"], "surrogate_scan_s": res["seconds"],
                                "exhaustive_solver": {"dt_dx1": ex["dt_dx1"], "kc": ex["kc"], "growth": ex["growth"],
                                                      "seconds": ex["seconds"]},
                                "verified_pick": {"dt_dx1": resv["dt_dx1"], "kc": resv["kc"], "solver": confirmed_v,
                                                  "candidates_solved": resv["verified"],
                                                  "seconds": resv["seconds"] + resv["verify_seconds"]}}}}


def run_surrogate(args):
    import torch
    torch.cuda.set_device(0)
    from paper_1502_01376_gb300 import build, hyb, surrogate as sg
    build.build()
    sampler = ClockSampler(0)
    sampler.start()
    time.sleep(0.5)
    r = measure_surrogate(hyb, sg, max(args.steps, 500), args.warmup, sampler)
    sampler.stop()
    line = {"metric": "NCI surrogate training samples/s (MLP 6->256x4->1, BF16 operands, FP32 accumulation)",
            "value": r["value"], "unit": r["unit"], "n_gpus": 1, "steps": r["steps"],
            "warmup": args.warmup, "ms_per_step": r["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
            "gpu_launches": r["gpu_launches"], "clocks": sampler.summary(), "config": r["config"]}
    print(json.dumps(line), flush=True)


def run_push(args):
    """The particle step that feeds the deposit (field gather with momentum-conserving
    interpolation, relativistic Boris push) on the drifting-plasma grid: 8 + 8 particles
    per cell (67 M), quadratic shapes, band-limited random E and B; each step pushes
    every particle once and its x^{n+1} offsets become the next step's x^n."""
    import numpy as np
    import torch
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    from paper_1502_01376_gb300 import build, hyb, workloads as wl
    build.build()
    stream = torch.cuda.current_stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    sampler = ClockSampler(0)
    sampler.start()
    time.sleep(0.5)
    peak, src = peaks()
    w = wl.DRIFT_PLASMA.scaled(ppc=args.ppc)
    E0, B0 = wl.band_limited_fields(w)
    fields = [a.astype(np.float32) for a in list(E0) + list(B0)]
    g = hyb.Grid(hyb.desc_from_workload(w), stream)
    E = [torch.from_numpy(f).to(dev) for f in fields[:3]]
    B = [torch.from_numpy(f).to(dev) for f in fields[3:]]
    J = [torch.zeros(w.shape, device=dev) for _ in range(3)]
    g.bind(E, B, J)
    cell, off, u, qm = wl.plasma_push_particles_torch(w, dev)
    n = qm.numel()
    buf = [off, torch.empty_like(off)]
    v3 = torch.empty_like(qm)
    state = {"i": 0}

    def step():
        a, b = buf[state["i"]], buf[1 - state["i"]]
        g.push(cell, a, u, qm, b, v3, order=w.shape_order)
        state["i"] = 1 - state["i"]

    ms = time_steps(step, args.steps, args.warmup, stream, flush, sampler)
    g.check()
    sampler.stop()
    per_particle = 2 * 4 + 2 * 4 + 3 * 4 + 4 + 2 * 4 + 2 * 4 + 3 * 4 + 2 * 4 + 4     # read cell, off, u, q/m; write cell, off, u, off_new, v3
    alg_bytes = per_particle * n + 6 * 4 * w.cells
    achieved = alg_bytes / (ms / 1e3) / 1e9
    line = {"metric": "particle pushes/s (field gather, momentum-conserving quadratic shapes, relativistic Boris) on 1 GB300",
            "value": n / (ms / 1e3), "unit": "particle-steps/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": None, "peak_source": src, "kernel": "k_push2d<float, 2>",
                         "bytes_per_launch": alg_bytes,
                         "bytes_per_unit": f"{per_particle} B per particle + 24 B per cell of fields"},
            "gpu_launches": args.steps, "clocks": sampler.summary(),
            "config": {"workload": f"drift_plasma_2d_4096x1024_push_{w.ppc}+{w.ppc}ppc_f32", "particles": n, "shape_order": w.shape_order,
                       "fields": "band-limited random E, B", "order": "particles stored in cell order",
                       "l2": "flushed between timed steps (256 MB write)"}}
    if not args.no_extras:
        from oracle import push as P
        k = 200000
        sel = torch.from_numpy(np.random.default_rng(1).choice(n, k, replace=False)).to(dev)
        ins = [t[sel].cpu().numpy() for t in (cell, buf[state["i"]], u, qm)]
        t0 = time.perf_counter()
        P.push(fields, ins[0], ins[1], ins[2], ins[3], w.dt, np.array([w.dx1, w.dx2]), w.shape_order)
        cpu_s = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": k / cpu_s, "unit": "particle-steps/s", "cores": 1, "kind": "oracle",
                                "sample": f"{k} particles of the workload, one oracle push ({cpu_s:.1f} s, numpy)"}
    g.close()
    print(json.dumps(line), flush=True)


def measure_batched(hyb, wl, steps, warmup, stream, flush, sampler, dev, strips="", split=""):
    """16 uneven 2D FP32 grids (sizes drawn with seed 3) plus the quasi-3D modes m = 0, 1, 2
    on 2048 x 512 complex fields, advanced together as one batch (CUDA-graph step)."""
    import numpy as np
    import torch
    rng = np.random.default_rng(3)
    descs, bufs, cells, alg_bytes = [], [], 0, 0
    sizes = [(int(rng.choice([512, 1024, 2048, 4096])), int(rng.choice([128, 256, 512, 1024]))) for _ in range(16)]
    for i, (n1, n2) in enumerate(sizes):
        w = wl.Workload(f"b{i}", 2, n1, n2, dx1=0.2, dx2=0.2, dt=0.08, precision=32, filt_kc=0.5, filt_w=0.2,
                        seed=100 + i)
        descs.append(hyb.desc_from_workload(w))
        E0, B0 = wl.band_limited_fields(w)
        J0, _ = wl.band_limited_fields(w.scaled(seed=w.seed + 50))
        mk = lambda arrs: [torch.from_numpy(a.astype(np.float32)).to(dev) for a in arrs]
        bufs.append((mk(E0), mk(B0), mk(J0)))
        cells += n1 * n2
        alg_bytes += 60 * n1 * n2
    nz, nr = 2048, 512
    for m in (0, 1, 2):
        dt = 0.9 * 2 / np.sqrt(np.pi ** 2 / 0.2 ** 2 + (4 * m * m + 6) / 0.2 ** 2)
        descs.append(hyb.make_desc(dims=20, n1=nz, n2=nr, dx1=0.2, dx2=0.2, dt=min(0.08, dt), precision=32,
                                   filt_kc=0.5, filt_w=0.2, azimuthal_m=m))
        cf = lambda s_: [(torch.randn(nr, nz, device=dev) + 1j * torch.randn(nr, nz, device=dev)).to(torch.complex64) * s_
                         for _ in range(3)]
        bufs.append((cf(1e-3), cf(1e-3), cf(1e-3)))
        cells += nz * nr
        alg_bytes += 120 * nz * nr
    b = hyb.Batch(descs, stream)
    for i, (E, B, J) in enumerate(bufs):
        b.bind(i, E, B, J)
    t0 = time.perf_counter()
    if strips:
        for kv in strips.split(","):
            n1_, h_ = (int(v) for v in kv.split(":"))
            b.set_rows_per_strip(n1_, h_)
        if split:
            b.set_role_ctas([int(v) for v in split.split(",")])
    else:
        b.tune(5)
    tune_s = time.perf_counter() - t0
    ms = time_steps(lambda: b.advance(1), steps, warmup, stream, flush, sampler)
    lps = b.launches_per_step
    single = b.single_launch
    # the other form of the step (graph of launches vs one persistent launch), timed the same way
    other = None
    try:
        b.single_launch = not single
    except hyb.HybError:
        pass
    else:
        ms_o = time_steps(lambda: b.advance(1), steps, warmup, stream, flush, sampler)
        other = {"form": "single persistent launch" if not single else "graph of launches",
                 "ms_per_step": ms_o, "launches_per_step": b.launches_per_step}
        b.single_launch = single
    config = {"workload": "batched_16x2d_uneven_plus_quasi3d_m012_2048x512", "instances_2d": sizes,
              "quasi3d_modes": [0, 1, 2], "quasi3d_grid": [nz, nr],
              "step": "single persistent launch" if single else "graph of launches",
              "role_ctas": dict(zip(("n1=4096", "n1=512", "n1=1024", "n1=2048", "quasi3d"), b.role_ctas())),
              "role_ms": dict(zip(("n1=4096", "n1=512", "n1=1024", "n1=2048", "quasi3d"), b.role_ms())),
              "other_form": other,
              "strips": "set by --batch-strips / --batch-split" if strips else "autotuned", "autotune_s": tune_s,
              "rows_per_strip": {n1: b.rows_per_strip(n1) for n1 in (512, 1024, 2048, 4096)},
              "current": "band-limited random J (no deposit in the timed step)",
              "l2": "flushed between timed steps (256 MB write)"}
    b.close()
    return ms, cells, alg_bytes, lps, config


def measure_3d(hyb, wl, steps, warmup, stream, flush, sampler, dev, rows3d=256):
    """3D FP32 drifting-plasma grid: the x1 transform as radix FFT (path 1) and as split-BF16
    DFT-GEMM (path 3), both timed, per-field error of each after 3 steps against the FP64 GPU
    path from the same initial state; and the radix path with k1-resident E, B."""
    import torch
    w = wl.DRIFT_PLASMA_3D
    if rows3d != w.n2:
        w = w.scaled(n2=rows3d, n3=rows3d, name=f"drift_plasma_3d_1024x{rows3d}x{rows3d}_f32")
    E0, B0 = wl.band_limited_fields(w)
    J0, _ = wl.band_limited_fields(w.scaled(seed=w.seed + 50))
    arrs = list(E0) + list(B0) + list(J0)
    x1 = x1_compare(hyb, w, arrs, stream, flush, sampler, steps, warmup, dev)
    g = hyb.Grid(hyb.desc_from_workload(w, path=1), stream)
    F = [torch.from_numpy(a).to(device=dev, dtype=torch.float32) for a in arrs]
    g.bind(F[0:3], F[3:6], F[6:9])
    g.set_resident(True)
    x1["ms_path1_resident"] = time_steps(lambda: g.advance(1), steps, warmup, stream, flush, sampler)
    x1["launches_path1_resident"] = g.launches_per_step
    g.close()
    del F
    best = min((1, 3, 4), key=lambda p_: x1[f"ms_path{p_}"])
    config = {"workload": w.name, "path": {1: "three-pass radix FFT", 3: "three-pass DFT-GEMM (2 BF16 parts)",
                                           4: "three-pass DFT-GEMM (3 BF16 parts)"}[best],
              "x1_transform": x1, "current": "band-limited random J",
              "l2": "flushed between timed steps (256 MB write)"}
    return x1[f"ms_path{best}"], w.cells, 60 * w.cells, x1[f"launches_path{best}"], config


def run_other(args):
    """Measurement lines for the non-headline configurations (same JSON keys)."""
    import numpy as np
    import torch
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    from paper_1502_01376_gb300 import build, hyb, workloads as wl
    build.build()
    stream = torch.cuda.current_stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    sampler = ClockSampler(0)
    sampler.start()
    time.sleep(0.5)
    peak, src = peaks()
    extra = {}
    if args.workload == "batched":
        ms, cells, alg_bytes, lps, extra["config"] = measure_batched(hyb, wl, args.steps, args.warmup, stream, flush,
                                                                     sampler, dev, args.batch_strips, args.batch_split)
        launches = lps * args.steps
        dtype = "f32"
    elif args.workload == "3d":
        ms, cells, alg_bytes, lps, extra["config"] = measure_3d(hyb, wl, args.steps, args.warmup, stream, flush,
                                                                sampler, dev, args.rows3d)
        launches = lps * args.steps
        dtype = "f32"
    elif args.workload == "x1_sweep":
        rows_out = []
        for n1 in (int(v) for v in args.sweep_n1.split(",")):
            n2 = args.sweep_cells // n1
            w = wl.Workload(f"sweep_{n1}", 2, n1, n2, dx1=0.2, dx2=0.2, dt=0.08, precision=32, filt_kc=0.5,
                            filt_w=0.2, seed=3)
            gen = np.random.default_rng(n1)
            arrs = [gen.standard_normal(w.shape) * 1e-3 for _ in range(9)]
            r = x1_compare(hyb, w, arrs, stream, flush, None, args.steps, args.warmup, dev)
            r["n1"], r["n2"] = n1, n2
            rows_out.append(r)
        best_row = rows_out[0]
        best = min((1, 3, 4), key=lambda p_: best_row[f"ms_path{p_}"])
        cells, alg_bytes = args.sweep_cells, 60 * args.sweep_cells
        ms = best_row[f"ms_path{best}"]
        launches = best_row[f"launches_path{best}"] * args.steps
        extra["config"] = {"workload": f"x1_transform_sweep_2d_{args.sweep_cells}_cells_f32",
                           "value_at": f"n1 = {rows_out[0]['n1']}",
                           "sweep": rows_out, "current": "random J", "l2": "flushed between timed steps"}
        dtype = "f32"
    else:
        w = wl.VACUUM_BEAM
        g = hyb.Grid(hyb.desc_from_workload(w), stream)
        E0, B0 = wl.band_limited_fields(w)
        mk = lambda arrs: [torch.from_numpy(a).to(dev) for a in arrs]
        J = [torch.zeros(w.shape, dtype=torch.float64, device=dev) for _ in range(3)]
        g.bind(mk(E0), mk(B0), J)
        p = wl.make_particles(w)
        cell, o0, o1, v3 = wl.ballistic_move(w, p, 0)
        g.deposit(torch.from_numpy(cell).to(dev), torch.from_numpy(o0).to(dev), torch.from_numpy(o1).to(dev),
                  torch.from_numpy(v3).to(dev), torch.from_numpy(p.q).to(dev), w.shape_order)
        g.check()
        cells, alg_bytes = w.cells, 120 * w.cells
        ms = time_steps(lambda: g.advance(1), args.steps, args.warmup, stream, flush, sampler)
        launches = g.launches_per_step * args.steps
        extra["config"] = {"workload": w.name, "path": "three-pass FP64", "l2": "flushed between timed steps"}
        dtype = "f64"
        g.close()
    sampler.stop()
    achieved = alg_bytes / (ms / 1e3) / 1e9
    line = {"metric": METRIC, "value": cells / (ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": dtype, "data": "synthetic",
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": None, "peak_source": src, "kernel": "whole step", "bytes_per_launch": alg_bytes},
            "gpu_launches": launches, "clocks": sampler.summary()}
    line.update(extra)
    print(json.dumps(line), flush=True)


def measure_resident(hyb, w, E, B, J, steps, warmup, stream, flush, fused_kms, peak):
    """The same workload with k1-resident E, B (hyb_set_resident): per step the forward FFT of
    j only, the k1-space updates and the inverse FFT of E, B into the real arrays (the fields a
    particle gather reads), against the fused single pass that transforms E, B, j every step."""
    Ec, Bc, Jc = [t.clone() for t in E], [t.clone() for t in B], [t.clone() for t in J]
    g = hyb.Grid(hyb.desc_from_workload(w, path=0), stream)
    g.bind(Ec, Bc, Jc)
    g.set_resident(True)
    ms = time_steps(lambda: g.advance(1), steps, warmup, stream, flush, None)
    out = {"value": w.cells / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "steps": steps,
           "kernel": g.step_kernel, "launches_per_step": g.launches_per_step,
           "row_transforms_per_step": {"resident": "3 forward (j) + 6 inverse (E, B)",
                                       "fused_single_pass": "8 forward + 5 inverse (E1..3, B2, B3, j1..3; B1 "
                                                            "in real space)"},
           "algorithmic_bytes_per_cell": {"resident_three_pass": 156, "fused_single_pass": BYTES_PER_CELL_STEP},
           "fused_kernel_ms": fused_kms,
           "achieved_gbs": 156 * w.cells / (ms / 1e3) / 1e9}
    out["frac"] = out["achieved_gbs"] / peak
    g.close()
    return out


def measure_configs(hyb, wl, stream, flush, dev):
    """Short measurements of the batched, 3D and surrogate configurations in the same run
    (each also has its own --workload mode with the full step count)."""
    import torch
    from paper_1502_01376_gb300 import surrogate as sg
    peak, src = peaks()
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    time.sleep(0.3)
    out = {}
    for name, fn in (("batched", lambda: measure_batched(hyb, wl, 20, 3, stream, flush, sampler, dev)),
                     ("3d", lambda: measure_3d(hyb, wl, 10, 3, stream, flush, sampler, dev))):
        ms, cells, alg_bytes, lps, config = fn()
        achieved = alg_bytes / (ms / 1e3) / 1e9
        out[name] = {"value": cells / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "dtype": "f32",
                     "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                                  "frac": achieved / peak, "peak_source": src, "kernel": "whole step",
                                  "bytes_per_launch": alg_bytes},
                     "launches_per_step": lps, "config": config}
        torch.cuda.empty_cache()
    # PIC step (push, deposit, advance with B time-centred) on the Table 1 box, with the fields
    # in real space (two advances per step) and k1-resident (B^n from the spectra)
    from paper_1502_01376_gb300 import pic
    out["pic_table1"] = {}
    for res in (False, True):
        pic.run(pic.TABLE1, steps=20, every=20, resident=res)                  # warm
        h = pic.run(pic.TABLE1, steps=400, every=400, resident=res)
        out["pic_table1"]["resident" if res else "real_space"] = {"ms_per_step": 1e3 * h.seconds / h.steps,
                                                                  "steps": h.steps}
    out["pic_table1"]["config"] = {"grid": [pic.TABLE1.n1, pic.TABLE1.n2], "particles_per_cell": 2 * pic.TABLE1.ppc,
                                   "timing": "wall clock over 400 steps on the host (one diagnostics call at the end)"}
    out["surrogate"] = measure_surrogate(hyb, sg, 3000, 20, sampler)
    out["surrogate"]["metric"] = "NCI surrogate training samples/s (MLP 6->256x4->1, BF16 operands, FP32 accumulation)"
    sampler.stop()
    out["clocks"] = sampler.summary()
    return out


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "surrogate":
        return run_surrogate(args)
    if args.workload == "push":
        return run_push(args)
    if args.workload != "drift_plasma":
        return run_other(args)
    import numpy as np
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    from paper_1502_01376_gb300 import build, hyb, workloads as wl
    if rank == 0 or ws == 1:
        build.build()
    if ws > 1:
        torch.distributed.barrier()
    w = wl.DRIFT_PLASMA
    if args.n1 != w.n1:
        w = w.scaled(n1=args.n1, n2=w.cells // args.n1, name=f"drift_plasma_2d_{args.n1}x{w.cells // args.n1}_f32")
    stream = torch.cuda.current_stream()
    grid = hyb.Grid(hyb.desc_from_workload(w, path=0), stream)
    E0, B0 = wl.band_limited_fields(w)
    E = [torch.from_numpy(a.astype(np.float32)).to(dev) for a in E0]
    B = [torch.from_numpy(a.astype(np.float32)).to(dev) for a in B0]
    J = [torch.zeros(w.shape, dtype=torch.float32, device=dev) for _ in range(3)]
    grid.bind(E, B, J)
    if args.quick:
        args.no_extras = True
        J0, _ = wl.band_limited_fields(w.scaled(seed=w.seed + 7))
        for c in range(3):
            J[c].copy_(torch.from_numpy(J0[c].astype(np.float32)))
        deposit_ms, n_particles = None, 0
    else:
        # J^{n+1/2} of the drifting plasma, deposited once (not part of the timed step)
        cell, off0, off1, v3, q = wl.plasma_move_torch(w, dev)
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        grid.deposit(cell, off0, off1, v3, q, w.shape_order)       # first call loads the kernel
        t0.record()
        grid.deposit(cell, off0, off1, v3, q, w.shape_order)
        t1.record()
        grid.check()
        deposit_ms = t0.elapsed_time(t1)
        n_particles = int(q.numel())
        del cell, off0, off1, v3, q
        torch.cuda.empty_cache()

    cells = w.cells
    # the accuracy check starts from this initial state (the timed loop keeps
    # driving the fields with the same current, which is not a physical run)
    E_init = [t.clone() for t in E] if not args.no_extras else None
    B_init = [t.clone() for t in B] if not args.no_extras else None
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MB > L2
    for _ in range(args.warmup):
        grid.advance(1)
    torch.cuda.synchronize()
    K = args.steps
    ek = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    for a, b in ek:          # torch creates the CUDA event on first record; the library records them later
        a.record(stream)
        b.record(stream)
    es = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    sampler = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    if sampler:
        sampler.start()
        time.sleep(0.5)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    if sampler:
        sampler.mark(True)
    # pass 1, the value: K steps bracketed by events, nothing recorded inside a step
    wall0 = time.perf_counter()
    for i in range(K):
        flush.zero_()
        es[i][0].record(stream)
        grid.advance(1)
        es[i][1].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    step_ms = [a.elapsed_time(b) for a, b in es]
    # pass 2, the roofline: K more steps with the library recording events around the kernel
    # itself on the stream it launches on
    for i in range(K):
        flush.zero_()
        grid.set_kernel_events(*ek[i])
        grid.advance(1)
    torch.cuda.synchronize()
    grid.set_kernel_events(None, None)
    kern_ms = [a.elapsed_time(b) for a, b in ek]
    if ws > 1:
        torch.distributed.barrier()
    if sampler:
        sampler.mark(False)
        sampler.stop()
    ms = statistics.mean(step_ms)
    kms = statistics.mean(kern_ms)
    ms, kms, value = replica_aggregate(ms, kms, cells, ws, dev)
    launches = grid.launches_per_step * K

    extras = {}
    if rank == 0 and not args.no_extras:
        # accuracy of the FP32 step against the FP64 GPU path from identical inputs
        g64 = hyb.Grid(hyb.desc_from_workload(w, precision=64, path=1), stream)
        E64 = [t.double() for t in E_init]
        B64 = [t.double() for t in B_init]
        J64 = [t.double() for t in J]
        g64.bind(E64, B64, J64)
        Ec = [t.clone() for t in E_init]
        Bc = [t.clone() for t in B_init]
        g32 = hyb.Grid(hyb.desc_from_workload(w, path=0), stream)
        g32.bind(Ec, Bc, J)
        nacc, ndrift = 10, 1000
        g32.advance(nacc)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        g64.advance(nacc)
        e1.record()
        torch.cuda.synchronize()
        ms64 = e0.elapsed_time(e1) / nacc
        names = ["E1", "E2", "E3", "B1", "B2", "B3"]

        def field_errs():
            return [float(torch.linalg.norm(a.double() - b) / torch.linalg.norm(b)) for a, b in zip(Ec + Bc, E64 + B64)]
        errs = field_errs()
        extras["accuracy"] = {"steps": nacc, "from": "initial state, same FP32-rounded inputs and J",
                              "max_rel_err_vs_fp64_gpu_path": max(errs),
                              "per_field": dict(zip(names, errs))}
        # the long-run drift of the same pair of runs (reported, not gated: the FP32 phase
        # error of the waves grows with the step count)
        g32.advance(ndrift - nacc)
        g64.advance(ndrift - nacc)
        torch.cuda.synchronize()
        errs_d = field_errs()
        extras["drift"] = {"steps": ndrift, "from": "the same initial state and J as accuracy",
                           "max_rel_err_vs_fp64_gpu_path": max(errs_d), "per_field": dict(zip(names, errs_d))}
        extras["fp64_gpu_path"] = {"value": cells / (ms64 / 1e3), "unit": UNIT, "ms_per_step": ms64}
        g64.close()
        g32.close()
        del E64, B64, J64, Ec, Bc
        # end to end through the public API with host buffers (pinned)
        Eh = [t.cpu().pin_memory() for t in E]
        Bh = [t.cpu().pin_memory() for t in B]
        Jh = [t.cpu().pin_memory() for t in J]
        for _ in range(3):
            grid.advance_host(Eh, Bh, Jh, 1)
        e2e_t = []
        for _ in range(20):
            tt = time.perf_counter()
            grid.advance_host(Eh, Bh, Jh, 1)
            e2e_t.append(time.perf_counter() - tt)
        e2e_s = statistics.mean(e2e_t)
        extras["e2e"] = {"value": cells / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 9 * 4 * cells,
                         "d2h_bytes_per_step": 6 * 4 * cells, "ms_per_step": 1e3 * e2e_s,
                         "ms_median": 1e3 * statistics.median(e2e_t), "ms_max": 1e3 * max(e2e_t), "calls": len(e2e_t)}
        if ws == 1:
            extras["cpu_baseline"] = cpu_baseline_sample(w)
        extras["k1_resident"] = measure_resident(hyb, w, E, B, J, min(K, 200), max(3, args.warmup), stream, flush,
                                                 kms, peaks()[0])
        if not args.no_configs:
            extras["configs"] = measure_configs(hyb, wl, stream, flush, dev)
    # FP64 diagnostics of the final state (energies, max |div B|, Gauss residual): synchronous call,
    # the first one allocates its scratch
    grid.diag()
    tt = time.perf_counter()
    grid.diag()
    diag_ms = 1e3 * (time.perf_counter() - tt)
    if rank == 0:
        peak, src = peaks()
        achieved = BYTES_PER_CELL_STEP * cells / (kms / 1e3) / 1e9
        kname = grid.step_kernel
        tr = profiled_traffic(cells, kname)
        traffic = tr["bytes"] if tr else None
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": K, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": w.name, "n1": w.n1, "n2": w.n2, "dx": w.dx1, "dt": w.dt,
                       "correct_j1": True, "filter_kc": w.filt_kc, "filter_w": w.filt_w,
                       "particles_deposited": n_particles, "deposit_ms": deposit_ms, "diag_ms": diag_ms,
                       "path": "fused" if grid.path == 2 else "three-pass",
                       "l2": "flushed between timed steps (256 MB write)", "parallelism": f"replicas x{ws}"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "traffic_detail": tr, "peak_source": src,
                         "kernel": kname,
                         "kernel_ms": kms, "bytes_per_launch": BYTES_PER_CELL_STEP * cells,
                         "kernel_timing": "events around the kernel on its stream, a second pass of K steps"},
            "gpu_launches": launches,
            "wall_s_timed": wall,
        }
        if kname == "k_fused_tm":
            # the same kernel against the FP32 pipes: its arithmetic counted from the factorization
            line["roofline"]["fp32_view"] = fp32_view(cells, kms, sampler)
        if sampler:
            line["clocks"] = sampler.summary()
        if "e2e" in extras:
            line["e2e"] = extras.pop("e2e")
        if "cpu_baseline" in extras:
            line["cpu_baseline"] = extras.pop("cpu_baseline")
        line.update(extras)
        print(json.dumps(line), flush=True)
    grid.close()
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
