"""Surrogate network kernels (forward, backward, Adam) against the FP64
oracle, training on the GPU root solver's data, and what the trained network
gains: the filter cutoff and time step it picks give less NCI growth (checked
by the root solver) than the unfiltered run, and it scans settings faster."""
import time

import numpy as np
import pytest

from oracle import mlp as omlp

from gpu_util import hyb_module, need_gpu, torch

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("width,depth,B", [(32, 2, 100), (256, 4, 128)])
def test_mlp_forward_and_gradients_match_oracle(width, depth, B):
    need_gpu()
    hyb = hyb_module()
    rng = np.random.default_rng(width)
    p = hyb.mlp_init_params(6, width, depth, seed=width)
    p[-1:] = 0.1
    net = hyb.MLP(6, width, depth, params=p)
    x = rng.uniform(-1, 1, (B, 6)).astype(np.float32)
    t = rng.uniform(0, 2, B).astype(np.float32)
    xg, tg = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    y = net.forward(xg).cpu().numpy()
    yo = omlp.forward(p.astype(np.float64), x, 6, width, depth)[0]
    assert np.linalg.norm(y - yo) / np.linalg.norm(yo) < 2e-3
    g, loss = net.gradients(xg, tg)
    go, lo = omlp.gradients(p.astype(np.float64), x, t, 6, width, depth)
    assert abs(loss - lo) / lo < 2e-3
    assert np.linalg.norm(g - go) / np.linalg.norm(go) < 5e-3
    # and against the unrounded FP64 network: only the BF16 operand rounding differs
    gx, _ = omlp.gradients(p.astype(np.float64), x, t, 6, width, depth, rnd=False)
    assert np.linalg.norm(g - gx) / np.linalg.norm(gx) < 5e-2
    net.close()


def test_adam_step_matches_oracle_update():
    need_gpu()
    hyb = hyb_module()
    rng = np.random.default_rng(3)
    p = hyb.mlp_init_params(6, 16, 2, seed=3)
    net = hyb.MLP(6, 16, 2, params=p)
    x = torch.from_numpy(rng.uniform(-1, 1, (64, 6)).astype(np.float32)).cuda()
    t = torch.from_numpy(rng.uniform(0, 1, 64).astype(np.float32)).cuda()
    g, _ = net.gradients(x, t)
    lr = 1e-2
    net.train_step(x, t, lr)
    p1 = net.get_params()
    # first Adam step with bias correction: m_hat = g, v_hat = g^2 -> step = lr g / (|g| + eps)
    expect = p - lr * g / (np.abs(g) + 1e-8)
    assert np.max(np.abs(p1 - expect)) < 1e-5
    net.close()


def test_surrogate_trains_and_picks_settings_with_less_growth():
    need_gpu()
    hyb = hyb_module()
    from paper_1502_01376_gb300 import surrogate as sg
    X, y, kept, n = sg.dataset(60000, seed=11)
    assert kept < n                                # Courant-unstable samples are flagged out
    Xv, yv, _, _ = sg.dataset(8000, seed=12)
    net = hyb.MLP(6, 256, 4, seed=5)
    hist = sg.train(net, X, y, steps=1500, batch=8192, lr=2e-3, seed=1)
    assert hist[-50:].mean() < 0.3 * hist[:10].mean()
    pred = net.forward(Xv)
    mse = float(torch.mean((pred - yv) ** 2))
    var = float(torch.var(yv))
    assert mse < 0.5 * var, (mse, var)
    # pick the cutoff and dt for the drifting-plasma run (gamma 50, square cells)
    dts = np.arange(0.2, 0.51, 0.05)
    kcs = np.arange(0.3, 1.01, 0.1)
    res = sg.pick(net, 50.0, 1.0, dts, kcs)
    confirmed = sg.max_growth_solver([res["dt_dx1"]], [1.0], [50.0], [res["kc"]])[0]
    unfiltered = sg.max_growth_solver([0.5], [1.0], [50.0], [1.0])[0]
    assert confirmed <= unfiltered
    # pruned by the surrogate, judged by the root solver on the 8 most promising candidates
    resv = sg.pick(net, 50.0, 1.0, dts, kcs, verify=8)
    confirmed_v = sg.max_growth_solver([resv["dt_dx1"]], [1.0], [50.0], [resv["kc"]])[0]
    assert confirmed_v <= unfiltered
    assert confirmed_v <= confirmed + 2e-3
    t0 = time.perf_counter()
    sg.max_growth_solver(res["all_dt"], np.ones(res["candidates"]), np.full(res["candidates"], 50.0), res["all_kc"])
    t_solver = time.perf_counter() - t0
    print(f"pick {res['dt_dx1']:.2f} {res['kc']:.2f} predicted {res['predicted']:.4f} confirmed {confirmed:.4f} "
          f"unfiltered {unfiltered:.4f}; scan {res['seconds']:.4f} s vs root solver {t_solver:.4f} s")
    net.close()
