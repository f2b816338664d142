"""Pins of the oracle against values the paper prints (tests/golden/paper_printed_values.txt)."""
import math
import os

import numpy as np
import pytest

from oracle import nci

HERE = os.path.dirname(os.path.abspath(__file__))


def golden():
    vals = {}
    with open(os.path.join(HERE, "golden", "paper_printed_values.txt")) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                k, v = (s.strip() for s in line.split("="))
                vals[k] = float(v)
    return vals


def test_table1_time_step_is_the_printed_one():
    g = golden()
    assert g["table1_wp_dt_over_dx1"] * g["table1_kp_dx1"] == pytest.approx(g["fig_embeam_dt"])
    assert g["table1_box_kp_l"] / g["table1_kp_dx1"] == pytest.approx(256)


def test_courant_square_cells_printed_value(orc):
    """Sec. 2.2 prints 0.537 (three digits) for dx1 = dx2."""
    g = golden()
    for dx in (0.1, 0.2, 1.0):
        lim = orc.courant(orc.grid(dims=2, n1=8, n2=8, dx1=dx, dx2=dx, dt=0.01 * dx))
        assert lim / dx == pytest.approx(g["courant_square_cells_dt_over_dx1"], abs=5e-4)


def _nci_params(g, **kw):
    return nci.NciParams(dt=g["fig_embeam_dt"], dx1=g["table1_kp_dx1"], dx2=g["table1_kp_dx2"],
                         gamma=g["table1_gamma"], wp2=g["table1_density_n_over_np"], order=2, **kw)


def test_bump_removes_zero_zero_nci_modes():
    """Sec. 4: with the printed k1 modification the (0, 0) modes have zero
    theoretical growth at the Table 1 parameters; without it they grow."""
    g = golden()
    plain = _nci_params(g)
    bump = _nci_params(g, kmod_l=g["bump_k1l_over_kg1"], kmod_u=g["bump_k1u_over_kg1"],
                       kmod_max=g["bump_dkmax_over_kg1"])
    _, _, G0 = nci.growth_scan(plain, 0, 0, 64, 64)
    k1s, _, G1 = nci.growth_scan(bump, 0, 0, 64, 64)
    assert G0.max() > 1e-2
    assert G1.max() == pytest.approx(g["bump_zero_zero_growth"], abs=1e-10)
    # the unmodified growth sits inside the modified k1 range
    i = np.unravel_index(G0.argmax(), G0.shape)[0]
    kg1 = 2 * math.pi / g["table1_kp_dx1"]
    assert g["bump_k1l_over_kg1"] <= k1s[i] / kg1 <= g["bump_k1u_over_kg1"]
