"""Pins of the oracle's charge-conserving deposit (Sec. 2.3).

* B-spline shape factors: partition of unity, first moment x, second moment
  (l+1)/12 for l >= 2 (quadratic reproduction) and f(1-f) for l = 1;
* the finite-difference continuity equation of Eq. continuity (written out
  here directly from the paper) holds to rounding for shapes l = 1, 2, 3 in
  2D and 3D;
* total current: sum of j dV equals q v for every particle (first moment);
* a particle at rest deposits nothing.
"""
import numpy as np
import pytest

from paper_1502_01376_gb300 import workloads as wl


@pytest.mark.parametrize("order", [1, 2, 3])
def test_shape_moments(orc, order):
    rng = np.random.default_rng(order)
    for x in rng.uniform(-3, 3, 25):
        i = np.arange(int(np.floor(x)) - 4, int(np.floor(x)) + 6)
        s = np.array([orc.shape(order, x - ii) for ii in i])
        assert np.sum(s) == pytest.approx(1.0, abs=1e-14)
        assert np.sum((i - x) * s) == pytest.approx(0.0, abs=1e-14)
        m2 = np.sum((i - x) ** 2 * s)
        if order >= 2:       # degree >= 2 splines reproduce quadratics: variance (l+1)/12
            assert m2 == pytest.approx((order + 1) / 12.0, abs=1e-14)
        else:                # linear weighting: f (1 - f) with f the fractional position
            f = x - np.floor(x)
            assert m2 == pytest.approx(f * (1 - f), abs=1e-14)
        assert np.all(s >= 0)


def _random_particles(d, n, ext, rng, max_step=0.95):
    cell = np.stack([rng.integers(0, e, n) for e in ext], axis=1).astype(np.int32)
    off0 = rng.uniform(0, 1, (n, d))
    off1 = off0 + rng.uniform(-max_step, max_step, (n, d))
    q = rng.uniform(-1, 1, n)
    v3 = rng.uniform(-0.5, 0.5, n)
    return (np.ascontiguousarray(cell), np.ascontiguousarray(off0), np.ascontiguousarray(off1),
            np.ascontiguousarray(v3), np.ascontiguousarray(q))


@pytest.mark.parametrize("order", [1, 2, 3])
def test_continuity_2d(orc, order):
    n1, n2, dx1, dx2, dt = 16, 12, 0.2, 0.3, 0.07
    g = orc.grid(n1=n1, n2=n2, dx1=dx1, dx2=dx2, dt=dt)
    rng = np.random.default_rng(10 + order)
    cell, off0, off1, v3, q = _random_particles(2, 40, (n1, n2), rng)
    J = orc.deposit(g, cell, off0, off1, v3, q, order)
    r0 = orc.charge(g, cell, off0, q, order)
    r1 = orc.charge(g, cell, off1, q, order)
    # Eq. continuity: (rho^{n+1}-rho^n)/dt + (j1[i1+1/2]-j1[i1-1/2])/dx1 + (j2[i2+1/2]-j2[i2-1/2])/dx2 = 0
    div = (J[0] - np.roll(J[0], 1, axis=1)) / dx1 + (J[1] - np.roll(J[1], 1, axis=0)) / dx2
    res = (r1 - r0) / dt + div
    assert np.max(np.abs(res)) < 1e-12 * np.max(np.abs(r0)) / dt
    # total current = sum q v (x1, x2) and q v3
    dV = dx1 * dx2
    assert np.sum(J[0]) * dV == pytest.approx(np.sum(q * (off1[:, 0] - off0[:, 0]) * dx1 / dt), rel=1e-12)
    assert np.sum(J[1]) * dV == pytest.approx(np.sum(q * (off1[:, 1] - off0[:, 1]) * dx2 / dt), rel=1e-12)
    assert np.sum(J[2]) * dV == pytest.approx(np.sum(q * v3), rel=1e-12)


@pytest.mark.parametrize("order", [1, 2, 3])
def test_continuity_3d(orc, order):
    n1, n2, n3 = 10, 8, 9
    dx = (0.2, 0.25, 0.3)
    dt = 0.05
    g = orc.grid(dims=3, n1=n1, n2=n2, n3=n3, dx1=dx[0], dx2=dx[1], dx3=dx[2], dt=dt)
    rng = np.random.default_rng(20 + order)
    cell, off0, off1, v3, q = _random_particles(3, 20, (n1, n2, n3), rng)
    J = orc.deposit(g, cell, off0, off1, v3, q, order)
    r0 = orc.charge(g, cell, off0, q, order)
    r1 = orc.charge(g, cell, off1, q, order)
    div = ((J[0] - np.roll(J[0], 1, axis=2)) / dx[0] + (J[1] - np.roll(J[1], 1, axis=1)) / dx[1]
           + (J[2] - np.roll(J[2], 1, axis=0)) / dx[2])
    res = (r1 - r0) / dt + div
    assert np.max(np.abs(res)) < 1e-12 * np.max(np.abs(r0)) / dt
    dV = dx[0] * dx[1] * dx[2]
    for a in range(3):
        assert np.sum(J[a]) * dV == pytest.approx(np.sum(q * (off1[:, a] - off0[:, a]) * dx[a] / dt), rel=1e-12)


def test_particle_at_rest_deposits_nothing(orc):
    g = orc.grid(n1=8, n2=8, dx1=0.1, dx2=0.1, dt=0.05)
    cell = np.array([[3, 4]], dtype=np.int32)
    off = np.array([[0.3, 0.6]])
    J = orc.deposit(g, cell, off, off.copy(), np.zeros(1), np.array([1.0]), 2)
    for j in J:
        assert np.max(np.abs(j)) == 0.0


def test_charge_total_and_periodic_wrap(orc):
    g = orc.grid(n1=8, n2=6, dx1=0.1, dx2=0.2, dt=0.05)
    cell = np.array([[0, 0], [7, 5]], dtype=np.int32)
    off = np.array([[0.1, 0.2], [0.9, 0.95]])
    q = np.array([1.0, -2.0])
    for order in (1, 2, 3):
        rho = orc.charge(g, cell, off, q, order)
        assert np.sum(rho) * 0.1 * 0.2 == pytest.approx(-1.0, abs=1e-14)


def test_beam_workload_deposit_is_x1_current(orc):
    """Beam particles of config 1 move only along x1: j2 = j3 = 0 and the
    net x1 current equals N q v1."""
    w = wl.VACUUM_BEAM.scaled(n_particles=64)
    g = orc.grid(n1=w.n1, n2=w.n2, dx1=w.dx1, dx2=w.dx2, dt=w.dt)
    p = wl.make_particles(w)
    cell, off0, off1, v3 = wl.ballistic_move(w, p, 3)
    J = orc.deposit(g, cell, off0, off1, v3, p.q, w.shape_order)
    assert np.max(np.abs(J[1])) == 0.0 and np.max(np.abs(J[2])) == 0.0
    assert np.sum(J[0]) * w.dx1 * w.dx2 == pytest.approx(64 * w.beam_q * w.beam_v1, rel=1e-12)
