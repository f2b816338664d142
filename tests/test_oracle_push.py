"""Pins of the particle-step oracle (gather with the momentum-conserving
interpolation of the Appendix, relativistic Boris push) against facts that do not
come from the oracle itself: B-spline identities, exact solutions of the push in
uniform fields, and convergence to the exact relativistic trajectory."""
import numpy as np
import pytest

from oracle import push as P


def _particles(rng, n, shape):
    cell = np.stack([rng.integers(0, s, n) for s in shape], axis=1)
    off = rng.uniform(0.0, 1.0, (n, len(shape)))
    return cell, off


@pytest.mark.parametrize("order", [1, 2, 3])
@pytest.mark.parametrize("dims", [2, 3])
def test_gather_constant_field_is_exact(order, dims):
    """Partition of unity: sum_i s_l(x - i) = 1, for every staggering."""
    rng = np.random.default_rng(order + 10 * dims)
    shape = (8, 6, 5)[:dims]
    vals = rng.standard_normal(6)
    fields = [np.full(shape[::-1], v) for v in vals]
    cell, off = _particles(rng, 200, shape)
    out = P.gather(fields, cell, off, order)
    assert np.max(np.abs(out - vals[None, :])) < 1e-13


@pytest.mark.parametrize("order", [1, 2, 3])
def test_gather_reproduces_linear_fields(order):
    """Centred B-splines reproduce linear functions: sum_i (i + sigma) s_l(x - i - sigma) = x.
    Each component holds the x1 (or x2) coordinate of its own staggered points."""
    rng = np.random.default_rng(order)
    n1, n2 = 32, 24
    i1 = np.arange(n1)[None, :].repeat(n2, 0).astype(float)
    i2 = np.arange(n2)[:, None].repeat(n1, 1).astype(float)
    st = P.STAGGER[2]
    fx = [i1 + 0.5 * s[0] for s in st]     # x1 coordinate of each component's points
    fy = [i2 + 0.5 * s[1] for s in st]
    cell = np.stack([rng.integers(4, n1 - 4, 300), rng.integers(4, n2 - 4, 300)], axis=1)
    off = rng.uniform(0.0, 1.0, (300, 2))
    x = cell + off
    assert np.max(np.abs(P.gather(fx, cell, off, order) - x[:, :1])) < 1e-12
    assert np.max(np.abs(P.gather(fy, cell, off, order) - x[:, 1:2])) < 1e-12


def test_gather_node_weights_closed_form():
    """A particle on an integer node: order 1 returns the node value; order 2 weights
    (1/8, 3/4, 1/8); order 3 weights (1/6, 2/3, 1/6).  E3 sits on integer nodes."""
    n1, n2 = 16, 8
    rng = np.random.default_rng(5)
    F = rng.standard_normal((n2, n1))
    fields = [np.zeros((n2, n1))] * 2 + [F] + [np.zeros((n2, n1))] * 3
    cell = np.array([[7, 3]])
    off = np.array([[0.0, 0.0]])
    w2 = {1: [0.0, 1.0, 0.0], 2: [0.125, 0.75, 0.125], 3: [1 / 6, 2 / 3, 1 / 6]}
    for order, w in w2.items():
        want = sum(w[a] * w[b] * F[3 + b - 1, 7 + a - 1] for a in range(3) for b in range(3))
        assert abs(P.gather(fields, cell, off, order)[0, 2] - want) < 1e-14


def test_gather_wraps_periodically():
    """A particle in the last cell sees the first column through the periodic wrap."""
    n1, n2 = 8, 4
    F = np.zeros((n2, n1))
    F[:, 0] = 1.0
    fields = [np.zeros((n2, n1))] * 2 + [F] + [np.zeros((n2, n1))] * 3
    out = P.gather(fields, np.array([[7, 1]]), np.array([[0.75, 0.0]]), 1)
    assert abs(out[0, 2] - 0.75) < 1e-14


def test_boris_pure_electric_kick_is_exact():
    rng = np.random.default_rng(1)
    u = rng.standard_normal((50, 3)) * 10
    E = rng.standard_normal((50, 3))
    qm = rng.choice([-1.0, 1.0], 50)
    un = P.boris(u, E, np.zeros((50, 3)), qm, 0.1)
    assert np.max(np.abs(un - (u + 0.1 * qm[:, None] * E))) < 1e-13


def test_boris_pure_magnetic_rotation_angle():
    """E = 0: |u| is kept and u turns about B by 2 atan(h |B| / gamma), in the sense of
    du/dt = (q/m) u x B / gamma."""
    u = np.array([[3.0, 0.0, 0.5]])
    B = np.array([[0.0, 0.0, 2.0]])
    dt, qm = 0.2, np.array([1.0])
    un = P.boris(u, np.zeros((1, 3)), B, qm, dt)
    gamma = np.sqrt(1.0 + np.sum(u * u))
    theta = 2.0 * np.arctan(0.5 * dt * 2.0 / gamma)
    assert abs(np.linalg.norm(un) - np.linalg.norm(u)) < 1e-13
    assert abs(un[0, 2] - 0.5) < 1e-14
    # u x B points to -x2 for u along +x1, B along +x3: clockwise in the (x1, x2) plane
    assert abs(np.arctan2(-un[0, 1], un[0, 0]) - theta) < 1e-13


def test_boris_exb_drift():
    """Crossed uniform fields with |E| << |B|: the mean velocity over many gyrations is
    E x B / |B|^2 (non-relativistic drift)."""
    E = np.array([[0.0, 1e-3, 0.0]])
    B = np.array([[0.0, 0.0, 1.0]])
    u = np.zeros((1, 3))
    dt, steps = 0.05, 40000
    v = np.zeros(3)
    for _ in range(steps):
        u = P.boris(u, E, B, np.array([1.0]), dt)
        v += u[0] / np.sqrt(1.0 + np.sum(u * u))
    v /= steps
    assert abs(v[0] - 1e-3) < 2e-5 and abs(v[1]) < 2e-5


def test_uniform_electric_field_second_order_to_exact_hyperbolic_motion():
    """From rest in a uniform E along x1 (q/m = 1): u(t) = E t exactly at the half steps
    and x(t) = (sqrt(1 + (E t)^2) - 1) / E; the leapfrog position error falls as dt^2."""
    Ex, T = 2.0, 4.0
    errs = []
    for n in (100, 200, 400):
        dt = T / n
        shape = (64, 4)
        fields = [np.full(shape[::-1], v) for v in (Ex, 0, 0, 0, 0, 0)]
        # u at -dt/2 from the exact solution, x at t = 0 in cell units (dx = 1)
        cell, off = np.array([[0, 0]]), np.array([[0.0, 0.5]])
        u = np.array([[-Ex * dt / 2, 0.0, 0.0]])
        x = 0.0
        for _ in range(n):
            cell, off, u, off_new, _, ok = P.push(fields, cell, off, u, np.array([1.0]), dt, np.array([1.0, 1.0]), 1)
            assert ok.all()
            x += off_new[0, 0] - off[0, 0]
            off = off_new
        exact = (np.sqrt(1.0 + (Ex * T) ** 2) - 1.0) / Ex
        assert abs(u[0, 0] - Ex * (T - dt / 2)) < 1e-12
        errs.append(abs(x - exact))
    assert 3.5 < errs[0] / errs[1] < 4.5 and 3.5 < errs[1] / errs[2] < 4.5


def test_renormalise_moves_particles_and_keeps_precision():
    cell = np.array([[0, 3], [7, 0], [2, 2], [1, 1]])
    off = np.array([[-0.25, 1.5], [1.25, -1.0], [0.5, 0.5], [2.5, 0.0]], dtype=np.float32)
    c, o, ok = P.renormalise(cell, off, (8, 4))
    assert ok.tolist() == [True, True, True, False]
    assert c.tolist() == [[7, 0], [0, 3], [2, 2], [1, 1]]
    assert o.dtype == np.float32
    assert o[:3].tolist() == [[0.75, 0.5], [0.25, 0.0], [0.5, 0.5]]
    # -tiny + 1 rounds to 1 in FP32: the particle stays in its cell at offset 0
    c, o, ok = P.renormalise(np.array([[3, 1]]), np.array([[-1e-9, 0.0]], dtype=np.float32), (8, 4))
    assert c.tolist() == [[3, 1]] and o.tolist() == [[0.0, 0.0]]


@pytest.mark.parametrize("order", [1, 2, 3])
def test_gather_reproduces_linear_fields_3d(order):
    """3D staggering: each component holding x1 + 2 x2 - x3 at its own points returns that
    combination at the particle (linear reproduction along every axis)."""
    rng = np.random.default_rng(30 + order)
    n1, n2, n3 = 16, 12, 10
    i3, i2, i1 = np.meshgrid(np.arange(n3), np.arange(n2), np.arange(n1), indexing="ij")
    st = P.STAGGER[3]
    fields = [(i1 + 0.5 * s[0]) + 2.0 * (i2 + 0.5 * s[1]) - (i3 + 0.5 * s[2]) for s in st]
    cell = np.stack([rng.integers(3, n - 3, 200) for n in (n1, n2, n3)], axis=1)
    off = rng.uniform(0.0, 1.0, (200, 3))
    x = cell + off
    want = x[:, 0] + 2.0 * x[:, 1] - x[:, 2]
    out = P.gather(fields, cell, off, order)
    assert np.max(np.abs(out - want[:, None])) < 1e-11


def test_push_moves_particles_by_v_dt():
    """No fields: u is kept and x^{n+1} - x^n = dt u / gamma / dx per axis (cell units)."""
    rng = np.random.default_rng(4)
    shape = (16, 8)
    fields = [np.zeros(shape[::-1]) for _ in range(6)]
    cell, off = _particles(rng, 100, shape)
    u = rng.standard_normal((100, 3)) * 5.0
    dt, dx = 0.1, np.array([0.2, 0.25])
    c2, o2, un, on, v3, ok = P.push(fields, cell, off, u, np.ones(100), dt, dx, 2)
    g = np.sqrt(1.0 + np.sum(u * u, axis=1))
    assert ok.all() and np.array_equal(un, u)
    assert np.max(np.abs(on - o2 - dt * u[:, :2] / g[:, None] / dx[None, :])) < 1e-15
    assert np.max(np.abs(v3 - u[:, 2] / g)) < 1e-15
