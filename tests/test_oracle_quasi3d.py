"""Pins of the quasi-3D (azimuthal-mode) oracle.  The per-mode equations are
not printed in the paper (Sec. 5), so they are pinned by the mathematics of a
perfectly conducting cylinder: the one-step map of a z mode has frequencies
with [w]^2 = k_z^2 + lambda_r, and the discrete radial eigenvalues lambda_r
converge at second order in dr to (j_{m,n}/R)^2 (TM, zeros of J_m) and
(j'_{m,n}/R)^2 (TE, zeros of J_m').  Also: the map conserves the discrete
energy (unit-modulus eigenvalues below the Courant limit)."""
import numpy as np
import pytest
from scipy import special

from oracle import quasi3d as q


def _radial_eigs(m, nr, R=1.0):
    dr = R / nr
    dz = 0.05
    dt = 0.5 * 2 / np.sqrt(np.pi ** 2 / dz ** 2 + 4 / dr ** 2)
    g = q.QGrid(nz=8, nr=nr, dz=dz, dr=dr, dt=dt, m=m)
    mu = np.linalg.eigvals(q.transfer_matrix(g, 1))
    w = np.abs(np.angle(mu)) / dt
    k = q.kz(g)[1]
    lam = (np.sin(w * dt / 2) / (dt / 2)) ** 2 - k ** 2
    return np.unique(np.round(np.sort(lam[lam > 1e-6]), 9)), mu


def _continuum(m, R=1.0, n=3):
    te = special.jnp_zeros(m, n) if m > 0 else special.jn_zeros(1, n)
    return np.sort(np.concatenate([special.jn_zeros(m, n), te])) ** 2 / R ** 2


@pytest.mark.parametrize("m", [0, 1, 2])
def test_cylinder_modes_converge_at_second_order(m):
    cont = _continuum(m)[:4]
    errs = []
    for nr in (12, 24, 48):
        lam, mu = _radial_eigs(m, nr)
        errs.append(np.max(np.abs(lam[:4] - cont) / cont))
        live = mu[np.abs(mu) > 1e-12]          # axis values forced to zero by regularity map to 0
        assert np.max(np.abs(np.abs(live) - 1.0)) < 1e-10          # neutral below Courant
    assert errs[2] < 2e-3
    assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.5       # second order


def test_axis_regularity_kept():
    g = q.QGrid(nz=16, nr=10, dz=0.1, dr=0.1, dt=0.02, m=2)
    rng = np.random.default_rng(1)
    E = [rng.standard_normal((10, 16)) + 1j * rng.standard_normal((10, 16)) for _ in range(3)]
    B = [rng.standard_normal((10, 16)) + 1j * rng.standard_normal((10, 16)) for _ in range(3)]
    J = [np.zeros((10, 16), complex) for _ in range(3)]
    q.step(g, E, B, J, 3)
    assert np.all(E[0][0] == 0) and np.all(E[2][0] == 0) and np.all(B[1][0] == 0)


@pytest.mark.parametrize("m", [0, 1, 2, 3, 5])
def test_quasi3d_courant_bound(m):
    """The radial operator's largest eigenvalue sits at the axis and is at most
    (4 m^2 + 6)/dr^2: just below dt = 2/sqrt(pi^2/dz^2 + (4 m^2 + 6)/dr^2) every
    mode is neutral; the 2D limit (4/dr^2) is not stable for m >= 1."""
    dz, dr, nr, nz = 0.2, 0.15, 10, 8
    dt = 0.995 * 2 / np.sqrt(np.pi ** 2 / dz ** 2 + (4 * m * m + 6) / dr ** 2)
    g = q.QGrid(nz=nz, nr=nr, dz=dz, dr=dr, dt=dt, m=m)
    worst = max(np.max(np.abs(np.linalg.eigvals(q.transfer_matrix(g, k)))) for k in range(nz))
    assert worst < 1 + 1e-12
    if m >= 1:
        g2 = q.QGrid(nz=nz, nr=nr, dz=dz, dr=dr, dt=0.95 * 2 / np.sqrt(np.pi ** 2 / dz ** 2 + 4 / dr ** 2), m=m)
        worst2 = max(np.max(np.abs(np.linalg.eigvals(q.transfer_matrix(g2, k)))) for k in range(nz))
        assert worst2 > 1.01
