"""FP64 oracle of the hybrid solver in quasi-3D geometry (Sec. 5): fields
expanded in azimuthal modes F(r, z, phi) = sum_m F_m(r, z) exp(i m phi); for
each mode m the z (x1) derivative is spectral (FFT along z, the same
sigma+/- symbols as the 2D solver) and the r (x2) derivatives are the Yee
finite differences of the cylindrical curl.  TEST INFRASTRUCTURE ONLY.

The paper defers the per-mode equations to its references, so they are
derived here from Maxwell's equations in (z, r, phi) with d/dphi -> i m:
  (curl A)_r   = (i m / r) A_z - dA_phi/dz
  (curl A)_phi = dA_r/dz - dA_z/dr
  (curl A)_z   = (1/r) d(r A_phi)/dr - (i m / r) A_r
Staggering is the 2D grid's with x1 = z, x2 = r: E_z at (i+1/2, j),
E_r at (i, j+1/2), E_phi at (i, j), B_z at (i, j+1/2), B_r at (i+1/2, j),
B_phi at (i+1/2, j+1/2), j like E; r_j = j dr, half points stored at j.
Axis (j = 0): values follow regularity of mode m (F(-r) = F(r, phi + pi)):
  E_z(0) is updated from the circulation of B_phi around a disc of radius
  dr/2 (d(r B_phi)/dr / r -> 4 B_phi(dr/2)/dr) for m = 0 and is 0 otherwise;
  E_phi(0), B_r(0) are 0 unless m = 1, where (i m / r) E_z -> i m E_z(dr)/dr
  and dB_z/dr(0) = 2 B_z(dr/2)/dr (B_z odd across the axis for m = 1).
Upper boundary: a perfect conductor at r = n_r dr (E_z = E_phi = 0 there).
The j_z correction (Eq. currentcorrection) and the k1 filter act on j as in 2D.
Fields are complex arrays [n_r][n_z]; z is periodic.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class QGrid:
    nz: int
    nr: int
    dz: float
    dr: float
    dt: float
    m: int = 0
    correct_jz: bool = True
    filt_kc: float = 0.0
    filt_w: float = 0.0
    ampere: float = 4.0 * np.pi


def kz(g: QGrid):
    """Signed wavenumbers of numpy's FFT order; Nyquist taken as +pi/dz."""
    kap = np.fft.fftfreq(g.nz, 1.0 / g.nz)
    kap[g.nz // 2] = g.nz // 2
    return 2.0 * np.pi * kap / (g.nz * g.dz)


def tables(g: QGrid):
    k = kz(g)
    ph = 0.5 * k * g.dz
    sp = 1j * k * np.exp(1j * ph)        # integer -> half-integer z points
    sm = 1j * k * np.exp(-1j * ph)       # half-integer -> integer z points
    with np.errstate(invalid="ignore", divide="ignore"):
        corr = np.where(k == 0, 1.0, np.sin(ph) / ph)
    F = np.ones_like(k)
    if 0.0 < g.filt_kc < 1.0:
        kn = np.pi / g.dz
        a = np.abs(k)
        kc, w = g.filt_kc * kn, g.filt_w * kn
        F = np.where(a <= kc - 0.5 * w, 1.0,
                     np.where(a >= kc + 0.5 * w, 0.0, np.cos(0.5 * np.pi * (a - kc + 0.5 * w) / w) ** 2))
    return sp, sm, corr, F


def step(g: QGrid, E, B, J, nsteps: int = 1):
    """E = (E_z, E_r, E_phi), B = (B_z, B_r, B_phi), J = (J_z, J_r, J_phi): complex
    [n_r][n_z] arrays, advanced in place from (E^n, B^{n-1/2}) with j^{n+1/2}."""
    sp, sm, corr, F = tables(g)
    dt, dr, m = g.dt, g.dr, g.m
    nr = g.nr
    j = np.arange(nr)[:, None].astype(float)
    r_i = j * dr                     # integer radii
    r_h = (j + 0.5) * dr             # half-integer radii
    im = 1j * m
    for _ in range(nsteps):
        Ez, Er, Ep = (np.fft.fft(a, axis=1) for a in E)
        Bz, Br, Bp = (np.fft.fft(a, axis=1) for a in B)
        Jz, Jr, Jp = (np.fft.fft(a, axis=1) for a in J)
        Jz = Jz * (F * (corr if g.correct_jz else 1.0))
        Jr = Jr * F
        Jp = Jp * F
        # ---- Faraday: B^{n+1/2} = B^{n-1/2} - dt curl E^n
        Ez_up = np.vstack([Ez[1:], np.zeros((1, g.nz))])          # E_z(j+1), wall value 0
        Ep_up = np.vstack([Ep[1:], np.zeros((1, g.nz))])          # E_phi(j+1), wall value 0
        r_up = np.vstack([r_i[1:], np.full((1, 1), nr * dr)])
        with np.errstate(invalid="ignore", divide="ignore"):
            curl_r = np.where(r_i > 0, im / np.where(r_i > 0, r_i, 1.0) * Ez, 0.0) - sp * Ep
        if m == 1:
            curl_r[0] = im * Ez[1] / dr - sp * Ep[0]
        curl_p = sp * Er - (Ez_up - Ez) / dr
        curl_z = (r_up * Ep_up - r_i * Ep) / (r_h * dr) - im / r_h * Er
        Bz = Bz - dt * curl_z
        Br = Br - dt * curl_r
        Bp = Bp - dt * curl_p
        if m != 1:
            Br[0] = 0.0
        # ---- Ampere: E^{n+1} = E^n + dt curl B^{n+1/2} - 4 pi dt j
        Bz_dn = np.vstack([np.zeros((1, g.nz)), Bz[:-1]])         # B_z(j-1/2), unused at j = 0
        Bp_dn = np.vstack([np.zeros((1, g.nz)), Bp[:-1]])
        r_dn = r_h - dr
        cE_r = im / r_h * Bz - sm * Bp
        cE_p = sm * Br - (Bz - Bz_dn) / dr
        with np.errstate(invalid="ignore", divide="ignore"):
            cE_z = (r_h * Bp - r_dn * Bp_dn) / np.where(r_i > 0, r_i * dr, 1.0) - im / np.where(r_i > 0, r_i, 1.0) * Br
        # axis rules
        cE_z[0] = 4.0 * Bp[0] / dr if m == 0 else 0.0
        cE_p[0] = (sm[None, :] * Br[0] - 2.0 * Bz[0] / dr)[0] if m == 1 else 0.0
        Er = Er + dt * cE_r - g.ampere * dt * Jr
        Ep = Ep + dt * cE_p - g.ampere * dt * Jp
        Ez = Ez + dt * cE_z - g.ampere * dt * Jz
        if m != 0:
            Ez[0] = 0.0
        if m != 1:
            Ep[0] = 0.0
        for dst, src in zip(E, (Ez, Er, Ep)):
            dst[:] = np.fft.ifft(src, axis=1)
        for dst, src in zip(B, (Bz, Br, Bp)):
            dst[:] = np.fft.ifft(src, axis=1)


def transfer_matrix(g: QGrid, kappa: int):
    """The one-step linear map (j = 0) of the 6 n_r complex amplitudes of z mode
    kappa, built by stepping unit vectors through `step` (nz small)."""
    n = 6 * g.nr
    k = kz(g)[kappa]
    z_int = np.arange(g.nz) * g.dz
    z_half = z_int + 0.5 * g.dz
    # staggered z positions: E_z, B_r, B_phi at half points
    zpos = [z_half, z_int, z_int, z_int, z_half, z_half]
    T = np.zeros((n, n), dtype=complex)
    for col in range(n):
        f, rr = divmod(col, g.nr)
        arrs = [np.zeros((g.nr, g.nz), dtype=complex) for _ in range(6)]
        arrs[f][rr] = np.exp(1j * k * zpos[f])
        E, B = arrs[:3], arrs[3:]
        J = [np.zeros((g.nr, g.nz), dtype=complex) for _ in range(3)]
        step(g, E, B, J)
        out = E + B
        for f2 in range(6):
            amp = np.sum(out[f2] * np.exp(-1j * k * zpos[f2])[None, :], axis=1) / g.nz
            T[f2 * g.nr:(f2 + 1) * g.nr, col] = amp
    return T
