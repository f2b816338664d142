"""Pins of the oracle's textbook FFT against brute force and numpy.fft."""
import numpy as np
import pytest


def brute_dft(x, sign=-1):
    n = len(x)
    out = np.zeros(n, dtype=np.complex128)
    for k in range(n):
        s = 0j
        for j in range(n):
            ang = sign * 2.0 * np.pi * ((j * k) % n) / n
            s += x[j] * complex(np.cos(ang), np.sin(ang))
        out[k] = s
    return out


@pytest.mark.parametrize("n", [1, 2, 4, 6, 8, 12, 16, 30, 32])
def test_complex_fft_matches_brute_force(orc, n):
    rng = np.random.default_rng(n)
    z = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    ref = brute_dft(z, -1)
    got = orc.fft(z)
    assert np.max(np.abs(got - ref)) <= 1e-13 * max(1.0, np.max(np.abs(ref)))
    ref_i = brute_dft(z, +1)
    got_i = orc.fft(z, inverse=True)
    assert np.max(np.abs(got_i - ref_i)) <= 1e-13 * max(1.0, np.max(np.abs(ref_i)))


@pytest.mark.parametrize("n", [64, 256, 1024, 4096])
def test_fft_matches_numpy(orc, n):
    rng = np.random.default_rng(7 + n)
    z = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    ref = np.fft.fft(z)
    got = orc.fft(z)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("n", [4, 6, 16, 30, 128, 4096])
def test_rfft_and_round_trip(orc, n):
    rng = np.random.default_rng(100 + n)
    x = rng.standard_normal(n)
    X = orc.rfft(x)
    assert X.shape == (n // 2 + 1,)
    ref = np.fft.rfft(x)
    assert np.max(np.abs(X - ref)) <= 1e-12 * np.max(np.abs(ref))
    y = orc.irfft(X, n)
    assert np.max(np.abs(y - x)) <= 1e-14 * max(1.0, np.max(np.abs(x))) * max(1.0, np.log2(n))


def test_fft_linearity_and_shift(orc):
    """Shift theorem: x[j-s] <-> X[k] exp(-2 pi i k s / n)."""
    n = 64
    rng = np.random.default_rng(3)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    s = 5
    X = orc.fft(x)
    Xs = orc.fft(np.roll(x, s))
    k = np.arange(n)
    assert np.allclose(Xs, X * np.exp(-2j * np.pi * k * s / n), atol=1e-12)
