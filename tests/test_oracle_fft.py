"""Pins of the oracle's own FFT: brute-force DFT sums and numpy's FFT."""
import numpy as np
import pytest

from oracle import fft_axis, fftn3, ifftn3


def brute_dft(x, sign):
    n = len(x)
    out = np.zeros(n, dtype=np.complex128)
    for q in range(n):
        acc = 0j
        for m in range(n):
            ang = sign * 2.0 * np.pi * ((m * q) % n) / n
            acc += x[m] * complex(np.cos(ang), np.sin(ang))
        out[q] = acc
    return out


@pytest.mark.parametrize("n", list(range(1, 41)) + [45, 48, 49, 50, 54, 56, 60, 63, 64])
def test_fft_matches_brute_force_sum(n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    for sign in (-1, 1):
        ref = brute_dft(x, sign)
        got = fft_axis(x.reshape(n, 1, 1), 0, sign).ravel()
        assert np.max(np.abs(got - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref)))


@pytest.mark.parametrize("shape", [(8, 12, 10), (16, 5, 9), (1, 7, 32), (27, 1, 1)])
def test_fftn_matches_numpy(shape):
    rng = np.random.default_rng(7)
    x = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    np.testing.assert_allclose(fftn3(x), np.fft.fftn(x), rtol=0, atol=1e-11 * np.sqrt(x.size))
    np.testing.assert_allclose(ifftn3(x), np.fft.ifftn(x), rtol=0, atol=1e-13 * np.sqrt(x.size))


@pytest.mark.parametrize("n", [128, 320, 96])
def test_fft_axis_each_axis(n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal((n, 3, 4)) + 1j * rng.standard_normal((n, 3, 4))
    for ax in range(3):
        y = np.moveaxis(x, 0, ax)
        np.testing.assert_allclose(fft_axis(y, ax), np.fft.fft(y, axis=ax), rtol=0, atol=1e-10)
