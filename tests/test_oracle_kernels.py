"""Pins of the Laplacian kernels, the correction block and the scale factor."""
import numpy as np
import pytest

from oracle import Problem, block_norm, correction_block, frequencies_squared, sinc_d2
from tests.dense_reference import infinite_d2, periodic_d2_closed


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 8, 9, 16, 17, 30])
def test_periodic_kernel_three_ways(n):
    """Closed form == FFT of -p^2 (numpy) == periodised infinite-grid kernel (Fig. 4)."""
    h = 0.25
    closed = periodic_d2_closed(n, h)[:, 0]          # D_per(m) for m = 0..n-1
    # (1) the angular-spectrum symbol -|p|^2, transformed with numpy's inverse FFT
    via_fft = np.fft.ifft(-frequencies_squared(n, h)).real
    np.testing.assert_allclose(closed, via_fft, rtol=0, atol=1e-10 / h ** 2)
    # (2) brute-force periodisation sum_q D_inf(m + q n), with the tail estimated
    Q = 20000
    m = np.arange(n)
    acc = np.zeros(n)
    for q in range(-Q, Q + 1):
        acc += infinite_d2(m + q * n, h)
    # tail beyond |q|>Q: |sum| <= 2 * 2/(h^2 n^2 Q) (alternating for odd n)
    np.testing.assert_allclose(closed, acc, rtol=0, atol=8.0 / (h * h * n * n * Q) + 1e-9)


def test_sinc_kernel_values():
    h = 0.5
    assert sinc_d2(np.array([0]), h)[0] == pytest.approx(-np.pi ** 2 / (3 * h * h))
    assert sinc_d2(np.array([1]), h)[0] == pytest.approx(2.0 / (h * h))
    assert sinc_d2(np.array([2]), h)[0] == pytest.approx(-2.0 / (4 * h * h))
    assert sinc_d2(np.array([-3]), h)[0] == pytest.approx(2.0 / (9 * h * h))


def test_correction_block_layout():
    t, h = 8, 0.25
    W = correction_block(t, h)
    # W[a, b] couples row t-1-? : the last voxel (a=t-1) and first voxel of the next
    # subdomain (b=0) are neighbours at distance 1.
    assert W[t - 1, 0] == pytest.approx(infinite_d2(1, h))
    assert W[0, t - 1] == pytest.approx(infinite_d2(2 * t - 1, h))
    assert W[3, 3] == pytest.approx(infinite_d2(t, h))
    # Toeplitz: W[a+1, b+1] == W[a, b]
    np.testing.assert_allclose(W[1:, 1:], W[:-1, :-1])


def test_block_norm_by_power_iteration():
    W = correction_block(8, 0.25)
    v = np.ones(8)
    for _ in range(5000):
        v = W.T @ (W @ v)
        v /= np.linalg.norm(v)
    assert block_norm(W) == pytest.approx(np.linalg.norm(W @ v), rel=1e-9)


def _medium(shape, seed=3):
    rng = np.random.default_rng(seed)
    return 1.0 + 0.4 * rng.random(shape)


def test_scale_factor_reduces_to_single_domain_form():
    """All a_d = 0 (periodic, one subdomain): c = -0.95i / ||k^2 - k0^2||_inf (Eq. c_scale)."""
    n = _medium((6, 6, 6))
    p = Problem(n, 0.25, 1.0, widths=((0, 0),) * 3, periodic=(True,) * 3)
    assert p.a == [0, 0, 0]
    k2 = (2 * np.pi * n / 1.0) ** 2
    k0 = 0.5 * (k2.min() + k2.max())
    assert p.c == pytest.approx(-0.95j / np.abs(k2 - k0).max(), rel=1e-13)


def test_scale_factor_independent_of_subdomain_count():
    """Eq. c_scale2 depends on a_d only, not on how many subdomains an axis has (Sec. 4.2.2)."""
    n = _medium((24, 6, 6))
    cs = []
    for s0 in (2, 3, 4):
        p = Problem(n, 0.25, 1.0, widths=((2, 2),) * 3, split=(s0, 1, 1), t=4)
        assert p.a == [2, 1, 1]
        cs.append(p.c)
    assert cs[0] == cs[1] == cs[2]
    p = Problem(n, 0.25, 1.0, widths=((2, 2),) * 3, split=(1, 1, 1), t=4)
    W = correction_block(4, 0.25)
    assert p.c == pytest.approx(-0.95j / (p.contrast + 3 * block_norm(W)), rel=1e-13)
    assert abs(cs[0]) < abs(p.c)


def test_degenerate_scale_factor():
    n = np.ones((4, 4, 4))
    p = Problem(n, 0.25, 1.0, periodic=(True,) * 3)
    assert p.c == pytest.approx(-0.95j / (0.05 * (2 * np.pi) ** 2), rel=1e-13)
