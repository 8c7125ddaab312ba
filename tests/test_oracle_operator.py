"""Pins of the oracle's decomposed operators against closed-form dense matrices."""
import numpy as np
import pytest

from oracle import Problem, relative_l2
from tests import dense_reference as dr

CASES = [
    # shape, split, periodic, t, widths
    ((12, 1, 1), (2, 1, 1), (False, True, True), 3, ((2, 2), (0, 0), (0, 0))),
    ((13, 1, 1), (3, 1, 1), (True, True, True), 2, ((0, 0), (0, 0), (0, 0))),
    ((8, 6, 5), (2, 2, 1), (False, False, False), 2, ((1, 1), (1, 1), (1, 1))),
    ((9, 8, 6), (3, 2, 1), (False, True, False), 3, ((1, 2), (0, 0), (1, 0))),
    ((6, 6, 6), (1, 1, 1), (False, False, False), 3, ((1, 1), (1, 1), (1, 1))),
    ((8, 8, 8), (2, 2, 2), (True, False, True), 4, ((0, 0), (1, 1), (0, 0))),
    # the ends of the truncation sweep (Fig. 7: t = 0..40)
    ((12, 1, 1), (2, 1, 1), (False, True, True), 0, ((2, 2), (0, 0), (0, 0))),
    ((100, 1, 1), (2, 1, 1), (False, True, True), 40, ((4, 4), (0, 0), (0, 0))),
]


def _problem(shape, split, periodic, t, widths, seed=0):
    rng = np.random.default_rng(seed)
    n = 1.0 + 0.5 * rng.random(shape)
    return Problem(n, 0.25, 1.0, widths=widths, split=split, periodic=periodic, t=t)


@pytest.mark.parametrize("case", CASES)
def test_apply_A_equals_dense_truncated_operator(case):
    p = _problem(*case)
    A = dr.dense_A_truncated(p.shape, p.sizes, p.t, p.h, p.a, p.periodic, p.k2, p.c)
    rng = np.random.default_rng(1)
    x = rng.standard_normal(p.shape) + 1j * rng.standard_normal(p.shape)
    ref = (A @ x.ravel()).reshape(p.shape)
    assert relative_l2(p.apply_A(x), ref) < 1e-13


@pytest.mark.parametrize("case", CASES)
def test_L_and_V_split(case):
    """L is the block-diagonal periodic part (Eq. LV_block); V = A - L."""
    p = _problem(*case)
    L = dr.dense_L(p.shape, p.sizes, p.h, p.k0sq, p.c)
    rng = np.random.default_rng(2)
    x = rng.standard_normal(p.shape) + 1j * rng.standard_normal(p.shape)
    assert relative_l2(p.apply_L(x), (L @ x.ravel()).reshape(p.shape)) < 1e-13
    A = dr.dense_A_truncated(p.shape, p.sizes, p.t, p.h, p.a, p.periodic, p.k2, p.c)
    assert relative_l2(p.apply_V(x), ((A - L) @ x.ravel()).reshape(p.shape)) < 1e-12


@pytest.mark.parametrize("case", CASES)
def test_V_norm_below_one(case):
    """||V||_2 <= 0.95 by the choice of c (Eq. c_scale2), checked on the dense matrix."""
    p = _problem(*case)
    L = dr.dense_L(p.shape, p.sizes, p.h, p.k0sq, p.c)
    A = dr.dense_A_truncated(p.shape, p.sizes, p.t, p.h, p.a, p.periodic, p.k2, p.c)
    assert np.linalg.norm(A - L, 2) <= 0.95 + 1e-12


def test_truncation_error_decays_with_t():
    """The truncated operator approaches the undecomposed one as t grows (Sec. 4.2.1)."""
    shape = (64, 1, 1)
    rng = np.random.default_rng(4)
    n = 1.0 + 0.3 * rng.random(shape)
    x = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    errs = []
    for t in (1, 2, 4, 8, 16, 32):
        p = Problem(n, 0.25, 1.0, widths=((4, 4), (0, 0), (0, 0)), split=(2, 1, 1),
                    periodic=(False, True, True), t=t)
        Ag = dr.dense_A_global(shape, p.h, p.periodic, p.k2, p.c)
        errs.append(relative_l2(p.apply_A(x), (Ag @ x.ravel()).reshape(shape)))
    assert all(b < a for a, b in zip(errs, errs[1:]))
    # the dropped far-image tail decays like 1/t (the kernel decays like 1/m^2)
    assert errs[-1] < 0.1 * errs[0]


def test_full_blocks_reproduce_undecomposed_operator():
    """With t = n (whole subdomains) and two subdomains, the only dropped terms are
    images |q| >= 2 and the periodic self term; check the remainder is exactly those."""
    shape = (16, 1, 1)
    rng = np.random.default_rng(5)
    n = 1.0 + 0.3 * rng.random(shape)
    p = Problem(n, 0.25, 1.0, split=(2, 1, 1), periodic=(False, True, True), t=8)
    x = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    Ag = dr.dense_A_global(shape, p.h, p.periodic, p.k2, p.c)
    # dropped terms: per subdomain D_per - D_inf restricted, minus the kept q=+-1 images
    M = np.zeros((16, 16))
    for o in (0, 8):
        i = np.arange(8)
        m = i[:, None] - i[None, :]
        acc = np.zeros((8, 8))
        for q in range(-4000, 4001):
            if abs(q) >= 2:
                acc += dr.infinite_d2(m + 8 * q, p.h)
        M[o:o + 8, o:o + 8] = acc
    got = p.apply_A(x).ravel()
    ref = Ag @ x.ravel() + p.c * (M @ x.ravel())
    assert np.max(np.abs(got - ref)) < 1e-3 * np.max(np.abs(ref))


def test_planted_transfer_sign_is_caught():
    """A flipped transfer sign in the oracle is detected by the dense pin."""
    p = _problem(*CASES[2])
    A = dr.dense_A_truncated(p.shape, p.sizes, p.t, p.h, p.a, p.periodic, p.k2, p.c)
    rng = np.random.default_rng(1)
    x = rng.standard_normal(p.shape) + 1j * rng.standard_normal(p.shape)
    ref = (A @ x.ravel()).reshape(p.shape)
    orig = p.neighbours
    p.neighbours = lambda d, s: tuple(reversed(orig(d, s)))
    assert relative_l2(p.apply_A(x), ref) > 1e-3


def test_planted_transposed_block_is_caught():
    p = _problem(*CASES[3])
    A = dr.dense_A_truncated(p.shape, p.sizes, p.t, p.h, p.a, p.periodic, p.k2, p.c)
    rng = np.random.default_rng(1)
    x = rng.standard_normal(p.shape) + 1j * rng.standard_normal(p.shape)
    ref = (A @ x.ravel()).reshape(p.shape)
    p.cW = p.cW.T.copy()
    assert relative_l2(p.apply_A(x), ref) > 1e-3


@pytest.mark.parametrize("shape,t", [((1, 1, 1), 1), ((2, 2, 2), 2), ((3, 3, 3), 3)])
def test_c_scale_bound_fails_when_layer_ranges_coincide(shape, t):
    """Eq. c_scale2 bounds ||V|| by the norms of its parts, one ||W|| per a_d. On an
    unsplit grid whose edge n is at most t, a voxel is in the first and the last t
    layers at once and receives both wrap terms, so that bound no longer holds
    (reading R15): the dense ||V|| exceeds 1 and the series diverges there."""
    n = np.full(shape, 1.2 + 0.0j)
    p = Problem(n, 0.25, 1.0, split=(1, 1, 1), periodic=(False, False, False), t=t)
    L = dr.dense_L(p.shape, p.sizes, p.h, p.k0sq, p.c)
    A = dr.dense_A_truncated(p.shape, p.sizes, p.t, p.h, p.a, p.periodic, p.k2, p.c)
    assert np.linalg.norm(A - L, 2) > 1.0
