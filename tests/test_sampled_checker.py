"""The per-voxel operator checker and the slab-by-slab FP64 plan constants used at
full benchmark sizes equal the oracle's apply_A, k0^2, contrast and c on small
grids (so a sampled GPU check means what it says)."""
import numpy as np
import pytest

from oracle import Problem


@pytest.mark.parametrize("shape,split,periodic,t,w", [((24, 20, 18), (2, 2, 2), (False,) * 3, 4, 3),
                                                     ((30, 16, 12), (3, 1, 2), (False, True, False), 3, 2),
                                                     ((16, 16, 16), (2, 2, 1), (False, False, False), 8, 4)])
def test_sampled_checker_matches_oracle(shape, split, periodic, t, w):
    from tests.test_gpu_sampled import host_constants, sampled_A

    rng = np.random.default_rng(3)
    n = (1.0 + 0.5 * rng.random(shape)).astype(np.complex64)
    widths = ((w, w),) * 3
    p = Problem(n, 0.25, 1.0, widths=widths, split=split, periodic=periodic, t=t)
    x = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    want = p.apply_A(x)
    params = dict(shape=shape, pixel=0.25, wavelength=1.0, widths=widths, periodic=periodic, split=split)
    consts = host_constants(n.real.astype(np.float32), params, t)
    assert abs(consts["k0sq"] - p.k0sq) <= 1e-12 * abs(p.k0sq)
    assert abs(consts["contrast"] - p.contrast) <= 1e-12 * p.contrast
    assert abs(consts["c"] - p.c) <= 1e-12 * abs(p.c)
    assert consts["sizes"] == [list(v) for v in p.sizes] and consts["a"] == list(p.a)

    def x_pencil(v, d, lo, hi):
        idx = list(v)
        idx[d] = slice(lo, hi)
        return x[tuple(idx)].reshape(-1)

    samples = [tuple(int(rng.integers(0, s)) for s in shape) for _ in range(60)]
    samples += [(0, 0, 0), tuple(s - 1 for s in shape)]
    got = sampled_A(consts, params, lambda v: n[v], x_pencil, samples)
    ref = np.array([want[v] for v in samples])
    assert np.max(np.abs(got - ref)) < 1e-10 * np.max(np.abs(ref))
