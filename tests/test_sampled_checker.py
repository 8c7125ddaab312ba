"""The per-voxel operator checker used at full benchmark sizes equals the oracle's
apply_A on small grids (so a sampled GPU check means what it says)."""
import numpy as np
import pytest

from oracle import Problem


class _FakePlan:
    def __init__(self, p):
        self.p = p

    def info(self):
        p = self.p
        return dict(c=p.c, k0sq=p.k0sq, t=p.t, sizes=[list(s) for s in p.sizes], a=list(p.a))


@pytest.mark.parametrize("shape,split,periodic,t,w", [((24, 20, 18), (2, 2, 2), (False,) * 3, 4, 3),
                                                     ((30, 16, 12), (3, 1, 2), (False, True, False), 3, 2),
                                                     ((16, 16, 16), (2, 2, 1), (False, False, False), 8, 4)])
def test_sampled_checker_matches_oracle(shape, split, periodic, t, w):
    from tests.test_gpu_sampled import sampled_A

    rng = np.random.default_rng(3)
    n = (1.0 + 0.5 * rng.random(shape)).astype(np.complex64)
    widths = ((w, w),) * 3
    p = Problem(n, 0.25, 1.0, widths=widths, split=split, periodic=periodic, t=t)
    x = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    want = p.apply_A(x)
    params = dict(shape=shape, pixel=0.25, wavelength=1.0, widths=widths, periodic=periodic)

    def x_pencil(v, d, lo, hi):
        idx = list(v)
        idx[d] = slice(lo, hi)
        return x[tuple(idx)].reshape(-1)

    samples = [tuple(int(rng.integers(0, s)) for s in shape) for _ in range(60)]
    samples += [(0, 0, 0), tuple(s - 1 for s in shape)]
    got = sampled_A(_FakePlan(p), params, lambda v: n[v], x_pencil, samples)
    ref = np.array([want[v] for v in samples])
    assert np.max(np.abs(got - ref)) < 1e-10 * np.max(np.abs(ref))
