"""Every mixed-radix FFT length (each n <= 512 with prime factors 2, 3, 5, 7) and
a spread of Bluestein lengths (other n <= 256) on each axis, so that each
length's row, strided and axis-0 pass kernels run once: the forward and
inverse 3-D DFT of one subdomain (Sec. 3.1) and the propagator (L+I)^-1
against the oracle. Bluestein transforms round a little more (two M-point
FFTs and the chirp products per transform): 4e-6 there."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import Problem, fftn3, ifftn3, relative_l2  # noqa: E402
from synth import random_field  # noqa: E402

OP_TOL = 2e-6


def _smooth7(v):
    for p in (2, 3, 5, 7):
        while v % p == 0:
            v //= p
    return v == 1


LENGTHS = [n for n in range(1, 513) if _smooth7(n)]
# every Bluestein convolution length M (32 ... 512) and primes across the range
BLUESTEIN = [11, 13, 17, 22, 23, 29, 31, 37, 41, 43, 47, 53, 59, 61, 67, 97, 101, 127, 131, 167, 191, 211, 251, 254]


def _sweep(axis, lengths, tol):
    import paper_2410_02395_gb300 as pkg

    bad = []
    for n in lengths:
        shape = [4, 4, 4]
        shape[axis] = n
        shape = tuple(shape)
        rng = np.random.default_rng(n)
        med = (1.0 + 0.4 * rng.random(shape)).astype(np.complex64)
        kw = dict(boundary_widths=((0, 0),) * 3, split=(1, 1, 1), truncation=1, periodic=(True,) * 3)
        plan = pkg.Plan(shape, 0.25, 1.0, torch.from_numpy(med).cuda(), **kw)
        ref = Problem(med, 0.25, 1.0, widths=kw["boundary_widths"], split=kw["split"], periodic=kw["periodic"], t=1)
        x = random_field(shape, seed=n + 7 * axis).astype(np.complex128)
        xd = torch.from_numpy(x.astype(np.complex64)).cuda()
        for which, want in (("FFT", fftn3(x)), ("IFFT", ifftn3(x)), ("PROPAGATE", ref.propagate(x))):
            got = plan.apply(which, xd).cpu().numpy().astype(np.complex128)
            err = relative_l2(got, want)
            if not err < tol:
                bad.append((n, which, err))
        plan.close()
    return bad


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_every_length_on_every_axis(axis):
    bad = _sweep(axis, LENGTHS, OP_TOL)
    assert not bad, bad


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_bluestein_lengths_on_every_axis(axis):
    bad = _sweep(axis, BLUESTEIN, 4e-6)
    assert not bad, bad
