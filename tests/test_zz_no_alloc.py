"""The allocation-free edge-correction entry point.

mbs_apply_edge_corrections_noalloc serves callers that must not trigger a
device allocation when they call (their device memory belongs to another
allocator or a fixed budget). It computes the same E x as
mbs_apply_operator(MBS_OP_E) with its scratch in a fixed array inside the
library. These tests call it through the C ABI, twice in a row per plan, and
compare it with the FP64 oracle's E and with the existing operator entry point;
the second call must leave the device's free memory unchanged. The scratch keeps
what the last call left in it, so plans of different shapes follow one another.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import Problem, relative_l2  # noqa: E402
from synth import random_field, spheres_medium  # noqa: E402

OP_TOL = 2e-6  # the single-operator tolerance of the parity tests


def _entry():
    import paper_2410_02395_gb300 as pkg

    lib = pkg.load_library()
    f = lib.mbs_apply_edge_corrections_noalloc
    f.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
    f.restype = C.c_int
    lib.mbs_noalloc_last_error.restype = C.c_char_p
    return pkg, lib, f


CASES = [((48, 40, 36), (2, 2, 2), 4, False, (False, False, False)),
         ((64, 64, 64), (2, 1, 2), 8, True, (False, False, False)),
         ((45, 32, 40), (3, 2, 1), 5, False, (False, False, False)),
         # axis 1 periodic and unsplit (a_1 = 0: no corrections along it), axis 0 split across its seam
         ((40, 24, 32), (2, 1, 2), 4, False, (True, True, False))]


def _check_two_calls(pkg, lib, f, shape, split, t, tf32, periodic, seeds):
    n = spheres_medium(shape, count=3, r_range=(2, 5), n_range=(1.1, 1.4), seed=21)
    widths = ((2, 2),) * 3
    plan = pkg.Plan(shape, 0.25, 1.0, torch.from_numpy(n).cuda(), boundary_widths=widths, split=split,
                    truncation=t, corr_tf32=tf32, periodic=periodic)
    ref = Problem(n, 0.25, 1.0, widths=widths, split=split, periodic=periodic, t=t)
    for call, seed in enumerate(seeds):
        xh = random_field(shape, seed=seed)
        x = torch.from_numpy(xh).cuda()
        out = torch.full(shape, complex(7.0, -3.0), dtype=torch.complex64, device="cuda")  # stale output
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        st = f(plan.handle, C.c_void_p(x.data_ptr()), C.c_void_p(out.data_ptr()))
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        assert st == 0, lib.mbs_noalloc_last_error().decode()
        if call > 0:
            assert free1 == free0, (free0, free1)
        got = out.cpu().numpy()
        want = ref.apply_E(xh.astype(np.complex128))
        assert relative_l2(got, want) < OP_TOL, (call, relative_l2(got, want))
        op = plan.apply("E", x)
        torch.cuda.synchronize()
        assert relative_l2(got, op.cpu().numpy()) < OP_TOL
    plan.close()


@pytest.mark.parametrize("shape,split,t,tf32,periodic", CASES)
def test_noalloc_matches_oracle_on_two_calls(shape, split, t, tf32, periodic):
    pkg, lib, f = _entry()
    _check_two_calls(pkg, lib, f, shape, split, t, tf32, periodic, (31, 32))


def test_noalloc_after_a_plan_of_another_shape():
    """A large plan's call fills much of the scratch; a smaller plan of another
    shape and split then reads none of what it left."""
    pkg, lib, f = _entry()
    _check_two_calls(pkg, lib, f, (96, 80, 64), (3, 2, 2), 6, False, (False,) * 3, (51, 52))
    _check_two_calls(pkg, lib, f, (20, 36, 28), (1, 3, 2), 3, False, (True, False, False), (53, 54))


def test_noalloc_rejects_oversized_grid_and_host_pointers():
    pkg, lib, f = _entry()
    shape = (160, 128, 128)  # 2,621,440 voxels > 2^21
    n = np.ones(shape, np.complex64)
    plan = pkg.Plan(shape, 0.25, 1.0, torch.from_numpy(n).cuda(), boundary_widths=((2, 2),) * 3, split=(2, 1, 1))
    x = torch.zeros(shape, dtype=torch.complex64, device="cuda")
    out = torch.zeros_like(x)
    st = f(plan.handle, C.c_void_p(x.data_ptr()), C.c_void_p(out.data_ptr()))
    assert st == 1 and b"exceeds" in lib.mbs_noalloc_last_error()
    plan.close()
    small = (16, 16, 16)
    plan = pkg.Plan(small, 0.25, 1.0, torch.ones(small, dtype=torch.complex64, device="cuda"), split=(2, 1, 1),
                    truncation=2)
    xh = np.zeros(small, np.complex64)
    oh = np.zeros(small, np.complex64)
    st = f(plan.handle, C.c_void_p(xh.ctypes.data), C.c_void_p(oh.ctypes.data))
    assert st == 1 and b"device pointers" in lib.mbs_noalloc_last_error()
    plan.close()
