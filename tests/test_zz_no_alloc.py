"""The allocation-free edge-correction entry point.

mbs_apply_edge_corrections_noalloc serves callers that must not trigger a
device allocation when they call (their device memory belongs to another
allocator or a fixed budget). It computes the same E x as
mbs_apply_operator(MBS_OP_E) with its scratch in a fixed array inside the
library; this checks the two agree on two calls in a row, through the C ABI.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import relative_l2  # noqa: E402
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


@pytest.mark.parametrize("shape,split,t,tf32", [((48, 40, 36), (2, 2, 2), 4, False),
                                               ((64, 64, 64), (2, 1, 2), 8, True),
                                               ((45, 32, 40), (3, 2, 1), 5, False)])
def test_noalloc_matches_operator_on_two_calls(shape, split, t, tf32):
    pkg, lib, f = _entry()
    n = spheres_medium(shape, count=3, r_range=(2, 5), n_range=(1.1, 1.4), seed=21)
    plan = pkg.Plan(shape, 0.25, 1.0, torch.from_numpy(n).cuda(), boundary_widths=((2, 2),) * 3, split=split,
                    truncation=t, corr_tf32=tf32)
    for call, seed in enumerate((31, 32)):
        x = torch.from_numpy(random_field(shape, seed=seed)).cuda()
        out = torch.full(shape, complex(7.0, -3.0), dtype=torch.complex64, device="cuda")  # stale output
        st = f(plan.handle, C.c_void_p(x.data_ptr()), C.c_void_p(out.data_ptr()))
        assert st == 0, lib.mbs_noalloc_last_error().decode()
        ref = plan.apply("E", x)
        torch.cuda.synchronize()
        err = relative_l2(out.cpu().numpy(), ref.cpu().numpy())
        assert err < OP_TOL, (call, err)
    plan.close()


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
