"""The C-ABI library builds, loads and exports every symbol include/mbs.h declares
(no compute calls: this runs without a GPU)."""
import ctypes
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    txt = open(os.path.join(ROOT, "include", "mbs.h")).read()
    return sorted(set(re.findall(r"MBS_API\s+[\w\s\*]+?\b(mbs_\w+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    import paper_2410_02395_gb300 as pkg

    pkg.build()
    return pkg.load_library()


def test_header_declares_the_paper_calls():
    syms = _declared_symbols()
    for s in ("mbs_plan_create", "mbs_apply_operator", "mbs_solve", "mbs_plan_destroy", "mbs_last_error"):
        assert s in syms


def test_library_exports_every_declared_symbol(lib):
    for s in _declared_symbols():
        assert hasattr(lib, s), s


def test_no_device_gives_error_status_not_fallback(lib):
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import numpy as np

    import paper_2410_02395_gb300 as pkg

    with pytest.raises(pkg.MBSError) as ei:
        pkg.Plan((8, 8, 8), 0.25, 1.0, np.ones((8, 8, 8), np.complex64))
    assert ei.value.status == 3  # MBS_ECUDA


def test_workspace_query_and_validation(lib):
    import paper_2410_02395_gb300 as pkg

    b1 = pkg.Plan.workspace_bytes((64, 64, 64), (1, 1, 1))
    b2 = pkg.Plan.workspace_bytes((256, 256, 256), (2, 2, 2))
    assert b2 > 4 * 256 ** 3 * 8 and b1 > 4 * 64 ** 3 * 8
    with pytest.raises(pkg.MBSError) as ei:
        pkg.Plan.workspace_bytes((64, 64, 64), (1, 1, 17))
    assert ei.value.status == 1
    with pytest.raises(pkg.MBSError) as ei:
        pkg.Plan.workspace_bytes((262, 8, 8), (1, 1, 1))     # 262 = 2 * 131: above the Bluestein range
    assert ei.value.status == 8
    with pytest.raises(pkg.MBSError) as ei:
        pkg.Plan.workspace_bytes((12, 8, 8), (2, 1, 1), truncation=7)   # t > subdomain edge 6
    assert ei.value.status == 1
    with pytest.raises(pkg.MBSError):
        pkg.Plan.workspace_bytes((12, 8, 8), (2, 1, 1), split_sizes=[[5, 6], [8], [8]])


def _smooth7(v):
    for p in (2, 3, 5, 7):
        while v % p == 0:
            v //= p
    return v == 1


def test_edge_length_rule(lib):
    """The header's size rule: every edge up to 256, and edges up to 512 whose prime
    factors are 2, 3, 5 and 7; anything else is MBS_EUNSUPPORTED."""
    import paper_2410_02395_gb300 as pkg

    for n in range(1, 520):
        ok = n <= 256 or (n <= 512 and _smooth7(n))
        try:
            pkg.Plan.workspace_bytes((8, 8, n), (1, 1, 1), truncation=1)
            got = True
        except pkg.MBSError as e:
            assert e.status == 8, (n, e.status)
            got = False
        assert got == ok, n


def test_degenerate_and_limit_arguments(lib):
    """Empty and out-of-range arguments are refused with a status, nothing runs."""
    import paper_2410_02395_gb300 as pkg

    def status(*args, **kw):
        try:
            pkg.Plan.workspace_bytes(*args, **kw)
            return 0
        except pkg.MBSError as e:
            return e.status

    assert status((0, 8, 8), (1, 1, 1)) == 1                 # empty grid
    assert status((8, 8, 8), (1, 9, 1)) == 1                 # more subdomains than voxels along an axis
    assert status((8, 8, 8), (1, 1, 1), truncation=41) == 1  # t above MBS_MAX_T
    assert status((64, 40, 40), (2, 1, 1), truncation=17) == 0  # a width without a specialised kernel
    assert status((64, 8, 8), (2, 1, 1), truncation=0) == 0     # t = 0: no corrections
    assert status((64, 40, 40), (2, 1, 1), truncation=33) == 1  # t above a subdomain edge (32)
    assert status((16 * 32, 8, 8), (16, 1, 1)) == 0          # MBS_MAX_SPLIT subdomains along an axis
    assert status((512, 8, 8), (1, 1, 1)) == 0               # MBS_MAX_EDGE
    assert status((1, 1, 1), (1, 1, 1), truncation=1) == 0   # a single voxel


def test_host_only_entry_points(lib):
    """Defaults, kernel-kind names and error text need no device."""
    import paper_2410_02395_gb300 as pkg

    opts = pkg._Options()
    lib.mbs_default_options(C.byref(opts))
    assert opts.truncation == 8 and opts.alpha == 0.75 and opts.absorb_kappa == 0.5
    assert opts.flags == 0 and opts.periodic_mask == 0 and not opts.split_sizes
    assert opts.tma_wait_cycles == 0
    lib.mbs_kernel_kind_name.restype = C.c_char_p
    names = [lib.mbs_kernel_kind_name(k).decode() for k in range(pkg.KERNEL_KINDS)]
    assert names == ["corr_x", "rows_first", "strided_fwd", "mid_axis0", "strided_inv", "rows_last", "corr_e",
                     "shell_update"]
    assert lib.mbs_kernel_kind_name(pkg.KERNEL_KINDS) == b""
    with pytest.raises(pkg.MBSError) as ei:
        pkg.Plan.workspace_bytes((8, 8, 262), (1, 1, 1))     # 262 = 2 x 131: no FFT for it
    lib.mbs_last_error.restype = C.c_char_p
    assert ei.value.status == 8 and b"262" in lib.mbs_last_error()


def test_workspace_grows_with_the_grid_and_the_residual_form(lib):
    import paper_2410_02395_gb300 as pkg

    b64 = pkg.Plan.workspace_bytes((64, 64, 64), (1, 1, 1))
    b128 = pkg.Plan.workspace_bytes((128, 64, 64), (2, 1, 1))
    assert b128 > 2 * b64 * 0.9
    br = pkg.Plan.workspace_bytes((64, 64, 64), (1, 1, 1), residual_form=True)
    assert br - b64 >= 64 ** 3 * 12   # r' (8 B) and the low word of x (4 B) per voxel
