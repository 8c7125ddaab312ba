"""The index-checking build (MBS_BOUNDS_CHECK): every kernel checks the index
range of its accesses to the grid arrays, skips any access outside the grid and
counts it in error words that the calls report. On the geometries below (uneven
and prime subdomain edges, a periodic seam, the 320 edge, activation masks, a
fused batch) nothing is reported and the iterates equal the normal build's."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import relative_l2  # noqa: E402
from synth import frequency_batch, point_source, spheres_medium  # noqa: E402


@pytest.fixture(scope="module")
def libs():
    import paper_2410_02395_gb300 as pkg

    path = pkg.build(bounds_check=True)
    checked = pkg.load_library(path)
    normal = pkg.load_library()
    assert checked.mbs_build_checks_bounds() == 1 and normal.mbs_build_checks_bounds() == 0
    return pkg, normal, checked


GEOMS = [
    dict(shape=(45, 32, 40), split=(2, 2, 2), t=4, split_sizes=[[25, 20], [14, 18], [24, 16]]),
    dict(shape=(84, 47, 53), split=(2, 1, 1), t=4, split_sizes=[[41, 43], [47], [53]]),
    dict(shape=(40, 16, 24), split=(2, 1, 3), t=4, periodic=(True, True, False)),
    dict(shape=(48, 48, 640), split=(2, 2, 2), t=8),
    dict(shape=(64, 48, 40), split=(2, 2, 2), t=6, activation=True),
]


@pytest.mark.parametrize("geom", range(len(GEOMS)))
def test_checked_build_reports_nothing_and_matches(libs, geom):
    pkg, normal, checked = libs
    kw = dict(GEOMS[geom])
    shape = kw.pop("shape")
    t = kw.pop("t")
    n = spheres_medium(shape, count=4, r_range=(2, 6), n_range=(1.1, 1.4), seed=81)
    src = torch.from_numpy(point_source(shape, tuple(s // 3 for s in shape))).cuda()
    xs = []
    for lib in (checked, normal):
        plan = pkg.Plan(shape, 0.25, 1.0, torch.from_numpy(n).cuda(), boundary_widths=((3, 3),) * 3,
                        truncation=t, graph_iters=5, library=lib, **kw)
        x, it, _ = plan.solve(src, tol=0.0, max_iter=12)   # raises if an index check fired
        assert it == 12
        for op in ("A", "PRECOND", "E"):
            plan.apply(op, torch.ones(shape, dtype=torch.complex64, device="cuda"))
        xs.append(x.cpu().numpy())
        plan.close()
    assert relative_l2(xs[0], xs[1]) < 1e-6


def test_checked_build_fused_batch(libs):
    pkg, normal, checked = libs
    problems = frequency_batch(count=3, seed=7, box=7.0, spheres=5, r_range=(0.5, 1.5), t=4)
    plans = []
    for params, n, src in problems:
        p = pkg.Plan(params["shape"], params["pixel"], params["wavelength"], torch.from_numpy(n).cuda(),
                     boundary_widths=params["widths"], split=params["split"], truncation=params["t"],
                     split_sizes=params["split_sizes"], library=checked)
        p.set_source(torch.from_numpy(src).cuda())
        plans.append(p)
    import ctypes as C

    arr = (C.c_void_p * len(plans))(*[p.handle for p in plans])
    h = C.c_void_p()
    checked.mbs_batch_create.argtypes = [C.POINTER(C.c_void_p), C.c_int32, C.POINTER(C.c_void_p), C.c_void_p,
                                         C.c_int32]
    assert checked.mbs_batch_create(C.byref(h), len(plans), arr, None, 5) == 0
    fused = C.c_int32()
    assert checked.mbs_batch_launches_per_iteration(h, C.byref(fused)) > 0 and fused.value == 1
    st = checked.mbs_batch_iterate(h, 10, C.c_double(0.0), 0, None, None, None)
    assert st in (0, 4), checked.mbs_last_error()
    checked.mbs_batch_destroy(h)
    for p in plans:
        p.close()
