"""Iteration parity with 320-voxel subdomain edges, the edge of the 1280^3 workload
(4 x 4 x 4 subdomains of 320^3), on each axis in turn.

The 320-edge kernels of the three FFT passes, the fused axis-2 corrections, the
layer update, the update epilogue and the FP64 residual run in the iteration mode
of Eq. wavesim_iter here and are compared with the oracle at equal iteration counts
(1 iteration launched kernel by kernel, 10 iterations as two replays of a CUDA
graph of 5), in the x form, the residual form and with 3xTF32 tensor-core
corrections. The other two axes are short so that the oracle stays fast.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import Problem, relative_l2  # noqa: E402
from synth import point_source, spheres_medium  # noqa: E402

ITER_TOL = 1e-4
GEOMS = {"axis0": (640, 48, 48), "axis1": (48, 640, 48), "axis2": (48, 48, 640)}
KW = dict(widths=((8, 8),) * 3, split=(2, 2, 2), t=8)


@pytest.fixture(scope="module")
def oracle_runs():
    """Per geometry: medium, source, the oracle's iterates after 1 and 10 iterations, its history."""
    out = {}
    for name, shape in GEOMS.items():
        n = spheres_medium(shape, count=6, r_range=(3, 12), n_range=(1.0, 1.5), seed=320 + len(out), margin=8)
        src = point_source(shape)
        ref = Problem(n, 0.25, 1.0, widths=KW["widths"], split=KW["split"], t=KW["t"])
        first = {}

        def keep(it, x, eps):
            if it == 0:
                first["x"] = x.copy()

        x10, it, hist = ref.solve(src, tol=0.0, max_iter=10, callback=keep)
        out[name] = (n, src, first["x"], x10, np.array(hist), ref)
    return out


@pytest.mark.parametrize("form", ["x", "residual", "tf32"])
@pytest.mark.parametrize("geom", sorted(GEOMS))
def test_320_edge_iterations_match_oracle(oracle_runs, geom, form):
    import paper_2410_02395_gb300 as pkg

    n, src, x1r, x10r, histr, ref = oracle_runs[geom]
    shape = GEOMS[geom]
    assert 320 in ref.sizes[int(geom[-1])]
    plan = pkg.Plan(shape, 0.25, 1.0, torch.from_numpy(n).cuda(), boundary_widths=KW["widths"], split=KW["split"],
                    truncation=KW["t"], graph_iters=5, residual_form=form == "residual", corr_tf32=form == "tf32")
    info = plan.info()
    assert info["graph_iters"] == 5
    s = torch.from_numpy(src).cuda()
    x1, it1, _ = plan.solve(s, tol=0.0, max_iter=1)
    assert it1 == 1
    assert relative_l2(x1.cpu().numpy(), x1r) < ITER_TOL
    x10, it10, _, hist = plan.solve(s, tol=0.0, max_iter=10, with_history=True)
    assert it10 == 10
    err = relative_l2(x10.cpu().numpy(), x10r)
    assert err < ITER_TOL, err
    np.testing.assert_allclose(hist, histr, rtol=1e-4, atol=1e-6)
    plan.close()


@pytest.mark.parametrize("geom", ["axis0", "axis1"])
def test_320_edge_tma_passes_equal_register_fed_passes(oracle_runs, geom):
    """The 320 tile of the TMA-fed passes is two boxes of 160; the axis-1 pass and
    the axis-0 pass (forward, propagator, inverse) fed that way give the same
    iterates, bit for bit, as the register-fed kernels."""
    import paper_2410_02395_gb300 as pkg

    n, src, _, _, _, _ = oracle_runs[geom]
    shape = GEOMS[geom]
    xs = []
    for kw in ({"force_tma": True}, {"no_tma": True}):
        plan = pkg.Plan(shape, 0.25, 1.0, torch.from_numpy(n).cuda(), boundary_widths=KW["widths"],
                        split=KW["split"], truncation=KW["t"], graph_iters=5, **kw)
        assert (plan.info()["tma_groups"] >= 1) == ("force_tma" in kw)
        x, it, _ = plan.solve(torch.from_numpy(src).cuda(), tol=0.0, max_iter=10)
        xs.append(x)
        plan.close()
    assert torch.equal(xs[0], xs[1])


# Axis-2 edges above 256 other than 320, whose row tiles use the general
# (row, element) enumeration of the first pass (343 = 7^3 with 21 warps per CTA,
# 270 with 16): the first pass copies x into its tile with cp.async there.
WIDE = {"343": (32, 32, 686), "270": (32, 32, 540)}


@pytest.mark.parametrize("edge", sorted(WIDE))
def test_wide_axis2_edge_iterations_match_oracle(edge):
    import paper_2410_02395_gb300 as pkg

    shape = WIDE[edge]
    n = spheres_medium(shape, count=5, r_range=(3, 10), n_range=(1.0, 1.5), seed=343, margin=8)
    src = point_source(shape)
    ref = Problem(n, 0.25, 1.0, widths=KW["widths"], split=KW["split"], t=KW["t"])
    assert int(edge) in ref.sizes[2]
    x10r, _, histr = ref.solve(src, tol=0.0, max_iter=10)
    plan = pkg.Plan(shape, 0.25, 1.0, torch.from_numpy(n).cuda(), boundary_widths=KW["widths"], split=KW["split"],
                    truncation=KW["t"], graph_iters=5)
    x10, it10, _, hist = plan.solve(torch.from_numpy(src).cuda(), tol=0.0, max_iter=10, with_history=True)
    assert it10 == 10
    err = relative_l2(x10.cpu().numpy(), x10r)
    assert err < ITER_TOL, err
    np.testing.assert_allclose(hist, np.array(histr), rtol=1e-4, atol=1e-6)
    plan.close()
