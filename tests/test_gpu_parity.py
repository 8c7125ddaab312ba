"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances (complex64 arithmetic, FP64 reductions):
  * single transforms / operators: relative L2 <= 2e-6 (FFT rounding ~ log2(n) ulp)
  * iterated solves at equal iteration count: relative L2 <= 1e-4 (the bar of the
    method's hot path for complex64 work)
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import Problem, relative_l2  # noqa: E402
from synth import point_source, random_field, spheres_medium  # noqa: E402

OP_TOL = 2e-6
ITER_TOL = 1e-4


def _pkg():
    import paper_2410_02395_gb300 as pkg

    pkg.load_library()
    return pkg


def make_pair(shape, split=(1, 1, 1), widths=((2, 2),) * 3, t=4, periodic=(False,) * 3, seed=5, split_sizes=None,
              pixel=0.25, wavelength=1.0, n=None, **plan_kw):
    pkg = _pkg()
    if n is None:
        n = spheres_medium(shape, count=4, r_range=(1.5, max(2.0, min(shape) / 4)), n_range=(1.1, 1.5), seed=seed)
    plan = pkg.Plan(shape, pixel, wavelength, torch.from_numpy(n).cuda(), boundary_widths=widths, split=split,
                    truncation=t, periodic=periodic, split_sizes=split_sizes, **plan_kw)
    ref = Problem(n, pixel, wavelength, widths=widths, split=split, periodic=periodic, t=t, split_sizes_=split_sizes)
    return plan, ref, n


CASES = {
    "cube_2x2x2": dict(shape=(48, 40, 36), split=(2, 2, 2), t=4),
    "ragged_3x1x2": dict(shape=(45, 21, 50), split=(3, 1, 2), t=3),
    "single_periodic": dict(shape=(32, 24, 20), split=(1, 1, 1), t=8, periodic=(True, True, True)),
    "single_nonperiodic": dict(shape=(30, 28, 27), split=(1, 1, 1), t=5),
    "periodic_split_seam": dict(shape=(40, 16, 24), split=(2, 1, 3), t=4, periodic=(True, True, False)),
    "uneven_sizes": dict(shape=(45, 32, 40), split=(2, 2, 2), t=4,
                         split_sizes=[[25, 20], [14, 18], [24, 16]]),
    "line_1d": dict(shape=(96, 1, 1), split=(3, 1, 1), t=6, periodic=(False, True, True),
                    widths=((8, 8), (0, 0), (0, 0))),
    "plane_2d": dict(shape=(1, 40, 64), split=(1, 2, 2), t=4, periodic=(True, False, False),
                     widths=((0, 0), (4, 4), (4, 4))),
    "tiny_t1": dict(shape=(12, 10, 8), split=(2, 2, 2), t=1),
    # truncation sweep (Sec. 4.2.1): wider corrections on the same geometry
    "t_sweep_2": dict(shape=(64, 48, 40), split=(2, 2, 2), t=2),
    "t_sweep_6": dict(shape=(64, 48, 40), split=(2, 2, 2), t=6),
    "t_sweep_12": dict(shape=(64, 48, 40), split=(2, 2, 2), t=12),
    "t_sweep_16": dict(shape=(64, 48, 40), split=(2, 2, 2), t=16),
    # t = 8 (the width of the benchmark workloads) takes the kernels specialised for it
    "t8_2x2x2": dict(shape=(40, 36, 48), split=(2, 2, 2), t=8),
    "t8_3x1x3": dict(shape=(48, 20, 60), split=(3, 1, 3), t=8, periodic=(False, True, False)),
    # edges with prime factors above 7 (Bluestein transforms) on every axis
    "prime_sizes": dict(shape=(84, 47, 53), split=(2, 1, 1), t=4, split_sizes=[[41, 43], [47], [53]]),
    "prime_mixed": dict(shape=(40, 22, 59), split=(2, 2, 1), t=3, split_sizes=[[16, 24], [11, 11], [59]],
                        periodic=(False, False, True)),
    # the boundary conditions of the paper's large example (Sec. 4.3): absorbing layers on the x
    # faces only, y and z periodic and split across their seams, uneven x subdomains
    "paper_geometry": dict(shape=(44, 32, 32), split=(2, 2, 2), t=4, periodic=(False, True, True),
                           widths=((6, 6), (0, 0), (0, 0)), split_sizes=[[24, 20], [16, 16], [16, 16]]),
}


TF32_CASES = ["cube_2x2x2", "uneven_sizes", "single_nonperiodic", "periodic_split_seam", "t_sweep_6", "prime_sizes",
              "paper_geometry"]
RES_CASES = ["cube_2x2x2", "single_periodic", "ragged_3x1x2", "line_1d", "t8_2x2x2", "t_sweep_16", "prime_sizes",
             "paper_geometry"]
PLAIN_CASES = ["cube_2x2x2", "uneven_sizes", "periodic_split_seam", "t8_2x2x2", "prime_sizes", "single_periodic"]


@pytest.fixture(scope="module", params=sorted(CASES) + ["tf32:" + c for c in TF32_CASES] +
                ["res:" + c for c in RES_CASES] + ["plain:" + c for c in PLAIN_CASES])
def pair(request):
    """(plan, oracle) on one case; "tf32:" cases run the edge corrections as 3xTF32
    tensor-core products (same tolerances: the split recovers FP32 accuracy);
    "res:" cases iterate in the residual form (same iterates in exact arithmetic);
    "plain:" cases iterate in the one-launch-per-step form with the stop test on
    the host."""
    name = request.param
    kw = {}
    if name.startswith("tf32:"):
        name = name[5:]
        kw["corr_tf32"] = True
    if name.startswith("res:"):
        name = name[4:]
        kw["residual_form"] = True
    if name.startswith("plain:"):
        name = name[6:]
        kw["plain_steps"] = True
    plan, ref, n = make_pair(**CASES[name], **kw)
    yield plan, ref
    plan.close()


def _gpu(plan, which, x):
    out = plan.apply(which, torch.from_numpy(x.astype(np.complex64)).cuda())
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.complex128)


def _per_subdomain(ref, x, fn):
    out = np.empty(ref.shape, dtype=np.complex128)
    for sl, _ in ref.boxes():
        out[sl] = fn(x[sl])
    return out


def test_plan_constants_match_oracle(pair):
    plan, ref = pair
    info = plan.info()
    assert info["a"] == list(ref.a)
    assert abs(info["k0sq"] - ref.k0sq) <= 1e-9 * abs(ref.k0sq)
    assert abs(info["contrast"] - ref.contrast) <= 1e-6 * ref.contrast
    assert abs(info["block_norm"] - ref.Wnorm) <= 1e-9 * max(ref.Wnorm, 1.0)
    assert abs(info["c"] - ref.c) <= 1e-6 * abs(ref.c)
    assert info["sizes"] == [list(s) for s in ref.sizes]


def test_forward_fft_per_subdomain(pair):
    """a3: unnormalised forward 3-D DFT of every subdomain (Sec. 3.1)."""
    from oracle import fftn3

    plan, ref = pair
    x = random_field(ref.shape, seed=11).astype(np.complex128)
    got = _gpu(plan, "FFT", x)
    want = _per_subdomain(ref, x, fftn3)
    assert relative_l2(got, want) < OP_TOL


def test_inverse_fft_per_subdomain(pair):
    """a5: inverse 3-D DFT with 1/prod(n) scaling."""
    from oracle import ifftn3

    plan, ref = pair
    x = random_field(ref.shape, seed=12).astype(np.complex128)
    got = _gpu(plan, "IFFT", x)
    want = _per_subdomain(ref, x, ifftn3)
    assert relative_l2(got, want) < OP_TOL


@pytest.mark.parametrize("which", ["E", "V", "L", "A", "PROPAGATE"])
def test_operator(pair, which):
    """a1-a2 (E, V), the fast convolution L and the propagator (L+I)^-1 (a3-a5)."""
    plan, ref = pair
    x = random_field(ref.shape, seed=13).astype(np.complex128)
    got = _gpu(plan, which, x)
    want = {"E": ref.apply_E, "V": ref.apply_V, "L": ref.apply_L, "A": ref.apply_A, "PROPAGATE": ref.propagate}[which](x)
    if which == "E" and not np.any(want):
        assert not np.any(got)
        return
    assert relative_l2(got, want) < OP_TOL, relative_l2(got, want)


def test_preconditioned_residual(pair):
    """a1-a6: Gamma^-1 (y - A x) for a random x and a point source."""
    plan, ref = pair
    src = point_source(ref.shape)
    plan.set_source(torch.from_numpy(src).cuda())
    x = random_field(ref.shape, seed=14).astype(np.complex128) * 1e-2
    got = _gpu(plan, "PRECOND", x)
    want = ref.preconditioned_residual(x, ref.scaled_source(src))
    assert relative_l2(got, want) < 5 * OP_TOL, relative_l2(got, want)


@pytest.mark.parametrize("n_iter", [1, 10, 60])
def test_iterations_match_oracle(pair, n_iter):
    """a1-a9: x after n iterations of Eq. wavesim_iter and the residual history."""
    plan, ref = pair
    src = point_source(ref.shape)
    x, it, res, hist = plan.solve(torch.from_numpy(src).cuda(), tol=0.0, max_iter=n_iter, with_history=True)
    xr, itr, histr = ref.solve(src, tol=0.0, max_iter=n_iter)
    assert it == itr == n_iter
    assert relative_l2(x.cpu().numpy(), xr) < ITER_TOL
    np.testing.assert_allclose(hist, histr, rtol=1e-4, atol=1e-6)
    assert hist[0] == 1.0


def test_solve_to_tolerance_small():
    """Stopping rule (Sec. 3.1): same iteration count and field as the oracle at tol."""
    plan, ref, n = make_pair((24, 20, 16), split=(2, 2, 1), widths=((3, 3), (3, 3), (2, 2)), t=4, seed=9)
    src = point_source(ref.shape)
    x, it, res, hist = plan.solve(torch.from_numpy(src).cuda(), tol=1e-4, max_iter=5000, with_history=True)
    xr, itr, histr = ref.solve(src, tol=1e-4, max_iter=5000)
    assert abs(it - itr) <= 1
    assert res < 1e-4
    assert relative_l2(x.cpu().numpy(), xr) < 1e-3
    h = np.array(hist)
    assert np.all(h[1:] <= h[:-1] * (1 + 1e-4) + 1e-6)   # monotone up to FP32 rounding
    plan.close()


def test_residual_form_reaches_below_the_x_form_floor():
    """The residual form converges to a tolerance the complex64 x-form cannot reach,
    to the oracle's converged solution of the same truncated system."""
    kw = dict(split=(2, 2, 1), widths=((3, 3), (3, 3), (2, 2)), t=4, seed=9)
    plan, ref, n = make_pair((24, 20, 16), residual_form=True, **kw)
    src = point_source(ref.shape)
    x, it, res = plan.solve(torch.from_numpy(src).cuda(), tol=1e-8, max_iter=20000)
    xr, itr, _ = ref.solve(src, tol=1e-11, max_iter=40000)
    assert res < 1e-8
    # the error of x is bounded by the conditioning of Gamma^-1 A times the gap
    # between the recursive and the true residual (complex64 rounding of the
    # transforms, summed over the iterations), ~1e-6 here
    assert relative_l2(x.cpu().numpy(), xr) < 5e-6
    plan.close()
    plain, _, _ = make_pair((24, 20, 16), **kw)
    _, it_x, res_x = plain.solve(torch.from_numpy(src).cuda(), tol=1e-8, max_iter=it)
    assert res_x > 1e-8   # the x-form stalls above it within the same iteration budget
    plain.close()


def test_host_buffers_equal_device_buffers():
    """Host (numpy) inputs/outputs go through the same kernels as device tensors."""
    plan, ref, n = make_pair((20, 16, 12), split=(2, 1, 2), t=3, seed=3)
    src = point_source(ref.shape)
    xd, itd, _ = plan.solve(torch.from_numpy(src).cuda(), tol=0.0, max_iter=15)
    xh, ith, _ = plan.solve(src, tol=0.0, max_iter=15)
    assert itd == ith == 15
    assert np.array_equal(xd.cpu().numpy(), xh)
    plan.close()


def test_zero_source_gives_zero_field():
    plan, ref, n = make_pair((16, 16, 16), split=(2, 2, 2), t=2, seed=4)
    z = np.zeros(ref.shape, np.complex64)
    x, it, res = plan.solve(torch.from_numpy(z).cuda(), tol=1e-6, max_iter=20)
    assert it == 1 and res == 0.0
    assert not torch.any(x != 0)
    plan.close()


def test_invalid_inputs_are_errors():
    pkg = _pkg()
    n = np.ones((8, 8, 8), np.complex64)
    with pytest.raises(pkg.MBSError) as ei:
        bad = n.copy()
        bad[1, 2, 3] = np.nan
        pkg.Plan((8, 8, 8), 0.25, 1.0, torch.from_numpy(bad).cuda())
    assert ei.value.status == 1
    with pytest.raises(pkg.MBSError) as ei:
        pkg.Plan((8, 8, 8), 0.25, -1.0, torch.from_numpy(n).cuda())
    assert ei.value.status == 1
    with pytest.raises(pkg.MBSError) as ei:
        pkg.Plan((8, 8, 8), 0.25, 1.0, torch.from_numpy(n).cuda(), split=(2, 1, 1), truncation=5)
    assert ei.value.status == 1


def test_nan_in_the_source_is_reported():
    """A non-finite residual stops the iteration with MBS_ENAN (fault made on the host)."""
    pkg = _pkg()
    plan, ref, n = make_pair((16, 16, 16), split=(2, 1, 1), t=2, seed=4)
    src = point_source(ref.shape)
    src[3, 3, 3] = np.nan
    with pytest.raises(pkg.MBSError) as ei:
        plan.solve(torch.from_numpy(src).cuda(), tol=1e-6, max_iter=50)
    assert ei.value.status == 5
    plan.close()


def test_over_relaxation_is_reported_as_divergence():
    """alpha = 4 breaks the convergence condition (alpha <= 1, Sec. 2): the residual
    keeps rising and the solve stops with MBS_EDIVERGE."""
    pkg = _pkg()
    plan, ref, n = make_pair((16, 16, 16), split=(2, 2, 1), t=2, seed=4, alpha=4.0)
    with pytest.raises(pkg.MBSError) as ei:
        plan.solve(torch.from_numpy(point_source(ref.shape)).cuda(), tol=1e-6, max_iter=2000)
    assert ei.value.status == 6
    plan.close()


def test_budget_exhausted_returns_last_iterate():
    plan, ref, n = make_pair((20, 16, 12), split=(2, 1, 2), t=3, seed=3)
    src = point_source(ref.shape)
    x, it, res = plan.solve(torch.from_numpy(src).cuda(), tol=1e-12, max_iter=17)
    xr, itr, _ = ref.solve(src, tol=0.0, max_iter=17)
    assert it == 17 and res > 1e-12
    assert relative_l2(x.cpu().numpy(), xr) < ITER_TOL
    plan.close()


def test_out_of_memory_is_reported_without_allocating():
    """A plan larger than the free device memory fails with MBS_ENOMEM before any
    allocation (the refractive index is not read before the memory check)."""
    import ctypes as C

    pkg = _pkg()
    lib = pkg.load_library()
    dummy = torch.ones((1, 1, 1), dtype=torch.complex64, device="cuda")
    opts = pkg._Options()
    lib.mbs_default_options(C.byref(opts))
    free0, _ = torch.cuda.mem_get_info()
    h = C.c_void_p()
    st = lib.mbs_plan_create(C.byref(h), (C.c_int64 * 3)(4096, 4096, 4096), 0.25, 1.0,
                             C.c_void_p(dummy.data_ptr()), (C.c_int32 * 6)(8, 8, 8, 8, 8, 8),
                             (C.c_int32 * 3)(8, 8, 8), C.byref(opts))
    assert st == 2, lib.mbs_last_error()
    assert not h.value
    free1, _ = torch.cuda.mem_get_info()
    assert abs(free1 - free0) < (64 << 20)


def test_plain_steps_form_solves_like_the_fused_form():
    """The one-launch-per-step form (host-side residual sums and stop test) stops
    at the same iteration as the fused form and the oracle, with the same field."""
    kw = dict(split=(2, 2, 1), widths=((3, 3), (3, 3), (2, 2)), t=4, seed=9)
    plan, ref, n = make_pair((24, 20, 16), plain_steps=True, **kw)
    fused, _, _ = make_pair((24, 20, 16), **kw)
    src = torch.from_numpy(point_source(ref.shape)).cuda()
    x, it, res, hist = plan.solve(src, tol=1e-4, max_iter=5000, with_history=True)
    xf, itf, resf = fused.solve(src, tol=1e-4, max_iter=5000)
    xr, itr, _ = ref.solve(point_source(ref.shape), tol=1e-4, max_iter=5000)
    assert it == itf and abs(it - itr) <= 1 and res < 1e-4
    assert relative_l2(x.cpu().numpy(), xf.cpu().numpy()) < 1e-4
    assert len(hist) == it and hist[0] == 1.0
    plan.close()
    fused.close()


def test_plain_steps_form_refuses_the_residual_form_and_batches():
    pkg = _pkg()
    with pytest.raises(pkg.MBSError) as ei:
        make_pair((16, 16, 16), split=(2, 1, 1), t=2, plain_steps=True, residual_form=True)
    assert ei.value.status == 1
    plan, _, _ = make_pair((16, 16, 16), split=(2, 1, 1), t=2, plain_steps=True)
    with pytest.raises(pkg.MBSError) as ei:
        pkg.Batch([plan])
    assert ei.value.status == 1
    plan.close()


@pytest.mark.parametrize("form", ["x", "residual", "plain"])
def test_warm_start_resumes_the_oracle_iteration(form):
    """Resume (Sec. 3.1: MBS converges from any start): 10 oracle iterations, then
    the GPU continues from that field for 10 more; the field and the residual
    history equal the oracle's iterations 11-20 (eps normalised by ||Gamma^-1 y||)."""
    kw = {"residual_form": form == "residual", "plain_steps": form == "plain"}
    plan, ref, n = make_pair((32, 24, 20), split=(2, 2, 1), widths=((3, 3), (3, 3), (2, 2)), t=4, seed=17, **kw)
    src = point_source(ref.shape)
    x10, _, _ = ref.solve(src, tol=0.0, max_iter=10)
    x20, _, hist20 = ref.solve(src, tol=0.0, max_iter=20)
    plan.set_source(torch.from_numpy(src).cuda())
    plan.set_initial_field(torch.from_numpy(x10.astype(np.complex64)).cuda())
    st, it, eps = plan.iterate(10, 0.0)
    assert it == 10
    x = plan.field(like=torch.zeros(1, device="cuda"))
    assert relative_l2(x.cpu().numpy(), x20) < ITER_TOL
    np.testing.assert_allclose(plan.history(10), hist20[10:], rtol=1e-4, atol=1e-6)
    plan.close()


def test_warm_start_needs_a_source():
    pkg = _pkg()
    plan, ref, n = make_pair((16, 16, 16), split=(2, 1, 1), t=2, seed=4)
    with pytest.raises(pkg.MBSError) as ei:
        plan.set_initial_field(np.zeros(ref.shape, np.complex64))
    assert ei.value.status == 1
    plan.close()
