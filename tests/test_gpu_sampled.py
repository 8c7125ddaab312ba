"""Sampled parity at the benchmark sizes (256^3 with 2x2x2 subdomains, 1280^3 with
4x4x4 subdomains of 320^3), in the benchmark's plan configuration.

At these sizes the oracle cannot transform the whole grid, but every output of
the operator A = L + V (Eq. LV_block) can be computed one by one: along each
axis, the voxel's pencil inside its subdomain times the periodic band-limited
kernel (closed form), plus the truncated t x t corrections of Sec. 3.1, plus
c k^2 x. The plan constants k0^2 (reading R1), ||k^2 - k0^2||_inf and c
(Eq. c_scale2) are computed here on the host in FP64 over the whole grid, slab
by slab, and the plan's own values (reduced on the device) must agree with them;
the sampled outputs use the host values. k^2 follows the oracle's
absorbing-layer reading (the per-axis ramps of oracle.absorbing_index, the
largest where layers meet).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import absorbing_index, axis_flags, block_norm, correction_block, split_sizes  # noqa: E402
from tests.dense_reference import periodic_d2_closed  # noqa: E402


def _axis_ramp(N, lo, hi, d, kappa):
    shape = [1, 1, 1]
    shape[d] = N
    w = [(0, 0)] * 3
    w[d] = (lo, hi)
    return (absorbing_index(np.ones(shape), w, kappa) - 1.0).imag.ravel() / kappa


def host_constants(n_real, params, t, kappa=0.5, slabs=16):
    """k0^2, contrast and c in FP64 on the host (torch CPU float64, multi-threaded),
    in slabs along axis 0.

    n_real is the (real) refractive index as a host float32 array. With the ramp
    r of the absorbing layers, n_eff = n + i kappa r and
    k^2 = (2 pi / lambda)^2 ((n^2 - kappa^2 r^2) + 2 i kappa n r)."""
    shape, lam, h = params["shape"], params["wavelength"], params["pixel"]
    ramps = [torch.from_numpy(_axis_ramp(shape[d], *params["widths"][d], d, kappa)) for d in range(3)]
    r12 = torch.maximum(ramps[1][:, None], ramps[2][None, :])
    s2 = (2 * np.pi / lam) ** 2
    nt = torch.from_numpy(np.ascontiguousarray(n_real))

    def k2_slabs(i0):
        nn = nt[i0:i0 + slabs].to(torch.float64)
        r = torch.maximum(r12[None], ramps[0][i0:i0 + slabs, None, None])
        return s2 * (nn * nn - (kappa * r) ** 2), s2 * (2.0 * kappa) * (nn * r)

    lo_r = lo_i = np.inf
    hi_r = hi_i = -np.inf
    for i0 in range(0, shape[0], slabs):
        kr, ki = k2_slabs(i0)
        lo_r, hi_r = min(lo_r, kr.min().item()), max(hi_r, kr.max().item())
        lo_i, hi_i = min(lo_i, ki.min().item()), max(hi_i, ki.max().item())
    k0sq = complex(0.5 * (lo_r + hi_r), 0.5 * (lo_i + hi_i))
    contrast = 0.0
    for i0 in range(0, shape[0], slabs):
        kr, ki = k2_slabs(i0)
        contrast = max(contrast, torch.hypot(kr - k0sq.real, ki - k0sq.imag).max().item())
    sizes = [split_sizes(shape[d], params["split"][d]) for d in range(3)]
    a = axis_flags(params["split"], params["periodic"])
    c = -0.95j / (contrast + sum(a) * block_norm(correction_block(t, h)))
    return dict(k0sq=k0sq, contrast=contrast, c=c, t=t, sizes=sizes, a=a)


def sampled_A(consts, params, n_at, x_pencil, samples, kappa=0.5):
    """Expected (A x)(v) for the voxels in ``samples``.

    n_at(v) returns n at a voxel; x_pencil(v, d, lo, hi) returns x along axis d
    through v for indices lo..hi-1."""
    c, k0sq, t, h, lam = consts["c"], consts["k0sq"], consts["t"], params["pixel"], params["wavelength"]
    shape, sizes, a = params["shape"], consts["sizes"], consts["a"]
    offs = [np.concatenate([[0], np.cumsum(s)[:-1]]).astype(int) for s in sizes]
    W = correction_block(t, h)
    ramps = [_axis_ramp(shape[d], *params["widths"][d], d, kappa) for d in range(3)]
    Dper = {}
    out = []
    for v in samples:
        acc = 0j
        for d in range(3):
            i = v[d]
            s = int(np.searchsorted(offs[d], i, side="right") - 1)
            o, nn = int(offs[d][s]), int(sizes[d][s])
            if nn not in Dper:
                Dper[nn] = periodic_d2_closed(nn, h)
            pen = x_pencil(v, d, o, o + nn)
            acc += c * (Dper[nn][i - o] @ pen)
            if a[d] == 0:
                continue
            S = len(sizes[d])
            per = params["periodic"][d]
            left = s - 1 if s > 0 else (S - 1 if per and S > 1 else None)
            right = s + 1 if s < S - 1 else (0 if per and S > 1 else None)
            if S == 1:
                left = right = None
            q = i - o
            if q >= nn - t:  # last t layers: row q-(n-t) of W on (right's first t - own first t)
                aa = q - (nn - t)
                f = -pen[:t]
                if right is not None:
                    f = f + x_pencil(v, d, int(offs[d][right]), int(offs[d][right]) + t)
                acc += c * (W[aa] @ f)
            if q < t:  # first t layers: row q of W^T on (left's last t - own last t)
                f = -pen[nn - t:]
                if left is not None:
                    lo = int(offs[d][left]) + int(sizes[d][left]) - t
                    f = f + x_pencil(v, d, lo, lo + t)
                acc += c * (W[:, q] @ f)
        ramp = max(ramps[0][v[0]], ramps[1][v[1]], ramps[2][v[2]])
        k2 = (2 * np.pi * (complex(n_at(v)) + 1j * kappa * ramp) / lam) ** 2
        acc += c * k2 * x_pencil(v, 0, v[0], v[0] + 1)[0]
        out.append(acc)
    return np.array(out)


def _samples(shape, widths, t, sizes, rng, count=48):
    """Random voxels plus voxels on subdomain edges, layer corners and absorbing faces."""
    pts = [tuple(int(rng.integers(0, s)) for s in shape) for _ in range(count)]
    offs = [np.concatenate([[0], np.cumsum(s)[:-1]]).astype(int) for s in sizes]
    for _ in range(count):
        v = []
        for d in range(3):
            s = int(rng.integers(0, len(sizes[d])))
            q = int(rng.choice([0, 1, t - 1, t, sizes[d][s] - t - 1, sizes[d][s] - t, sizes[d][s] - 1]))
            v.append(int(offs[d][s]) + min(max(q, 0), sizes[d][s] - 1))
        pts.append(tuple(v))
    pts.append((0, 0, 0))
    pts.append(tuple(s - 1 for s in shape))
    return pts


def _run(shape, split, pixel=0.25, lam=1.0, widths=8, t=8, seed=5):
    import paper_2410_02395_gb300 as pkg

    g = torch.Generator(device="cuda").manual_seed(seed)
    n = (1.0 + 0.5 * torch.rand(shape, generator=g, device="cuda")).to(torch.complex64)
    params = dict(shape=shape, pixel=pixel, wavelength=lam, widths=((widths, widths),) * 3,
                  periodic=(False, False, False), split=split)
    plan = pkg.Plan(shape, pixel, lam, n, boundary_widths=params["widths"], split=split, truncation=t)
    consts = host_constants(n.real.cpu().numpy(), params, t)
    info = plan.info()
    assert abs(info["k0sq"] - consts["k0sq"]) <= 1e-9 * abs(consts["k0sq"])
    assert abs(info["contrast"] - consts["contrast"]) <= 1e-6 * consts["contrast"]
    assert abs(info["c"] - consts["c"]) <= 1e-6 * abs(consts["c"])
    assert info["sizes"] == consts["sizes"] and info["a"] == consts["a"]
    x = torch.complex(torch.randn(shape, generator=g, device="cuda"), torch.randn(shape, generator=g, device="cuda"))
    out = plan.apply("A", x)
    torch.cuda.synchronize()
    rng = np.random.default_rng(seed)
    samples = _samples(shape, widths, t, consts["sizes"], rng)

    def x_pencil(v, d, lo, hi):
        idx = list(v)
        idx[d] = slice(lo, hi)
        return x[tuple(idx)].cpu().numpy().astype(np.complex128).reshape(-1)

    def n_at(v):
        return complex(n[v].item())

    want = sampled_A(consts, params, n_at, x_pencil, samples)
    got = np.array([complex(out[v].item()) for v in samples])
    plan.close()
    return got, want


def test_sampled_A_on_the_256_workload():
    got, want = _run((256, 256, 256), (2, 2, 2))
    err = np.abs(got - want) / np.abs(want).max()
    assert err.max() < 1e-5


def test_sampled_A_on_the_1280_workload():
    free, _ = torch.cuda.mem_get_info()
    if free < 160e9:
        pytest.skip("needs about 160 GB of free device memory")
    got, want = _run((1280, 1280, 1280), (4, 4, 4))
    err = np.abs(got - want) / np.abs(want).max()
    assert err.max() < 1e-5
