"""Seeded media and sources shaped like the paper's workloads.

The paper's structures are random packed spheres made with an external tool
(Sec. 4, first paragraph) that is not available here; the generators below draw
comparable structures from ``numpy.random.default_rng(seed)``. They return the
refractive index *without* absorbing layers (the solver adds those) and the
source map S of the Helmholtz equation (Sec. 2, Eq. helmholtz).

Nothing here computes any step of the modified Born series.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "frequency_batch",
    "spheres_medium",
    "fill_spheres_medium",
    "gaussian_random_field_medium",
    "point_source",
    "gaussian_beam_plane_source",
    "packed_spheres_medium",
    "plane_source",
    "random_field",
    "CONFIGS",
    "config_problem",
]


def _paint_sphere(n, centre, radius, value):
    """Set every voxel whose centre lies within ``radius`` of ``centre``."""
    lo = [max(0, int(np.floor(c - radius))) for c in centre]
    hi = [min(s, int(np.ceil(c + radius)) + 1) for c, s in zip(centre, n.shape)]
    if any(h <= l for l, h in zip(lo, hi)):
        return 0
    g = np.ogrid[lo[0]:hi[0], lo[1]:hi[1], lo[2]:hi[2]]
    d2 = (g[0] - centre[0]) ** 2 + (g[1] - centre[1]) ** 2 + (g[2] - centre[2]) ** 2
    mask = d2 <= radius * radius
    view = n[lo[0]:hi[0], lo[1]:hi[1], lo[2]:hi[2]]
    view[mask] = value
    return int(mask.sum())


def spheres_medium(shape, count, r_range, n_range, seed, background=1.0, margin=0,
                   dtype=np.complex64):
    """Background index plus ``count`` spheres painted in draw order.

    Radii are uniform in ``r_range`` (pixels), centres uniform in the box shrunk
    by ``margin`` pixels on every face, real indices uniform in ``n_range``.
    Later spheres overwrite earlier ones where they overlap.
    """
    rng = np.random.default_rng(seed)
    n = np.full(shape, background, dtype=dtype)
    for _ in range(count):
        r = rng.uniform(*r_range)
        c = [rng.uniform(margin, max(margin, s - margin)) for s in shape]
        v = rng.uniform(*n_range)
        _paint_sphere(n, c, r, v)
    return n


def fill_spheres_medium(shape, fill, r_range, n_range, seed, background=1.0, margin=0,
                        dtype=np.complex64, max_spheres=1_000_000):
    """Add random spheres (overlap allowed) until at least ``fill`` of the voxels differ
    from the background."""
    rng = np.random.default_rng(seed)
    n = np.full(shape, background, dtype=dtype)
    total = int(np.prod(shape))
    covered = np.zeros(shape, dtype=bool)
    ncov = 0
    for _ in range(max_spheres):
        if ncov >= fill * total:
            break
        r = rng.uniform(*r_range)
        c = [rng.uniform(margin, max(margin, s - margin)) for s in shape]
        v = rng.uniform(*n_range)
        lo = [max(0, int(np.floor(cc - r))) for cc in c]
        hi = [min(s, int(np.ceil(cc + r)) + 1) for cc, s in zip(c, shape)]
        if any(h <= l for l, h in zip(lo, hi)):
            continue
        g = np.ogrid[lo[0]:hi[0], lo[1]:hi[1], lo[2]:hi[2]]
        mask = (g[0] - c[0]) ** 2 + (g[1] - c[1]) ** 2 + (g[2] - c[2]) ** 2 <= r * r
        sl = (slice(lo[0], hi[0]), slice(lo[1], hi[1]), slice(lo[2], hi[2]))
        cv = covered[sl]
        ncov += int((mask & ~cv).sum())
        cv |= mask
        n[sl][mask] = v
    return n


def packed_spheres_medium(shape, radius, clearance, value, seed, background=1.0, margin=(0, 0, 0),
                          periodic=(False, False, False), max_failures=2000, dtype=np.complex64,
                          return_centres=False):
    """Spheres of one ``radius`` and index ``value`` placed by random sequential
    addition: candidate centres are drawn uniformly in the box shrunk by
    ``margin[d]`` pixels on both faces of axis d, and a candidate is kept when
    its centre lies at least 2 radius + clearance from every kept centre
    (distances wrap on the periodic axes). Placement stops after
    ``max_failures`` rejections in a row. Spheres that cross a periodic face are
    painted on both sides. The kind of structure the paper's large example uses
    (Sec. 4.3: tightly packed spheres of radius 6 wavelengths with a clearance of
    6 wavelengths, index 1.33 + 0.01i in a background of 1)."""
    rng = np.random.default_rng(seed)
    n = np.full(shape, background, dtype=dtype)
    dmin = 2.0 * radius + clearance
    cell = dmin
    ncell = [max(1, int(s // cell)) for s in shape]
    grid = {}
    centres = []
    lo = [float(m) for m in margin]
    hi = [float(s - m) for s, m in zip(shape, margin)]
    fails = 0
    while fails < max_failures:
        c = np.array([rng.uniform(l, max(l, h)) for l, h in zip(lo, hi)])
        key = [min(int(c[d] // cell), ncell[d] - 1) for d in range(3)]
        ok = True
        for off in np.ndindex(3, 3, 3):
            k = []
            for d in range(3):
                v = key[d] + off[d] - 1
                if periodic[d]:
                    v %= ncell[d]
                elif v < 0 or v >= ncell[d]:
                    break
                k.append(v)
            if len(k) < 3:
                continue
            for j in grid.get(tuple(k), ()):
                dv = np.abs(centres[j] - c)
                for d in range(3):
                    if periodic[d]:
                        dv[d] = min(dv[d], shape[d] - dv[d])
                if float(dv @ dv) < dmin * dmin:
                    ok = False
                    break
            if not ok:
                break
        if not ok:
            fails += 1
            continue
        fails = 0
        grid.setdefault(tuple(key), []).append(len(centres))
        centres.append(c)
    for c in centres:
        shifts = [[0.0] + ([float(shape[d]), -float(shape[d])] if periodic[d] else []) for d in range(3)]
        for s0 in shifts[0]:
            for s1 in shifts[1]:
                for s2 in shifts[2]:
                    _paint_sphere(n, (c[0] + s0, c[1] + s1, c[2] + s2), radius, value)
    if return_centres:
        return n, np.array(centres).reshape(-1, 3)
    return n


def plane_source(shape, axis=0, index=0, dtype=np.complex64):
    """Unit amplitude on the whole plane ``axis == index`` (a plane wave's source)."""
    s = np.zeros(shape, dtype=dtype)
    idx = [slice(None)] * 3
    idx[axis] = index
    s[tuple(idx)] = 1.0
    return s


def gaussian_random_field_medium(shape, mean, std, corr_len, seed, dtype=np.complex64):
    """``mean`` plus a Gaussian random field: white noise smoothed by the kernel
    exp(-r^2/corr_len^2) (covariance proportional to exp(-r^2/(2 corr_len^2))),
    rescaled to standard deviation ``std``. The smoothing is a periodic convolution
    done with numpy's real FFT (input synthesis only)."""
    rng = np.random.default_rng(seed)
    noise = rng.standard_normal(shape)
    spec = np.fft.rfftn(noise)
    g = []
    for s in shape:
        d = np.minimum(np.arange(s), s - np.arange(s)).astype(np.float64)
        g.append(np.exp(-(d ** 2) / corr_len ** 2))
    kern = np.fft.rfftn(g[0][:, None, None] * g[1][None, :, None] * g[2][None, None, :])
    field = np.fft.irfftn(spec * kern, s=shape)
    field -= field.mean()
    sd = field.std()
    if sd > 0:
        field *= std / sd
    return (mean + field).astype(dtype)


def point_source(shape, position=None, dtype=np.complex64):
    """Unit source in one voxel (default: the voxel at index shape//2)."""
    s = np.zeros(shape, dtype=dtype)
    if position is None:
        position = tuple(x // 2 for x in shape)
    s[tuple(position)] = 1.0
    return s


def gaussian_beam_plane_source(shape, axis=2, index=16, waist=64.0, dtype=np.complex64):
    """Flat-phase Gaussian profile exp(-rho^2/waist^2) on the plane ``axis == index``,
    rho measured in pixels from the centre of that plane."""
    s = np.zeros(shape, dtype=dtype)
    others = [a for a in range(3) if a != axis]
    c = [(shape[a] - 1) / 2.0 for a in others]
    g0 = (np.arange(shape[others[0]]) - c[0]) ** 2
    g1 = (np.arange(shape[others[1]]) - c[1]) ** 2
    prof = np.exp(-(g0[:, None] + g1[None, :]) / waist ** 2)
    idx = [slice(None)] * 3
    idx[axis] = index
    s[tuple(idx)] = prof
    return s


def random_field(shape, seed, dtype=np.complex64):
    """Complex field with independent standard normal real and imaginary parts."""
    rng = np.random.default_rng(seed)
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)).astype(dtype)


# Workload table. Sizes, media and sources follow the configurations the paper's
# experiments are shaped like (Sec. 4): 4 points per wavelength, random spheres,
# absorbing layers, point or plane sources.
CONFIGS = {
    "C1": dict(shape=(64, 64, 64), pixel=0.25, wavelength=1.0, split=(1, 1, 1),
               periodic=(True, True, True), widths=8, t=8, tol=1e-5,
               medium=("spheres", dict(count=6, r_range=(3, 8), n_range=(1.2, 1.5), seed=101, margin=8)),
               source=("point", dict())),
    "C2": dict(shape=(256, 256, 256), pixel=0.25, wavelength=1.0, split=(2, 2, 2),
               periodic=(False, False, False), widths=8, t=8, tol=1e-5,
               medium=("spheres", dict(count=40, r_range=(4, 20), n_range=(1.0, 1.6), seed=102, margin=8)),
               source=("point", dict())),
    "C3": dict(shape=(512, 512, 512), pixel=0.25, wavelength=1.0, split=(4, 4, 4),
               periodic=(False, False, False), widths=8, t=8, tol=1e-5,
               medium=("grf", dict(mean=1.33, std=0.08, corr_len=6.0, seed=103)),
               source=("beam", dict(axis=2, index=16, waist=64.0))),
    # C2 on an edge with a prime factor above 7 (subdomains of 123 = 3 x 41)
    "C2P": dict(shape=(246, 246, 246), pixel=0.25, wavelength=1.0, split=(2, 2, 2),
                periodic=(False, False, False), widths=8, t=8, tol=1e-5,
                medium=("spheres", dict(count=40, r_range=(4, 20), n_range=(1.0, 1.6), seed=102, margin=8)),
                source=("point", dict())),
    "C5": dict(shape=(1280, 1280, 1280), pixel=0.25, wavelength=1.0, split=(4, 4, 4),
               periodic=(False, False, False), widths=8, t=8, tol=1e-4,
               medium=("fill", dict(fill=0.30, r_range=(5, 40), n_range=(1.0, 1.5), seed=105, margin=8)),
               source=("point", dict())),
    # The geometry of the paper's large example (Sec. 4.3): 330 x 320 x 320
    # wavelengths at 4 points per wavelength, absorbing layers of 5 wavelengths on
    # the x faces only, y and z periodic, a plane source at x = 0 of the structure,
    # packed spheres of radius 6 and clearance 6 wavelengths. On one GPU the y and
    # z axes are split too (periodic seams), into 7-smooth subdomain edges.
    "P43": dict(shape=(1320, 1280, 1280), pixel=0.25, wavelength=1.0, split=(5, 4, 4),
                split_sizes=((280, 280, 256, 252, 252), (320,) * 4, (320,) * 4),
                periodic=(False, True, True), widths=((20, 20), (0, 0), (0, 0)), t=8, tol=1e-6,
                medium=("packed", dict(radius=24.0, clearance=24.0, value=1.33 + 0.01j, seed=107,
                                       margin=(44, 0, 0), periodic=(False, True, True))),
                source=("plane", dict(axis=0, index=20))),
}


def config_problem(name, shape=None):
    """Return ``(params, n, source)`` for a named workload.

    ``shape`` overrides the grid (for reduced-size cases); the medium recipe is
    kept. ``params`` holds the plan parameters as plain Python values.
    """
    cfg = dict(CONFIGS[name])
    if shape is not None:
        cfg["shape"] = tuple(shape)
    shp = tuple(cfg["shape"])
    kind, kw = cfg["medium"]
    if kind == "spheres":
        n = spheres_medium(shp, **kw)
    elif kind == "fill":
        n = fill_spheres_medium(shp, **kw)
    elif kind == "packed":
        n = packed_spheres_medium(shp, **kw)
    elif kind == "grf":
        n = gaussian_random_field_medium(shp, **kw)
    else:
        raise ValueError(kind)
    skind, skw = cfg["source"]
    if skind == "point":
        src = point_source(shp, **skw)
    elif skind == "beam":
        src = gaussian_beam_plane_source(shp, **skw)
    elif skind == "plane":
        src = plane_source(shp, **skw)
    else:
        raise ValueError(skind)
    w = cfg["widths"]
    widths = tuple(tuple(p) for p in w) if isinstance(w, tuple) else ((w, w), (w, w), (w, w))
    params = dict(shape=shp, pixel=cfg["pixel"], wavelength=cfg["wavelength"],
                  split=tuple(cfg["split"]), periodic=tuple(cfg["periodic"]),
                  widths=widths, t=cfg["t"], tol=cfg["tol"])
    if cfg.get("split_sizes") is not None and shape is None:  # explicit sizes hold for the full grid only
        params["split_sizes"] = [list(v) for v in cfg["split_sizes"]]
    return params, n, src


def _smooth7(v):
    for p in (2, 3, 5, 7):
        while v % p == 0 and v > 1:
            v //= p
    return v == 1


def _split2(total, lo=8):
    """Two 7-smooth parts of ``total``, as equal as possible (None if there are none)."""
    best = None
    for a in range(total // 2, lo - 1, -1):
        b = total - a
        if _smooth7(a) and _smooth7(b):
            if best is None or abs(b - a) < abs(best[1] - best[0]):
                best = (b, a) if b >= a else (a, b)
    return best


def frequency_batch(count=64, seed=104, box=24.0, lam_range=(0.8, 1.2), ppw=4, spheres=30,
                    r_range=(1.0, 5.0), n_range=(1.0, 1.5), widths=8, t=8, tol=1e-5):
    """Independent frequency solves on one physical box (transient simulations
    solve every frequency separately, Sec. 1): wavelength uniform in
    ``lam_range``, pixel lambda/ppw, grid round(box/pixel) (raised until it splits
    into two 7-smooth halves per axis), split 2x2x2; the same seeded spheres
    (centres, radii in the box's length unit) rasterised on every grid, a point
    source at the centre. Returns a list of ``(params, n, source)``."""
    rng = np.random.default_rng(seed)
    lams = rng.uniform(*lam_range, size=count)
    margin = 2.0
    sph = [(rng.uniform(margin, box - margin, size=3), rng.uniform(*r_range), rng.uniform(*n_range))
           for _ in range(spheres)]
    out = []
    for lam in lams:
        h = lam / ppw
        N = int(round(box / h))
        while _split2(N) is None:
            N += 1
        sizes = list(_split2(N))
        shp = (N, N, N)
        n = np.ones(shp, dtype=np.complex64)
        for c, r, v in sph:
            _paint_sphere(n, [ci / h for ci in c], r / h, v)
        src = point_source(shp)
        params = dict(shape=shp, pixel=h, wavelength=float(lam), split=(2, 2, 2), periodic=(False,) * 3,
                      widths=((widths, widths),) * 3, t=t, tol=tol, split_sizes=[sizes, sizes, sizes])
        out.append((params, n, src))
    return out

