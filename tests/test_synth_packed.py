"""The seeded generators of the paper-geometry workload (packed spheres with a
clearance, periodic wrap on y and z, a plane source): invariants checked on the
CPU."""
import numpy as np

from synth import config_problem, packed_spheres_medium, plane_source


def _wrapped_distances(c, shape, periodic):
    d = np.abs(c[:, None, :] - c[None, :, :])
    for ax in range(3):
        if periodic[ax]:
            d[..., ax] = np.minimum(d[..., ax], shape[ax] - d[..., ax])
    return np.sqrt((d ** 2).sum(-1))


def test_packed_spheres_keep_their_clearance_across_periodic_faces():
    shape, r, cl, per = (80, 64, 64), 6.0, 4.0, (False, True, True)
    n, c = packed_spheres_medium(shape, r, cl, 1.33 + 0.01j, seed=3, margin=(10, 0, 0), periodic=per,
                                 return_centres=True)
    assert len(c) > 10
    dist = _wrapped_distances(c, shape, per)
    np.fill_diagonal(dist, np.inf)
    assert dist.min() >= 2 * r + cl - 1e-9
    assert (c[:, 0] >= 10).all() and (c[:, 0] <= shape[0] - 10).all()
    # every voxel within the radius of a centre (wrapped on y, z) holds the sphere's index
    g = np.stack(np.meshgrid(*[np.arange(s) for s in shape], indexing="ij"), -1).reshape(-1, 3).astype(float)
    inside = np.zeros(len(g), bool)
    for cc in c:
        d = np.abs(g - cc)
        for ax in (1, 2):
            d[:, ax] = np.minimum(d[:, ax], shape[ax] - d[:, ax])
        inside |= (d ** 2).sum(1) <= r * r
    flat = n.reshape(-1)
    assert np.all(flat[inside] == np.complex64(1.33 + 0.01j))
    assert np.all(flat[~inside] == 1.0)


def test_packed_spheres_are_seeded():
    a = packed_spheres_medium((40, 40, 40), 4.0, 2.0, 1.5, seed=9)
    b = packed_spheres_medium((40, 40, 40), 4.0, 2.0, 1.5, seed=9)
    c = packed_spheres_medium((40, 40, 40), 4.0, 2.0, 1.5, seed=10)
    assert np.array_equal(a, b) and not np.array_equal(a, c)


def test_plane_source_and_paper_geometry_recipe():
    s = plane_source((6, 5, 4), axis=0, index=2)
    assert s[2].sum() == 20 and np.count_nonzero(s) == 20
    params, n, src = config_problem("P43", shape=(66, 64, 64))
    assert params["periodic"] == (False, True, True)
    assert params["widths"] == ((20, 20), (0, 0), (0, 0))
    assert "split_sizes" not in params  # explicit sizes belong to the full grid
    assert np.count_nonzero(src) == 64 * 64 and np.all(src[20] == 1)


def test_paper_geometry_split_fits_the_library():
    """The full-size P43 split: the sizes add up to the grid, every edge is a
    mixed-radix length of at most 512 (2, 3, 5, 7 only) and at least 2t on every
    corrected axis, and the absorbing layers sit on the x faces only."""
    from synth import CONFIGS

    cfg = CONFIGS["P43"]
    shape, sizes, t = cfg["shape"], cfg["split_sizes"], cfg["t"]
    assert [sum(s) for s in sizes] == list(shape)
    assert [len(s) for s in sizes] == list(cfg["split"])
    for s in sizes:
        for n in s:
            m = n
            for q in (2, 3, 5, 7):
                while m % q == 0:
                    m //= q
            assert m == 1 and 2 * t <= n <= 512, n
    assert cfg["widths"] == ((20, 20), (0, 0), (0, 0)) and cfg["periodic"] == (False, True, True)
