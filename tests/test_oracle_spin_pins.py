"""Pins of the oracle's spin images (Section 2.1) and their point samples.

The definition is the FP64 form (``oracle.spin_images``: positions, projection and bilinear
weights in double, summed in double); the single-precision same-order mode
(``oracle.spin_images_fp32``, weights summed as integers in units of 2^-24) is a second check of
a GPU evaluation.  Every property below is checked on both, and the FP32 mode is pinned to the
FP64 definition by the per-bin deviation bound the FP64 form returns.

* the m^2 samples of a triangle lie in it, one in each of the m^2 congruent sub-triangles, and
  average to its centroid;
* a point sample at a bin centre puts its whole weight in that bin; midway between two centres
  it splits half and half; in general the four bilinear weights sum to 1 and reproduce the
  sample's (alpha, beta) as their weighted mean of bin centres;
* a small mesh well inside the support volume keeps its whole mass (m^2 per triangle);
* a rotation of the mesh about the central axis, or a mirror image through a plane containing
  it, leaves the image unchanged (up to the float rounding of the moved vertices);
* nothing outside the support volume contributes.
"""
import math

import numpy as np
import pytest

from synth import fixtures as F
from synth import meshes as M

R = float(np.float32(0.3))
N = 16


def tiny_triangle(centre, size=2e-6):
    c = np.asarray(centre, np.float64)
    return c + size * np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0]])


@pytest.fixture(params=["fp64", "fp32"])
def mode(request):
    return request.param


def image(v, t, m=3, n=N, mode="fp64"):
    import oracle

    fx = F._with_origin(v, t)
    fn = oracle.spin_images if mode == "fp64" else oracle.spin_images_fp32
    return fn(fx[0], fx[1], fx[2], [fx[3]], R, n, m)[0]


@pytest.mark.parametrize("m", [1, 2, 3, 5])
def test_samples_cover_the_triangle_uniformly(m):
    import oracle

    rng = np.random.default_rng(m)
    v = rng.uniform(-1, 1, size=(3, 3)).astype(np.float32)
    smp = oracle.spin_samples(v, [[0, 1, 2]], m)[0].astype(np.float64)
    assert smp.shape == (m * m, 3)
    A, B, C = v.astype(np.float64)
    np.testing.assert_allclose(smp.mean(axis=0), (A + B + C) / 3, atol=1e-6)
    # barycentric coordinates of the samples: inside, and one per sub-triangle
    M2 = np.stack([B - A, C - A], 1)
    ab = np.linalg.lstsq(M2, (smp - A).T, rcond=None)[0].T
    assert (ab > 0).all() and (ab.sum(axis=1) < 1).all()
    cells = set()
    for a, b in ab:
        i, j = math.floor(a * m), math.floor(b * m)
        cells.add((i, j, (a * m - i) + (b * m - j) < 1.0))  # upward or downward sub-triangle
    assert len(cells) == m * m


def bin_centre(c, r):
    return (c + 0.5) * R / N, (r + 0.5 - N / 2) * R / N


def test_sample_at_a_bin_centre_fills_one_bin(mode):
    a, b = bin_centre(5, 9)
    img = image(tiny_triangle([a, 0.0, b]), [[0, 1, 2]], m=3, mode=mode)
    assert img.sum() == pytest.approx(9.0, rel=1e-5)
    assert img[9, 5] == pytest.approx(9.0, rel=1e-3)


def test_sample_between_two_centres_splits_evenly(mode):
    a0, b = bin_centre(5, 9)
    a1, _ = bin_centre(6, 9)
    img = image(tiny_triangle([0.5 * (a0 + a1), 0.0, b]), [[0, 1, 2]], m=2, mode=mode)
    assert img[9, 5] == pytest.approx(2.0, rel=1e-3)
    assert img[9, 6] == pytest.approx(2.0, rel=1e-3)
    assert img.sum() == pytest.approx(4.0, rel=1e-5)


@pytest.mark.parametrize("seed", range(5))
def test_bilinear_weights_reproduce_the_sample_position(seed, mode):
    rng = np.random.default_rng(seed)
    alpha = rng.uniform(1.0, N - 1.0) * R / N
    beta = (rng.uniform(1.0, N - 1.0) - N / 2) * R / N
    phi = rng.uniform(0, 2 * math.pi)
    img = image(tiny_triangle([alpha * math.cos(phi), alpha * math.sin(phi), beta], 1e-7),
                [[0, 1, 2]], m=1, mode=mode).astype(np.float64)
    assert img.sum() == pytest.approx(1.0, abs=1e-6)
    r, c = np.nonzero(img)
    assert len(r) <= 4
    ca = sum(img[i, j] * bin_centre(j, i)[0] for i, j in zip(r, c))
    cb = sum(img[i, j] * bin_centre(j, i)[1] for i, j in zip(r, c))
    assert ca == pytest.approx(alpha, abs=2e-6)
    assert cb == pytest.approx(beta, abs=2e-6)


def test_small_mesh_inside_keeps_its_mass_and_is_invariant(mode):
    rng = np.random.default_rng(7)
    m = M.displaced_icosphere(rng, 2)
    v = m.vertices * 0.06 + np.array([0.12, 0.03, -0.01])
    img = image(v, m.triangles, m=3, mode=mode)
    assert img.sum() == pytest.approx(9 * m.num_triangles, rel=1e-5)
    # rotation about the central axis (z) and a mirror image through the xz plane
    for rot in (np.array([[math.cos(1.1), -math.sin(1.1), 0], [math.sin(1.1), math.cos(1.1), 0],
                          [0, 0, 1]]), np.diag([1.0, -1.0, 1.0])):
        img2 = image(v @ rot.T, m.triangles, m=3, mode=mode)
        assert np.abs(img2 - img).max() <= 2e-3 * img.max()


def test_geometry_outside_the_volume_adds_nothing(mode):
    # beyond the radius, above the slab, below the slab
    for centre in ([0.31, 0.0, 0.0], [0.0, 0.1, 0.16], [0.1, 0.0, -0.151]):
        assert image(tiny_triangle(centre), [[0, 1, 2]], mode=mode).sum() == 0.0


def test_fp64_bilinear_weights_are_exact_at_dyadic_positions():
    # alpha and beta on dyadic fractions of a bin (R = 1, N = 8: bins of 1/8): the four weights
    # are exact products of (1 - fu), fu, (1 - fv), fv with fu = 1/4, fv = 3/8
    import oracle

    Rd, Nd = 1.0, 8
    alpha = (3 + 0.5 + 0.25) / Nd          # u = 3.25
    beta = (5 + 0.5 + 0.375) / Nd - 0.5    # v = 5.375
    v = tiny_triangle([alpha, 0.0, beta], 1e-9)
    fx = F._with_origin(v, [[0, 1, 2]])
    img = oracle.spin_images(fx[0], fx[1], fx[2], [fx[3]], Rd, Nd, 1)[0].astype(np.float64)
    want = {(5, 3): 0.75 * 0.625, (5, 4): 0.25 * 0.625, (6, 3): 0.75 * 0.375, (6, 4): 0.25 * 0.375}
    for (r, c), w in want.items():
        assert img[r, c] == pytest.approx(w, abs=1e-6)
    assert img.sum() == pytest.approx(1.0, abs=1e-6)


def _scenes():
    import synth

    yield synth.tiny_scene(), 32, 3
    yield synth.tiny_scene(4), 64, 2
    sc = synth.scenes.clutter_scene(seed=6, target_subdivisions=3, n_clutter=3, tri_lo=500,
                                    tri_hi=4000)
    yield sc, 64, 3


def test_fp32_mode_lies_within_the_bound_of_the_fp64_definition():
    import oracle

    for s, n, m in _scenes():
        rng = np.random.default_rng(n)
        o = np.unique(rng.integers(0, s.num_vertices, 48)).astype(np.int32)
        ref, bound = oracle.spin_images(s.vertices, s.normals, s.triangles, o, R, n, m,
                                        return_bound=True)
        f32 = oracle.spin_images_fp32(s.vertices, s.normals, s.triangles, o, R, n, m)
        dev = np.abs(f32.astype(np.float64) - ref.astype(np.float64))
        assert (dev <= bound).all(), (dev / bound).max()
        assert ref.sum() > 0
        # the bound is a small fraction of the mass, so it cannot hide a misplaced weight
        assert bound.sum() < 5e-3 * ref.sum()
        assert np.median(bound[ref > 1]) < 1e-2


def test_bound_grows_where_a_sample_sits_on_the_volume_boundary():
    # a sample at alpha = R exactly may be inside or outside in single precision: its bins
    # carry the whole weight in the bound
    import oracle

    v = tiny_triangle([R, 0.0, 0.01], 1e-9)
    fx = F._with_origin(v, [[0, 1, 2]])
    img, bound = oracle.spin_images(fx[0], fx[1], fx[2], [fx[3]], R, N, 1, return_bound=True)
    assert bound[0].max() >= 1.0
