"""Pins of the oracle's FP32 same-operation-order mode (CPU).

- The FP32 projection stays within the error bound the generation kernel relies on,
  |T32 - T64| <= 10 u (|dx| + |dy| + |dz|), u = 2^-24, on random points and normals.
- With an axis-aligned normal and a mesh on a coarse dyadic grid every FP32 operation is exact,
  so the FP32 images equal the FP64 definition and no item differs.
- A vertical edge whose squared distance to the axis lies just below a bin's alpha^2 but rounds
  onto it in FP32 is outside that circle in FP64 and on it in FP32: the FP32 mode must report the
  item as differing and its image must differ from the FP64 image in that column.
"""
import numpy as np

from synth import fixtures as F

U = 2.0 ** -24


def test_projection_error_bound(oracle_mod):
    rng = np.random.default_rng(7)
    for _ in range(50):
        s = rng.uniform(-2, 2, 3).astype(np.float32)
        n = rng.normal(size=3).astype(np.float32)
        p = (s + rng.uniform(-0.5, 0.5, (200, 3))).astype(np.float32)
        t32 = oracle_mod.project_fp32(p, s, n).astype(np.float64)
        t64 = oracle_mod.project_fp64(p, s, n)
        d = p.astype(np.float64) - s.astype(np.float64)
        bound = 10 * U * np.abs(d).sum(axis=1, keepdims=True)
        assert (np.abs(t32 - t64) <= bound).all()


def dyadic_scene():
    # a fan of triangles around the origin vertex, coordinates on a 1/64 grid
    v = [(0.0, 0.0, 0.0)]
    t = []
    ring = [(0.125, 0.0), (0.0625, 0.125), (-0.0625, 0.1875), (-0.1875, 0.0), (-0.0625, -0.125),
            (0.1875, -0.0625)]
    for k, (x, y) in enumerate(ring):
        v.append((x, y, -0.125 + 0.046875 * k))
    for k in range(len(ring)):
        t.append((0, 1 + k, 1 + (k + 1) % len(ring)))
    v = np.array(v, np.float32)
    n = np.tile(np.array([0.0, 0.0, 1.0], np.float32), (len(v), 1))
    return v, n, np.array(t, np.int32)


def test_exact_inputs_give_identical_images(oracle_mod):
    v, n, t = dyadic_scene()
    o = np.arange(len(v), dtype=np.int32)
    want = oracle_mod.rici_fp64(v, n, t, o, 0.5, 16)
    got, cnt = oracle_mod.rici_fp32(v, n, t, o, 0.5, 16)
    assert cnt["crossings"] > 0
    assert cnt["items_differing_from_fp64"] == 0
    assert np.array_equal(got, want)


def test_fp32_alone_decides_a_near_tie_differently(oracle_mod):
    v, n, t, c = F.radius_tie_scene()
    o = np.array([0], np.int32)
    want = oracle_mod.rici_fp64(v, n, t, o, 0.3, 64)
    got, cnt = oracle_mod.rici_fp32(v, n, t, o, 0.3, 64)
    assert cnt["items_differing_from_fp64"] >= 1
    assert not np.array_equal(got[0][:, c], want[0][:, c])
