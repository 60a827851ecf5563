"""Clutterbox inputs (Section 4.1, steps 1-6a) on the CPU: levels, placement and indexing."""
import numpy as np
import pytest

import synth


def test_levels_add_one_object_each_and_keep_the_reference_first():
    levels = synth.scenes.clutterbox(seed=3, n=5, box_side=3.0, tri_lo=80, tri_hi=600)
    assert len(levels) == 5
    ref = levels[0]
    assert len(ref.mesh_vertex_offsets) == 1
    for k, lv in enumerate(levels, start=1):
        assert len(lv.mesh_vertex_offsets) == k
        # the reference object's vertices, normals and triangles are the first of every level
        assert np.array_equal(lv.vertices[: ref.num_vertices], ref.vertices)
        assert np.array_equal(lv.normals[: ref.num_vertices], ref.normals)
        assert np.array_equal(lv.triangles[: ref.num_triangles], ref.triangles)
        if k > 1:  # each level extends the previous one
            prev = levels[k - 2]
            assert np.array_equal(lv.vertices[: prev.num_vertices], prev.vertices)
            assert lv.num_vertices > prev.num_vertices


@pytest.mark.parametrize("s", [2.0, 3.0, 4.5])
def test_every_object_lies_inside_the_box(s):
    levels = synth.scenes.clutterbox(seed=4, n=6, box_side=s, tri_lo=80, tri_hi=600)
    v = levels[-1].vertices.astype(np.float64)
    assert np.abs(v).max() <= s / 2 + 1e-5
    # each object is fitted to the unit sphere (then rotated and moved): no two of its vertices
    # are more than 2 apart, and some are nearly 2 apart
    offs = levels[-1].mesh_vertex_offsets + [levels[-1].num_vertices]
    for a, b in zip(offs[:-1], offs[1:]):
        o = v[a:b]
        d = np.sqrt(((o[:, None, :] - o[None, :, :]) ** 2).sum(axis=2)).max()
        assert 1.5 < d <= 2.0 + 1e-5


def test_seeded_and_rejects_a_box_too_small_for_a_unit_sphere():
    a = synth.scenes.clutterbox(seed=5, n=3, tri_lo=80, tri_hi=600)
    b = synth.scenes.clutterbox(seed=5, n=3, tri_lo=80, tri_hi=600)
    assert all(np.array_equal(x.vertices, y.vertices) for x, y in zip(a, b))
    with pytest.raises(ValueError):
        synth.scenes.clutterbox(seed=5, n=3, box_side=1.5)
