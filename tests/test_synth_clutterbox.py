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


def test_histograms_and_heatmaps_on_the_host():
    """The driver's host-side binning: rank histograms, rank-0 fractions, clutter fractions and
    the clutter-versus-rank heatmap (no GPU: device results are stood in for by CPU tensors)."""
    import torch

    from paper_2007_02306_gb300 import clutterbox

    prep = {"sizes": [[4, 200]]}  # one run: level 1 (4 reference vertices), level 2 (200 images)
    results = [{"rank": torch.tensor([0, 0, 0, 0], dtype=torch.int32)},
               {"rank": torch.tensor([0, 3, 0, 120], dtype=torch.int32)}]
    # stand-ins for the library's (A_all, A_object, clutter) tensors
    a_all = torch.tensor([1.0, 2.0, 4.0, 1.0], dtype=torch.float64)
    a_obj = torch.tensor([1.0, 1.0, 0.4, 0.05], dtype=torch.float64)
    areas = [(a_all, a_all.clone(), torch.zeros(4, dtype=torch.float64)),
             (a_all, a_obj, (a_all - a_obj) / a_all)]
    h = clutterbox.histograms(prep, results, areas, clutter_bins=10)[0]
    assert h["rank0_fraction"] == [1.0, 0.5]
    hist = h["histograms"][1]
    assert hist.size == 200 and hist.sum() == 4
    assert hist[0] == 2 and hist[3] == 1 and hist[120] == 1
    np.testing.assert_allclose(h["clutter"][0], 0.0)
    np.testing.assert_allclose(h["clutter"][1], [0.0, 0.5, 0.9, 0.95])
    heat = h["heatmap"][1]
    assert heat.shape == (10, len(clutterbox.RANK_EDGES) - 1)
    assert heat.sum() == 4
    assert heat[0, 0] == 1      # clutter 0, rank 0
    assert heat[5, 2] == 1      # clutter 0.5, rank 3 (bin 2-4)
    assert heat[9, 0] == 1      # clutter 0.9, rank 0
    assert heat[9, 7] == 1      # clutter 0.95, rank 120 (bin 100-999)
