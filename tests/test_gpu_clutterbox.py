"""Clutterbox driver (Section 4.1) on the GPU against the oracle: ranks and rank histograms of
every level of small seeded runs, bit for bit."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rici():
    import torch

    import paper_2007_02306_gb300 as p
    from paper_2007_02306_gb300 import build

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    p.load_library()
    return p


@pytest.mark.parametrize("mode", [0, 2])
def test_clutterbox_runs_match_the_oracle(rici, oracle_mod, mode):
    from paper_2007_02306_gb300 import clutterbox

    runs = [synth.scenes.clutterbox(seed=s, n=3, box_side=3.0, tri_lo=80, tri_hi=700)
            for s in (11, 12)]
    R, N = 0.3, 32
    got = clutterbox.run(runs, R, N, mode=mode, clutter=True)
    for levels, g in zip(runs, got):
        ref = levels[0]
        o_ref = np.arange(ref.num_vertices, dtype=np.int32)
        rd = oracle_mod.rici_fp64(ref.vertices, ref.normals, ref.triangles, o_ref, R, N)
        match = np.arange(ref.num_vertices, dtype=np.int64)
        for k, lv in enumerate(levels):
            o = np.arange(lv.num_vertices, dtype=np.int32)
            cd = oracle_mod.rici_fp64(lv.vertices, lv.normals, lv.triangles, o, R, N)
            r = oracle_mod.crss_search(rd, cd, match)["rank"]
            assert np.array_equal(g["ranks"][k], r), k
            h = np.bincount(r, minlength=lv.num_vertices)
            assert np.array_equal(g["histograms"][k], h), k
            assert g["rank0_fraction"][k] == pytest.approx(h[0] / r.size)
            # Eq. clutter around the reference vertices (object = the reference object)
            a_all, a_obj = oracle_mod.clutter_areas(lv.vertices, lv.normals, lv.triangles, o_ref,
                                                    np.float32(R), ref.num_vertices)
            c = (a_all - a_obj) / a_all
            assert np.abs(g["clutter"][k] - c).max() <= 1e-9, k
            assert g["heatmap"][k].sum() == r.size
            if k == 0:  # the reference alone: no clutter anywhere
                assert np.abs(g["clutter"][k]).max() <= 1e-12
        # level 1 searches the reference descriptors against themselves
        assert g["rank0_fraction"][0] == 1.0
