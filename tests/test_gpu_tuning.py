"""Launch tunings change speed, never results; the autotuners measure and pick valid tunings.

Every generation tuning (warps per oriented point, and the grid cells per reach and
big-triangle radius that only the clutter measure and spin images read) must give images
bit-identical to the default tuning on a small batch of uneven clutter scenes (and to the oracle
on sampled origins under the most different tuning); every
tensor-core tile grouping must give the default's ranks, distances and top-1.  The autotuners
must return one of their candidates and leave the tuning in force unchanged, and the cached
tuner must store and apply its choice.
"""
import json

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

N, R = 64, 0.3


@pytest.fixture(scope="module")
def rici():
    import torch

    import paper_2007_02306_gb300 as p
    from paper_2007_02306_gb300 import build

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    p.load_library()
    p.set_tuning(None)
    yield p
    p.set_tuning(None)


@pytest.fixture(scope="module")
def scenes():
    import torch

    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    out = []
    for s in [synth.tiny_scene()] + synth.scene_batch(seed=43, n_scenes=3, tri_hi=30_000,
                                                      total_hi=80_000):
        out.append({"scene": s, "vertices": d(s.vertices), "normals": d(s.normals),
                    "triangles": d(s.triangles),
                    "origins": d(np.arange(s.num_vertices, dtype=np.int32))})
    return out


def images(rici, scenes):
    import torch

    outs = rici.rici_generate_batch(scenes, R, N)
    assert rici.sync_status() == 0
    return [o.view(torch.int16).cpu().numpy().view(np.uint16) for o in outs]


GEN_CANDIDATES = [{"gen_cells_per_reach": c, "gen_big_radius": b, "gen_warps": w, "tc_group_m": 8}
                  for c in (2, 3, 4) for b in (0.125, 0.25, 0.5, 1.0) for w in (4, 8)]


def test_every_generation_tuning_gives_the_same_images(rici, scenes, oracle_mod):
    rici.set_tuning(None)
    ref = images(rici, scenes)
    for t in GEN_CANDIDATES:
        rici.set_tuning(t)
        got = images(rici, scenes)
        for a, b in zip(got, ref):
            assert np.array_equal(a, b), t
    # the most different tuning against the oracle on sampled origins of the largest scene
    rici.set_tuning({"gen_cells_per_reach": 4, "gen_big_radius": 0.5, "gen_warps": 8,
                     "tc_group_m": 8})
    got = images(rici, scenes)
    rici.set_tuning(None)
    k = int(np.argmax([sc["scene"].num_triangles for sc in scenes]))
    s = scenes[k]["scene"]
    o = np.random.default_rng(3).choice(s.num_vertices, 12, replace=False).astype(np.int32)
    want = oracle_mod.rici_fp64(s.vertices, s.normals, s.triangles, o, R, N)
    assert np.array_equal(got[k][o], want)


def search_scenes(rici):
    import torch

    out = []
    for seed, (q, h) in enumerate([(200, 3000), (300, 700), (129, 5000)]):
        nd, hay, m = synth.images.needle_haystack_set(np.random.default_rng(seed), q, h, N)
        d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
        out.append({"needles": d(nd), "haystack": d(hay), "true_match": d(m)})
    return out


def test_every_tile_grouping_gives_the_same_ranks(rici):
    sc = search_scenes(rici)
    rici.set_tuning(None)
    ref = [{k: v.cpu().numpy() for k, v in r.items()} for r in rici.crss_search_batch(sc, N)]
    assert rici.sync_status() == 0
    for g in (1, 2, 3, 16, 64):
        rici.set_tuning(dict(rici.get_tuning(), tc_group_m=g))
        got = rici.crss_search_batch(sc, N)
        assert rici.sync_status() == 0
        for a, b in zip(got, ref):
            for k in b:
                assert np.array_equal(a[k].cpu().numpy(), b[k]), (g, k)
    rici.set_tuning(None)


def test_autotuners_pick_a_candidate_and_restore_the_tuning(rici, scenes):
    rici.set_tuning(None)
    before = rici.get_tuning()
    best, ms = rici.autotune_generate_batch(scenes, R, N, repeats=1)
    assert rici.get_tuning() == before and ms > 0
    assert best in GEN_CANDIDATES or dict(best, tc_group_m=8) in GEN_CANDIDATES
    assert rici.sync_status() == 0
    best, ms = rici.autotune_search_batch(search_scenes(rici), N, repeats=1)
    assert rici.get_tuning() == before and ms > 0
    assert best["tc_group_m"] in (2, 4, 8, 16, 32)
    assert rici.sync_status() == 0


def test_cached_tuner_stores_and_applies(rici, scenes, tmp_path):
    import torch

    from paper_2007_02306_gb300 import autotune

    path = str(tmp_path / "tuning.json")
    rici.set_tuning(None)
    name = torch.cuda.get_device_name()
    t = autotune.tune_batch(scenes, search_scenes(rici), R, N, gpu_name=name, sample=2, path=path)
    assert rici.get_tuning() == t
    assert len(json.load(open(path))) == 2
    # the tuned batch still produces the default's images
    got = images(rici, scenes)
    rici.set_tuning(None)
    ref = images(rici, scenes)
    for a, b in zip(got, ref):
        assert np.array_equal(a, b)
