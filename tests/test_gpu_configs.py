"""GPU parity on the benchmark workloads, with every oracle input computed by the oracle itself.

* Clutter scene (10 meshes, 229,756 triangles): every needle image (target alone, 10,242) and
  every haystack image (114,892) equal to the FP64 oracle, then every exact search form on the
  GPU images equal to the oracle's search of the oracle's images for 64 sampled needles.
* Precision form: 2^20 RICI images (N = 64, R = 0.3) of 6,473 seeded subdivision-2 icospheres
  with the stated heavy-tailed plateaus, 65,536 needles taken before clutter plateaus: every
  base image equal to the oracle's, all five fast search forms identical on every needle, and the
  oracle's ranks of 128 sampled needles against all 2^20 of its own images.
* Large scene (5,019,510 triangles): the 100,000 x 2,509,797 search on the scene's own RICI
  images (R = 0.3) with the int8 tensor-core form.  The oracle cannot image 2.5M points, so
  each of 6 sampled needles is checked on the images that decide its result: the oracle images
  the needle, its true match, its top-1, every haystack image the GPU finds strictly closer
  than the true match, and 24 random others, and their distances must equal the GPU's full
  distance row (an int64 kernel separate from the search), whose count of strictly closer
  images and first minimum must be the search's rank and top-1.
* Saturation: a bin crossed more than 65,535 times stores 65,535, as in the oracle.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

R = 0.3
N = 64
KEYS = ("true_distance", "rank", "top1")


@pytest.fixture(scope="module")
def rici():
    import torch

    import paper_2007_02306_gb300 as p
    from paper_2007_02306_gb300 import build

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    p.load_library()
    return p


def dev(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host_u16(t):
    import torch

    return t.view(torch.int16).cpu().numpy().view(np.uint16)


# ------------------------------------------------------------------ clutter scene

@pytest.fixture(scope="module")
def clutter(rici, oracle_mod):
    s = synth.clutter_scene()
    Vt, Tt = s.target_vertices, s.target_triangles
    on = np.arange(Vt, dtype=np.int32)
    oh = np.arange(s.num_vertices, dtype=np.int32)
    v, n, t = dev(s.vertices), dev(s.normals), dev(s.triangles)
    gnd = rici.rici_generate(v, n, t[:Tt], dev(on), R, N)
    ghy = rici.rici_generate(v, n, t, dev(oh), R, N)
    assert rici.sync_status() == 0
    tgt = s.target_only()
    ond = oracle_mod.rici_fp64(tgt.vertices, tgt.normals, tgt.triangles, on, R, N)
    ohy = oracle_mod.rici_fp64(s.vertices, s.normals, s.triangles, oh, R, N)
    return {"scene": s, "gpu_needles": gnd, "gpu_haystack": ghy, "needles": ond, "haystack": ohy}


def test_clutter_scene_every_image_equals_the_oracle(clutter):
    assert np.array_equal(host_u16(clutter["gpu_needles"]), clutter["needles"])
    hy = host_u16(clutter["gpu_haystack"])
    bad = np.nonzero((hy != clutter["haystack"]).any(axis=(1, 2)))[0]
    assert bad.size == 0, f"{bad.size} haystack images differ, first {bad[:8]}"


@pytest.mark.parametrize("mode", [1, 3, 4, 5, 6])
def test_clutter_scene_search_on_real_images(rici, oracle_mod, clutter, mode):
    Vt = clutter["scene"].target_vertices
    match = np.arange(Vt, dtype=np.int64)
    r = rici.crss_search(clutter["gpu_needles"], clutter["gpu_haystack"], dev(match), mode=mode)
    assert rici.sync_status() == 0
    got = {k: r[k].cpu().numpy() for k in KEYS}
    rng = np.random.default_rng(64)
    s = np.unique(np.concatenate([[0, Vt - 1], rng.choice(Vt, 62, replace=False)]))
    ref = oracle_mod.crss_search(clutter["needles"][s], clutter["haystack"], match[s])
    for k in KEYS:
        assert np.array_equal(got[k][s], ref[k]), k
    # the ranks are not all trivial: clutter moves some true matches off rank 0
    assert (got["rank"] > 0).any() and (got["rank"] == 0).any()


# ------------------------------------------------------------------ precision form

def test_precision_form_from_rici_images(rici, oracle_mod):
    import torch

    H, Q = 1 << 20, 65536
    scenes = synth.scenes.precision_form_scenes(31, 6473)
    tails, match, clutter_pl = synth.images.precision_form_recipe(31, H, Q, N)
    # base images: the GPU in one batched call, the oracle scene by scene
    gen = []
    for sc in scenes:
        gen.append({"vertices": dev(sc.vertices), "normals": dev(sc.normals),
                    "triangles": dev(sc.triangles),
                    "origins": dev(np.arange(sc.num_vertices, dtype=np.int32))})
    base = torch.empty((sum(sc.num_vertices for sc in scenes), N, N), dtype=torch.uint16,
                       device="cuda")
    k = 0
    for g, sc in zip(gen, scenes):
        g["out"] = base[k:k + sc.num_vertices]
        k += sc.num_vertices
    rici.rici_generate_batch(gen, R, N)
    assert rici.sync_status() == 0
    hay = base[:H]
    ohay = np.concatenate([oracle_mod.rici_fp64(sc.vertices, sc.normals, sc.triangles,
                                                np.arange(sc.num_vertices), R, N)
                           for sc in scenes])[:H]
    assert np.array_equal(host_u16(hay), ohay)
    del gen, base
    # heavy tails, needles, clutter: the same list applied on both sides
    synth.images.apply_plateaus_torch(hay, tails)
    synth.images.apply_plateaus(ohay, tails)
    nd = hay.view(torch.int16)[dev(match)].view(torch.uint16)  # copies
    ond = ohay[match].copy()
    synth.images.apply_plateaus_torch(hay, clutter_pl)
    synth.images.apply_plateaus(ohay, clutter_pl)
    assert np.array_equal(host_u16(nd), ond)
    ti = np.unique(tails["image"])
    d = np.diff(ohay[ti].astype(np.int32), axis=2)
    assert np.abs(d).max() > 127  # the tails reach the int64 path of every form
    m = dev(match)
    res = {}
    for mode in (3, 1, 4, 5, 6):
        r = rici.crss_search(nd, hay, m, mode=mode)
        assert rici.sync_status() == 0
        res[mode] = {k: r[k].cpu().numpy() for k in KEYS}
        del r
    for mode in (1, 4, 5, 6):
        for k in KEYS:
            assert np.array_equal(res[mode][k], res[3][k]), (mode, k)
    rng = np.random.default_rng(128)
    s = np.unique(np.concatenate([[0, Q - 1], rng.choice(Q, 126, replace=False)]))
    ref = oracle_mod.crss_search(ond[s], ohay, match[s])
    for k in KEYS:
        assert np.array_equal(res[3][k][s], ref[k]), k
    del hay, nd, m
    torch.cuda.empty_cache()


# ------------------------------------------------------------------ large scene

def test_large_scene_search_on_its_own_images(rici, oracle_mod):
    import torch

    s = synth.large_scene()
    V, Vt, Tt = s.num_vertices, s.target_vertices, s.target_triangles
    rng = np.random.default_rng(5)
    on = np.sort(rng.choice(Vt, 100_000, replace=False)).astype(np.int32)
    v, n, t = dev(s.vertices), dev(s.normals), dev(s.triangles)
    hay = rici.rici_generate(v, n, t, dev(np.arange(V, dtype=np.int32)), R, N)
    nd = rici.rici_generate(v, n, t[:Tt], dev(on), R, N)
    assert rici.sync_status() == 0
    match = on.astype(np.int64)
    r = rici.crss_search(nd, hay, dev(match), mode=rici.SEARCH_INT8_TC)
    assert rici.sync_status() == 0
    got = {k: r[k].cpu().numpy() for k in KEYS}
    del r
    pick = np.unique(np.concatenate([[0, len(on) - 1], rng.choice(len(on), 4, replace=False)]))
    sub = nd.view(torch.int16)[dev(pick)].view(torch.uint16)
    rows = rici.crss_search(sub, hay, dev(match[pick]), mode=rici.SEARCH_EXACT_SLOW,
                            return_distances=True)
    assert rici.sync_status() == 0
    dist = rows["distances"].cpu().numpy()
    tgt = s.target_only()
    for q, i in enumerate(pick):
        row = dist[q]
        dt = got["true_distance"][i]
        assert row[match[i]] == dt
        assert got["rank"][i] == int((row < dt).sum())
        assert got["top1"][i] == int(np.argmin(row))
        closer = np.nonzero(row < dt)[0]
        js = np.unique(np.concatenate([[match[i], got["top1"][i]], closer[:64],
                                       rng.choice(V, 24, replace=False)]))
        ond = oracle_mod.rici_fp64(tgt.vertices, tgt.normals, tgt.triangles, on[i:i + 1], R, N)
        ohy = oracle_mod.rici_fp64(s.vertices, s.normals, s.triangles, js, R, N)
        assert np.array_equal(host_u16(nd[int(i)])[None], ond)
        assert np.array_equal(host_u16(hay.view(torch.int16)[dev(js)]), ohy)
        od = oracle_mod.crss_search(np.repeat(ond, len(js), 0), ohy,
                                    np.arange(len(js), dtype=np.int64))["true_distance"]
        assert np.array_equal(od, row[js])
    del hay, nd
    torch.cuda.empty_cache()


# ------------------------------------------------------------------ saturation

def test_counts_saturate_at_uint16_max(rici, oracle_mod):
    # a vertical plane of 2 triangles crossing the support volume at distance 0.1 from the axis,
    # repeated 40,000 times: every circle of radius > 0.1 crosses it 80,000 times
    v = np.array([[0.1, -1.0, -1.0], [0.1, 1.0, -1.0], [0.1, 1.0, 1.0], [0.1, -1.0, 1.0],
                  [0.0, 0.0, 0.0]], np.float32)
    nrm = np.array([[1, 0, 0]] * 4 + [[0, 0, 1]], np.float32)
    tri = np.tile(np.array([[0, 1, 2], [0, 2, 3]], np.int32), (40_000, 1))
    got = host_u16(rici.rici_generate(dev(v), dev(nrm), dev(tri), dev(np.array([4], np.int32)),
                                      R, N))
    assert rici.sync_status() == 0
    ref = oracle_mod.rici_fp64(v, nrm, tri, [4], R, N)
    assert np.array_equal(got, ref)
    assert got.max() == 65535 and (got == 65535).sum() > N
