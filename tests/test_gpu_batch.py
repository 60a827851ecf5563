"""Batched run: many scenes of uneven size generated and searched in one set of launches.

Scenes follow the batched workload's recipe (a target plus 1-15 clutter meshes of uneven size;
here 24 scenes of 10k-300k triangles so the test stays short).  Per scene: needle images of a
seeded sample of target vertices with the target alone, haystack images of every scene vertex,
and a tensor-core search of the needles against their own scene.  The batched results must equal
one rici_generate / crss_search call per scene bit for bit, sampled images (and every image and
rank of the two smallest scenes, from the oracle's own images) must equal the oracle, every exact
search form must agree, and the whole batched run recorded into a CUDA graph must replay to the
same results.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

N, R, NEEDLES = 64, 0.3, 256


@pytest.fixture(scope="module")
def rici():
    import torch

    import paper_2007_02306_gb300 as p
    from paper_2007_02306_gb300 import build

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    p.load_library()
    return p


@pytest.fixture(scope="module")
def batch():
    import torch

    scenes = synth.scene_batch(seed=41, n_scenes=24, tri_hi=60_000, total_hi=300_000)
    rng = np.random.default_rng(2)
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    out = []
    for s in scenes:
        q = min(NEEDLES, s.target_vertices)
        needle_o = np.sort(rng.choice(s.target_vertices, q, replace=False)).astype(np.int32)
        out.append({
            "scene": s, "needle_origins": needle_o,
            "V": d(s.vertices), "Nrm": d(s.normals), "T": d(s.triangles),
            "Tt": d(s.triangles[: s.target_triangles]),
            "on": d(needle_o), "oh": d(np.arange(s.num_vertices, dtype=np.int32)),
            "match": d(needle_o.astype(np.int64)),
        })
    return out


def host_u16(t):
    import torch

    return t.view(torch.int16).cpu().numpy().view(np.uint16)


def run_batch(rici, b, ws_gen=None, ws_search=None, gen_outs=None, search_outs=None):
    gen = []
    k = 0
    for x in b:
        gen.append({"vertices": x["V"], "normals": x["Nrm"], "triangles": x["Tt"], "origins": x["on"],
                    "out": None if gen_outs is None else gen_outs[k]})
        gen.append({"vertices": x["V"], "normals": x["Nrm"], "triangles": x["T"], "origins": x["oh"],
                    "out": None if gen_outs is None else gen_outs[k + 1]})
        k += 2
    imgs = rici.rici_generate_batch(gen, R, N, workspace_tensor=ws_gen)
    srch = [{"needles": imgs[2 * i], "haystack": imgs[2 * i + 1], "true_match": x["match"]}
            for i, x in enumerate(b)]
    res = rici.crss_search_batch(srch, N, workspace_tensor=ws_search, outputs=search_outs)
    return imgs, res


def test_batch_equals_per_scene_calls_and_oracle(rici, oracle_mod, batch):
    imgs, res = run_batch(rici, batch)
    assert rici.sync_status() == 0
    rng = np.random.default_rng(9)
    for i, x in enumerate(batch):
        s = x["scene"]
        nd = rici.rici_generate(x["V"], x["Nrm"], x["Tt"], x["on"], R, N)
        hy = rici.rici_generate(x["V"], x["Nrm"], x["T"], x["oh"], R, N)
        one = rici.crss_search(nd, hy, x["match"], mode=rici.SEARCH_TENSOR)
        assert rici.sync_status() == 0
        assert np.array_equal(host_u16(imgs[2 * i]), host_u16(nd))
        assert np.array_equal(host_u16(imgs[2 * i + 1]), host_u16(hy))
        for k in ("rank", "true_distance", "top1"):
            assert np.array_equal(res[i][k].cpu().numpy(), one[k].cpu().numpy()), (i, k)
        if i % 6 == 0:  # oracle: sampled haystack images of some scenes
            pick = rng.choice(s.num_vertices, 3, replace=False)
            ref = oracle_mod.rici_fp64(s.vertices, s.normals, s.triangles, pick, R, N)
            assert np.array_equal(host_u16(imgs[2 * i + 1])[pick], ref)
    # oracle: the two smallest scenes in full, images and ranks computed from the oracle's own
    # images (needles with the target alone, haystack with the whole scene)
    small = sorted(range(len(batch)), key=lambda i: batch[i]["scene"].num_triangles)[:2]
    for i in small:
        x, s = batch[i], batch[i]["scene"]
        tgt = s.target_only()
        ond = oracle_mod.rici_fp64(tgt.vertices, tgt.normals, tgt.triangles, x["needle_origins"],
                                   R, N)
        ohy = oracle_mod.rici_fp64(s.vertices, s.normals, s.triangles,
                                   np.arange(s.num_vertices), R, N)
        assert np.array_equal(host_u16(imgs[2 * i]), ond)
        assert np.array_equal(host_u16(imgs[2 * i + 1]), ohy)
        ro = oracle_mod.crss_search(ond, ohy, x["needle_origins"].astype(np.int64))
        for k in ("rank", "true_distance", "top1"):
            assert np.array_equal(res[i][k].cpu().numpy(), ro[k]), (i, k)


@pytest.mark.parametrize("mode", [1, 4, 5, 6])
def test_batch_search_forms_agree(rici, batch, mode):
    """Every exact form of the multi-scene search gives the tensor-core form's ranks, true
    distances and top-1 on the batch's images (each needle against its own scene only)."""
    imgs, res = run_batch(rici, batch)
    srch = [{"needles": imgs[2 * i], "haystack": imgs[2 * i + 1], "true_match": x["match"]}
            for i, x in enumerate(batch)]
    other = rici.crss_search_batch(srch, N, mode=mode)
    assert rici.sync_status() == 0
    for i in range(len(batch)):
        for k in ("rank", "true_distance", "top1"):
            assert np.array_equal(other[i][k].cpu().numpy(), res[i][k].cpu().numpy()), (i, k)


def test_batch_run_replays_from_a_cuda_graph(rici, batch):
    import torch

    imgs, res = run_batch(rici, batch)  # eager reference (also sizes the workspaces)
    torch.cuda.synchronize()
    ref = [{k: v.clone() for k, v in r.items()} for r in res]
    gen_outs = [torch.empty_like(t) for t in imgs]
    search_outs = [{k: torch.empty_like(v) for k, v in r.items()} for r in res]
    gen_scenes = []
    for x in batch:
        gen_scenes.append({"vertices": x["V"], "normals": x["Nrm"], "triangles": x["Tt"], "origins": x["on"]})
        gen_scenes.append({"vertices": x["V"], "normals": x["Nrm"], "triangles": x["T"], "origins": x["oh"]})
    ws_gen = torch.empty(rici.binding.generate_batch_workspace_bytes(gen_scenes, N) + 256,
                         dtype=torch.uint8, device="cuda")
    srch = [{"needles": gen_outs[2 * i], "haystack": gen_outs[2 * i + 1]} for i in range(len(batch))]
    ws_s = torch.empty(rici.binding.search_batch_workspace_bytes(srch, N) + 256, dtype=torch.uint8,
                       device="cuda")
    off_g = (-ws_gen.data_ptr()) % 256
    off_s = (-ws_s.data_ptr()) % 256
    wg, wsr = ws_gen[off_g:], ws_s[off_s:]
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        run_batch(rici, batch, wg, wsr, gen_outs, search_outs)  # warm-up on the capture stream
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        run_batch(rici, batch, wg, wsr, gen_outs, search_outs)
    for _ in range(2):
        for o in search_outs:
            for v in o.values():
                v.fill_(-7)
        g.replay()
        torch.cuda.synchronize()
        assert rici.sync_status() == 0
        for r0, r1 in zip(ref, search_outs):
            for k in r0:
                assert torch.equal(r0[k], r1[k]), k
        for a, b2 in zip(imgs, gen_outs):
            assert torch.equal(a.view(torch.int16), b2.view(torch.int16))


def run_single_call(rici, b, ws=None, outputs=None):
    scenes = [{"vertices": x["V"], "normals": x["Nrm"], "triangles": x["T"],
               "target_triangles": x["scene"].target_triangles, "needle_origins": x["on"],
               "haystack_origins": x["oh"], "true_match": x["match"]} for x in b]
    return rici.batch_run(scenes, R, N, workspace_tensor=ws, outputs=outputs), scenes


def test_single_call_batch_run_equals_the_two_batched_calls(rici, batch):
    imgs, res = run_batch(rici, batch)
    one, _ = run_single_call(rici, batch)
    assert rici.sync_status() == 0
    for i in range(len(batch)):
        assert np.array_equal(host_u16(one[i]["needle_images"]), host_u16(imgs[2 * i]))
        assert np.array_equal(host_u16(one[i]["haystack_images"]), host_u16(imgs[2 * i + 1]))
        for k in ("rank", "true_distance", "top1"):
            assert torch_equal(one[i][k], res[i][k]), (i, k)


def torch_equal(a, b):
    import torch

    return bool(torch.equal(a, b))


def test_single_call_batch_run_replays_from_a_cuda_graph(rici, batch):
    import torch

    ref, scenes = run_single_call(rici, batch)
    torch.cuda.synchronize()
    ref = [{k: v.clone() for k, v in r.items()} for r in ref]
    outs = [{k: torch.empty_like(v) for k, v in r.items()} for r in ref]
    nb = rici.binding.batch_run_workspace_bytes(scenes, N, outs)
    ws = torch.empty(nb + 256, dtype=torch.uint8, device="cuda")
    ws = ws[(-ws.data_ptr()) % 256:]
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        run_single_call(rici, batch, ws, outs)  # warm-up on the capture stream
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        run_single_call(rici, batch, ws, outs)
    for o in outs:
        for v in o.values():
            v.fill_(7)
    g.replay()
    torch.cuda.synchronize()
    assert rici.sync_status() == 0
    for r0, r1 in zip(ref, outs):
        for k in r0:
            assert torch.equal(r0[k], r1[k]), k


def test_per_call_tuning_gives_the_same_results_and_leaves_the_setting(rici, batch):
    """rici_batch_run_ex: a tuning in force for one call only (different grid, warps and tile
    grouping) gives the results of the process-wide setting, and does not change that setting."""
    scenes = [{"vertices": x["V"], "normals": x["Nrm"], "triangles": x["T"],
               "target_triangles": x["scene"].target_triangles, "needle_origins": x["on"],
               "haystack_origins": x["oh"], "true_match": x["match"]} for x in batch[:6]]
    rici.set_tuning(None)
    before = rici.get_tuning()
    ref = rici.batch_run(scenes, R, N)
    other = {"gen_cells_per_reach": 4, "gen_big_radius": 1.0, "gen_warps": 8, "tc_group_m": 3}
    got = rici.batch_run(scenes, R, N, tuning=other)
    assert rici.sync_status() == 0
    assert rici.get_tuning() == before
    for a, b in zip(ref, got):
        for k in ("needle_images", "haystack_images"):
            assert np.array_equal(host_u16(a[k]), host_u16(b[k])), k
        for k in ("rank", "true_distance", "top1"):
            assert np.array_equal(a[k].cpu().numpy(), b[k].cpu().numpy()), k
