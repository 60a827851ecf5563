"""GPU parity of RICI generation against the FP64 CPU oracle: bit-exact images.

Sizes: the tiny scene (all origins), fixtures with closed forms, constructed near-ties that
force the FP64 re-evaluation path, edge cases (no triangles, odd and maximal resolutions,
zero normals, repeated origins) and the full clutter scene that the benchmark times
(230k triangles, every scene vertex imaged) checked on sampled origins.
"""
import numpy as np
import pytest

import synth
from synth import fixtures as F

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


def dev(a, dtype=None):
    import torch

    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def gpu_images(rici, v, n, t, o, R, N, mode=0, counters=None):
    import torch

    out = rici.rici_generate(dev(v, torch.float32), dev(n, torch.float32), dev(t, torch.int32),
                             dev(np.asarray(o), torch.int32), R, N, mode=mode, counters=counters)
    st = rici.sync_status()
    assert st == 0, f"device status {st}"
    return out.cpu().numpy()


@pytest.mark.parametrize("N", [32, 64])
def test_tiny_scene_all_origins_bit_exact(rici, oracle_mod, N):
    s = synth.tiny_scene()
    o = np.arange(s.num_vertices)
    ref = oracle_mod.rici_fp64(s.vertices, s.normals, s.triangles, o, 0.3, N)
    got = gpu_images(rici, s.vertices, s.normals, s.triangles, o, 0.3, N)
    assert np.array_equal(got, ref)


def test_fp64_mode_bit_exact(rici, oracle_mod):
    s = synth.tiny_scene(9)
    o = np.arange(s.num_vertices)
    ref = oracle_mod.rici_fp64(s.vertices, s.normals, s.triangles, o, 0.3, 32)
    got = gpu_images(rici, s.vertices, s.normals, s.triangles, o, 0.3, 32, mode=rici.GEN_FP64)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("N,R", [(1, 0.3), (7, 0.3), (8, 0.5), (33, 0.2), (128, 0.3), (64, 1.7)])
def test_resolutions_and_radii(rici, oracle_mod, N, R):
    s = synth.tiny_scene(2)
    o = np.arange(0, s.num_vertices, 3)
    ref = oracle_mod.rici_fp64(s.vertices, s.normals, s.triangles, o, R, N)
    got = gpu_images(rici, s.vertices, s.normals, s.triangles, o, R, N)
    assert np.array_equal(got, ref)


def test_closed_form_fixtures(rici, oracle_mod):
    for v, n, t, o in (F.vertical_plane(0.1513), F.vertical_cylinder(0.12, 0.05),
                       F.off_axis_sphere(0.13, 0.02, 0.09, subdivisions=5)):
        ref = oracle_mod.rici_fp64(v, n, t, [o], 0.3, 64)
        got = gpu_images(rici, v, n, t, [o], 0.3, 64)
        assert np.array_equal(got, ref)


def test_near_ties_take_fp64_path_and_stay_exact(rici, oracle_mod):
    """Dyadic vertices on layer planes and on circle radii: predicates with zero margin."""
    import torch

    N, R = 16, 0.5
    rng = np.random.default_rng(8)
    # coordinates on a 1/64 grid: beta_r = (2r-15)/64 and alpha_c = (2c+1)/64 are hit exactly
    v = (rng.integers(-20, 21, size=(400, 3)) / 64.0).astype(np.float32)
    t = np.stack([rng.choice(400, 3, replace=False) for _ in range(1500)]).astype(np.int32)
    origins_v = np.zeros((6, 3), np.float32)
    origins_n = np.array([(0, 0, 1), (0, 0, -1), (1, 0, 0), (0, 1, 0), (0, 0, 3), (0, -2, 0)], np.float32)
    V = np.concatenate([v, origins_v])
    Nr = np.concatenate([np.zeros_like(v), origins_n])
    o = np.arange(400, 406)
    ref = oracle_mod.rici_fp64(V, Nr, t, o, R, N)
    cnt = torch.zeros(4, dtype=torch.int64, device="cuda")
    got = gpu_images(rici, V, Nr, t, o, R, N, counters=cnt)
    assert np.array_equal(got, ref)
    c = cnt.cpu().numpy()
    assert c[2] > 0, f"expected FP64 band re-evaluations, counters={c}"


def test_random_triangle_soup_exact(rici, oracle_mod):
    rng = np.random.default_rng(21)
    v = rng.uniform(-0.4, 0.4, size=(3000, 3)).astype(np.float32)
    t = rng.integers(0, 3000, size=(6000, 3)).astype(np.int32)
    n = rng.normal(size=(3000, 3)).astype(np.float32)
    n[::50] = 0.0  # zero normals select the identity rotations
    o = rng.integers(0, 3000, size=300)
    o[:10] = o[0]  # repeated origins
    ref = oracle_mod.rici_fp64(v, n, t, o, 0.3, 64)
    got = gpu_images(rici, v, n, t, o, 0.3, 64)
    assert np.array_equal(got, ref)


def test_large_and_degenerate_triangles(rici, oracle_mod):
    rng = np.random.default_rng(5)
    v = rng.uniform(-3, 3, size=(300, 3)).astype(np.float32)  # triangles far larger than R
    v[:20] = rng.uniform(-0.1, 0.1, size=(20, 3))
    t = rng.integers(0, 300, size=(800, 3)).astype(np.int32)
    t[:30, 1] = t[:30, 0]  # degenerate: repeated vertex
    n = rng.normal(size=(300, 3)).astype(np.float32)
    o = np.arange(20)
    ref = oracle_mod.rici_fp64(v, n, t, o, 0.3, 32)
    got = gpu_images(rici, v, n, t, o, 0.3, 32)
    assert np.array_equal(got, ref)


def test_coarse_curve_order_exact(rici, oracle_mod):
    """One far triangle stretches the scene's box of triangle centres, so every other triangle
    falls into one Morton bin and the sorted records follow no curve: the bounding spheres of
    their chunks and groups are then as wide as the mesh, and the images must not change."""
    m = synth.meshes.displaced_icosphere(np.random.default_rng(8), 4)  # 5,120 triangles
    far = np.array([[1e4, 1e4, 1e4], [1e4 + 1, 1e4, 1e4], [1e4, 1e4 + 1, 1e4]])
    v = np.concatenate([m.vertices, far]).astype(np.float32)
    t = np.concatenate([m.triangles, m.triangles[:700],  # repeated triangles
                        [[len(m.vertices), len(m.vertices) + 1, len(m.vertices) + 2]]])
    t = t.astype(np.int32)
    n = synth.meshes.area_weighted_normals(v.astype(np.float64), t).astype(np.float32)
    o = np.random.default_rng(9).choice(len(m.vertices), 96, replace=False)
    for R in (0.3, 1.2):
        ref = oracle_mod.rici_fp64(v, n, t, o, R, 32)
        got = gpu_images(rici, v, n, t, o, R, 32)
        assert np.array_equal(got, ref), R


def test_batch_scene_boundaries_inside_chunks_and_groups(rici, oracle_mod):
    """Scenes of 1,000, 37 and 2,100 triangles share 32-record chunks and 1,024-record groups at
    their boundaries; each origin must see only its own scene's triangles."""
    import torch

    rng = np.random.default_rng(12)
    scenes, want = [], []
    for nt in (1000, 37, 2100):
        nv = max(3, nt // 2)
        v = rng.uniform(-0.5, 0.5, size=(nv, 3)).astype(np.float32)
        t = rng.integers(0, nv, size=(nt, 3)).astype(np.int32)
        nrm = rng.normal(size=(nv, 3)).astype(np.float32)
        o = rng.choice(nv, min(nv, 40), replace=False).astype(np.int32)
        scenes.append({"vertices": dev(v), "normals": dev(nrm), "triangles": dev(t),
                       "origins": dev(o)})
        want.append(oracle_mod.rici_fp64(v, nrm, t, o, 0.3, 32))
    outs = rici.rici_generate_batch(scenes, 0.3, 32)
    torch.cuda.synchronize()
    assert rici.sync_status() == 0
    for out, ref in zip(outs, want):
        assert np.array_equal(out.view(torch.int16).cpu().numpy().view(np.uint16), ref)


def test_empty_inputs(rici):
    import torch

    s = synth.tiny_scene()
    no_tris = np.zeros((0, 3), np.int32)
    got = gpu_images(rici, s.vertices, s.normals, no_tris, np.arange(5), 0.3, 32)
    assert got.shape == (5, 32, 32) and not got.any()
    out = rici.rici_generate(dev(s.vertices), dev(s.normals), dev(s.triangles),
                             torch.zeros(0, dtype=torch.int32, device="cuda"), 0.3, 32)
    assert out.shape == (0, 32, 32)


def test_bad_indices_and_nonfinite_report_status(rici):
    import torch

    s = synth.tiny_scene()
    t = s.triangles.copy()
    t[5, 1] = s.num_vertices + 7
    rici.rici_generate(dev(s.vertices), dev(s.normals), dev(t), dev(np.arange(4), torch.int32), 0.3, 32)
    assert rici.sync_status() & rici.binding.ERR_INDEX_OUT_OF_RANGE
    v = s.vertices.copy()
    v[s.triangles[3, 0], 2] = np.nan
    rici.rici_generate(dev(v), dev(s.normals), dev(s.triangles), dev(np.arange(4), torch.int32), 0.3, 32)
    assert rici.sync_status() & rici.binding.ERR_NONFINITE_INPUT
    bad_o = np.array([0, s.num_vertices], np.int32)
    rici.rici_generate(dev(s.vertices), dev(s.normals), dev(s.triangles), dev(bad_o), 0.3, 32)
    assert rici.sync_status() & rici.binding.ERR_INDEX_OUT_OF_RANGE
    assert rici.sync_status() == 0


def test_clutter_scene_full_size_sampled_origins(rici, oracle_mod):
    """The benchmark's workload and launch: every scene vertex imaged at N=64, R=0.3."""
    import torch

    s = synth.clutter_scene()
    o_all = np.arange(s.num_vertices, dtype=np.int32)
    cnt = torch.zeros(4, dtype=torch.int64, device="cuda")
    out = rici.rici_generate(dev(s.vertices), dev(s.normals), dev(s.triangles), dev(o_all), 0.3, 64,
                             counters=cnt)
    assert rici.sync_status() == 0
    rng = np.random.default_rng(0)
    sample = np.unique(np.concatenate([[0, s.num_vertices - 1, s.target_vertices - 1,
                                        s.target_vertices], rng.integers(0, s.num_vertices, 200)]))
    ref = oracle_mod.rici_fp64(s.vertices, s.normals, s.triangles, sample, 0.3, 64)
    pick = lambda imgs, idx: imgs.view(torch.int16)[torch.from_numpy(idx).cuda()].view(torch.uint16)  # noqa: E731
    got = pick(out, sample).cpu().numpy()
    assert np.array_equal(got, ref)
    # needles: the target alone, same vertex indices
    tgt = s.target_only()
    nd = rici.rici_generate(dev(tgt.vertices), dev(tgt.normals), dev(tgt.triangles),
                            dev(np.arange(s.target_vertices, dtype=np.int32)), 0.3, 64)
    assert rici.sync_status() == 0
    ts = sample[sample < s.target_vertices]
    ref_t = oracle_mod.rici_fp64(tgt.vertices, tgt.normals, tgt.triangles, ts, 0.3, 64)
    assert np.array_equal(pick(nd, ts).cpu().numpy(), ref_t)
    c = cnt.cpu().numpy()
    assert c[1] > 0 and c[2] < c[1] * 0.02, f"FP64 band fraction too high: {c}"


@pytest.mark.parametrize("N", [64, 128])
def test_unaligned_output_buffer(rici, oracle_mod, N):
    """Output rows start 2 bytes off an 8-byte boundary: the scalar store path, same images."""
    import torch

    s = synth.tiny_scene()
    o = np.arange(0, s.num_vertices, 5, dtype=np.int32)
    base = torch.zeros(len(o) * N * N + 1, dtype=torch.int16, device="cuda")
    out = base[1:].view(len(o), N, N).view(torch.uint16)
    assert out.data_ptr() % 8 == 2
    rici.rici_generate(dev(s.vertices), dev(s.normals), dev(s.triangles), dev(o), 0.3, N, out=out)
    assert rici.sync_status() == 0
    got = out.view(torch.int16).cpu().numpy().view(np.uint16)
    want = oracle_mod.rici_fp64(s.vertices, s.normals, s.triangles, o, 0.3, N)
    assert np.array_equal(got, want)
    assert base[0].item() == 0  # nothing written before the buffer
