"""GPU parity of CRSS search against the int64 CPU oracle: exact ranks, distances, top-1.

Covers RICI-like synthetic image sets (narrow deltas, heavy tails, 16-bit extremes), planted
ties, every resolution class (the packed-int8 CUDA-core kernel for N in {8,16,32,64,128}
and the generic int64 path otherwise), both search modes, images generated by the GPU from
the tiny scene, invalid true-match indices, and the benchmark's full-size search
(10,242 needles x 114,892 haystack images) on sampled needles.
"""
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


def dev(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def run(rici, needles, hay, match=None, mode=0, dist=False):
    r = rici.crss_search(dev(needles), dev(hay), None if match is None else dev(match.astype(np.int64)),
                         mode=mode, return_distances=dist)
    assert rici.sync_status() == 0
    return {k: v.cpu().numpy() for k, v in r.items()}


def check(got, ref, dist=False):
    assert np.array_equal(got["true_distance"], ref["true_distance"])
    assert np.array_equal(got["rank"], ref["rank"])
    assert np.array_equal(got["top1"], ref["top1"])
    if dist:
        assert np.array_equal(got["distances"], ref["distances"])


def dataset(seed, Q, H, N, **kw):
    rng = np.random.default_rng(seed)
    return synth.images.needle_haystack_set(rng, Q, H, N, **kw)


@pytest.mark.parametrize("mode", [0, 1, 2, 3, 4, 5, 6])
def test_small_set_all_outputs(rici, oracle_mod, mode):
    nd, hay, m = dataset(1, 64, 700, 64)
    ref = oracle_mod.crss_search(nd, hay, m, return_distances=True)
    got = run(rici, nd, hay, m, mode=mode, dist=True)
    check(got, ref, dist=True)


@pytest.mark.parametrize("N", [8, 16, 32, 128, 12, 2])
@pytest.mark.parametrize("mode", [1, 3, 4, 5, 6])
def test_resolutions(rici, oracle_mod, N, mode):
    nd, hay, m = dataset(2, 40, 300, N)
    ref = oracle_mod.crss_search(nd, hay, m)
    check(run(rici, nd, hay, m, mode=mode), ref)


@pytest.mark.parametrize("mode", [1, 3, 4, 5, 6])
def test_heavy_tails_and_extremes(rici, oracle_mod, mode):
    rng = np.random.default_rng(3)
    nd, hay, m = synth.images.needle_haystack_set(rng, 60, 900, 64, tail_image_fraction=0.3,
                                                  tail_row_fraction=0.2)
    # 16-bit extremes in a few needles and haystack images (wide on both sides)
    nd[5, 10, 20:] = 65535
    nd[6, :, ::2] = 0
    nd[6, :, 1::2] = 65535
    hay[m[7], 3, :31] = 65535
    hay[17, :, 1::2] = 65535
    hay[18] = 0
    ref = oracle_mod.crss_search(nd, hay, m, return_distances=True)
    got = run(rici, nd, hay, m, mode=mode, dist=True)
    check(got, ref, dist=True)


def test_tensor_accumulator_exact_at_the_narrow_limit(rici, oracle_mod):
    """Largest sums the fp16 operands allow: every delta +-32 (|S| up to 4032 * 3072)."""
    N = 64
    col = np.arange(N)
    up = np.tile((32 * col).astype(np.uint16), (N, 1))          # deltas +32 everywhere
    down = np.tile((32 * (N - 1 - col)).astype(np.uint16), (N, 1))  # deltas -32 everywhere
    zig = np.tile(np.where(col % 2 == 0, 0, 32).astype(np.uint16), (N, 1))  # +32/-32 alternating
    rng = np.random.default_rng(12)
    rnd = np.cumsum(rng.choice([-32, 32], size=(6, N, N)), axis=2)
    rnd = (rnd - rnd.min(axis=2, keepdims=True)).astype(np.uint16)
    ims = np.concatenate([np.stack([up, down, zig, np.zeros((N, N), np.uint16)]), rnd])
    nd = ims.copy()
    hay = np.concatenate([ims[::-1], ims])
    m = np.arange(len(nd)) + len(ims)
    ref = oracle_mod.crss_search(nd, hay, m, return_distances=True)
    assert ref["distances"].max() == 64 * 63 * 64 ** 2  # +32 against -32 at every position
    check(run(rici, nd, hay, m, mode=3, dist=True), ref, dist=True)


def test_tensor_class_exact_at_its_partial_sum_bound(rici, oracle_mod):
    """The fp16 class's bound: a haystack image with n deltas of +45 against a needle with
    deltas of -127 at the same positions gives partial sums up to n (45^2 + 2 * 127 * 45), just
    below 2^24 for n = 1,246 (in the class) and above it for n = 1,247 (the dense kernel)."""
    N = 64

    def image(n, step, base):
        img = np.zeros((N, N), np.int64)
        flat = np.zeros(N * (N - 1), np.int64)
        flat[:n] = step
        img[:, 1:] = flat.reshape(N, N - 1)
        return (base + np.cumsum(img, axis=1)).astype(np.uint16)

    h_in, h_out = image(1246, 45, 0), image(1247, 45, 0)
    n_in, n_out = image(1246, -127, 127 * 63), image(1247, -127, 127 * 63)
    rng = np.random.default_rng(14)
    noise = synth.images.rici_like_images(rng, 6, N)
    hay = np.stack([h_in, h_in.copy(), h_out, h_out.copy(), np.zeros((N, N), np.uint16), *noise])
    nd = np.stack([n_in, n_out, n_in, n_out, noise[0]])
    m = np.array([0, 2, 1, 3, 5], np.int64)
    ref = oracle_mod.crss_search(nd, hay, m, return_distances=True)
    assert ref["distances"][0, 0] == 1246 * (127 ** 2 + 45 ** 2 + 2 * 127 * 45)
    check(run(rici, nd, hay, m, mode=3, dist=True), ref, dist=True)


def test_int8_accumulators_exact_at_the_int8_limit(rici, oracle_mod):
    """Largest sums the int8 operands allow: deltas +-127 everywhere (|G1| = 4032 * 127^2,
    the squared-delta limbs at q = 126, r = 1), in every combination of signs."""
    N = 64
    col = np.arange(N)
    up = np.tile((127 * col).astype(np.uint16), (N, 1))           # deltas +127 everywhere
    down = np.tile((127 * (N - 1 - col)).astype(np.uint16), (N, 1))  # deltas -127 everywhere
    zig = np.tile(np.where(col % 2 == 0, 0, 127).astype(np.uint16), (N, 1))  # +127/-127
    rng = np.random.default_rng(13)
    rnd = np.cumsum(rng.choice([-127, 127, -126, 11, -12], size=(6, N, N)), axis=2)
    rnd = (rnd - rnd.min(axis=2, keepdims=True)).astype(np.uint16)
    ims = np.concatenate([np.stack([up, down, zig, np.zeros((N, N), np.uint16)]), rnd])
    nd = ims.copy()
    hay = np.concatenate([ims[::-1], ims])
    m = np.arange(len(nd)) + len(ims)
    ref = oracle_mod.crss_search(nd, hay, m, return_distances=True)
    assert ref["distances"].max() == 64 * 63 * 254 ** 2  # +127 against -127 at every position
    check(run(rici, nd, hay, m, mode=5, dist=True), ref, dist=True)


@pytest.mark.parametrize("mode", [3, 5, 6])
@pytest.mark.parametrize("Q,H", [(1, 1), (65, 129), (129, 257), (300, 1000)])
def test_tensor_ragged_tiles(rici, oracle_mod, Q, H, mode):
    nd, hay, m = dataset(11, Q, H, 64)
    check(run(rici, nd, hay, m, mode=mode), oracle_mod.crss_search(nd, hay, m))


@pytest.mark.parametrize("N", [64, 32, 16])
@pytest.mark.parametrize("mode", [1, 4, 5])
def test_dense_bands_and_ragged_tiles(rici, oracle_mod, N, mode):
    """CUDA-core forms (dense and sparse-needle) over many haystack tiles: bands of several tiles, a ragged last tile whose
    tail ends inside a thread's image groups, and a partial last needle tile; needles sampled
    from the first, middle and last needle tiles are checked against the oracle."""
    Q, H = 3541, 2048 * 10 + 77
    nd, hay, m = dataset(21, Q, H, N)
    m[-1] = H - 1  # a true match in the last, ragged haystack group
    nd[-1] = hay[H - 1]
    rng = np.random.default_rng(22)
    free = np.setdiff1d(np.arange(H), m)
    pick = np.r_[0:4, 1500:1504, Q - 9:Q]

    def stepped(img, rows, h):
        # raise each listed row from its first non-zero delta on: that delta changes by h, so
        # the clutter-resistant distance to img grows by h^2 per row
        out = img.copy()
        for r in rows:
            nz = np.flatnonzero(np.diff(img[r].astype(np.int64))) + 1
            if nz.size:
                out[r, nz[0]:] += h
        return out

    # true matches a little off their needles, and closer copies spread over the haystack
    # (one in the ragged tail), so the ranks are not all zero
    for i, k in enumerate(pick):
        hay[m[k]] = stepped(nd[k], range(3), 2)
        spots = rng.choice(free, size=i % 4, replace=False)
        if k == Q - 1:
            spots = np.r_[spots, H - 2]
        for pos in spots:
            hay[pos] = stepped(nd[k], [5], 1)
    got = run(rici, nd, hay, m, mode=mode)
    ref = oracle_mod.crss_search(nd[pick], hay, m[pick])
    assert ref["rank"].max() >= 3
    for k in ("true_distance", "rank", "top1"):
        assert np.array_equal(got[k][pick], ref[k]), k


@pytest.mark.parametrize("mode", [1, 4, 5, 6])
def test_degenerate_needles(rici, oracle_mod, mode):
    """Needles with no non-zero delta (constant rows: distance 0 to everything), one non-zero
    delta, a non-zero delta only in the last column, and one full row of +-127 deltas."""
    N = 64
    nd, hay, m = dataset(9, 12, 600, N)
    nd[0] = 7                       # constant image: no entries
    nd[1] = 0
    nd[1, 30, 40:] = 3              # a single non-zero delta
    nd[2] = 0
    nd[2, 63, 63] = 5               # only the last column of the last row
    nd[3, 5] = np.where(np.arange(N) % 2 == 0, 0, 127).astype(np.uint16)  # +-127 on a whole row
    hay[m[0]] = 0
    ref = oracle_mod.crss_search(nd, hay, m, return_distances=True)
    check(run(rici, nd, hay, m, mode=mode, dist=True), ref, dist=True)


@pytest.mark.parametrize("mode", [0, 1, 4, 5, 6])
def test_ties_keep_best_rank(rici, oracle_mod, mode):
    nd, hay, m = dataset(4, 50, 500, 32)
    for k in range(0, 50, 3):  # duplicates of true matches elsewhere in the haystack
        hay[(m[k] + 17) % 500] = hay[m[k]]
    ref = oracle_mod.crss_search(nd, hay, m)
    check(run(rici, nd, hay, m, mode=mode), ref)


def test_identity_match_default(rici, oracle_mod):
    rng = np.random.default_rng(5)
    ims = synth.images.rici_like_images(rng, 120, 64)
    ref = oracle_mod.crss_search(ims, ims)
    got = run(rici, ims, ims)
    check(got, ref)
    assert (got["rank"] == 0).all()


def test_gpu_generated_tiny_scene_self_search(rici, oracle_mod):
    import torch

    s = synth.tiny_scene()
    o = np.arange(s.num_vertices, dtype=np.int32)
    ims = rici.rici_generate(dev(s.vertices), dev(s.normals), dev(s.triangles), dev(o), 0.3, 32)
    r = rici.crss_search(ims, ims)
    assert rici.sync_status() == 0
    assert (r["rank"].cpu().numpy() == 0).all()
    ref_imgs = oracle_mod.rici_fp64(s.vertices, s.normals, s.triangles, o, 0.3, 32)
    ref = oracle_mod.crss_search(ref_imgs, ref_imgs)
    check({k: v.cpu().numpy() for k, v in r.items()}, ref)
    del torch


def test_invalid_true_match_sets_status(rici):
    import torch

    nd, hay, m = dataset(6, 10, 50, 16)
    m[3] = 50
    r = rici.crss_search(dev(nd), dev(hay), dev(m.astype(np.int64)))
    assert rici.sync_status() & rici.binding.ERR_INDEX_OUT_OF_RANGE
    assert r["rank"][3].item() == -1
    del torch


def test_single_haystack_and_single_needle(rici, oracle_mod):
    nd, hay, m = dataset(7, 1, 1, 64)
    check(run(rici, nd, hay, m), oracle_mod.crss_search(nd, hay, m))
    nd, hay, m = dataset(8, 1, 257, 64)  # ragged haystack tile
    check(run(rici, nd, hay, m), oracle_mod.crss_search(nd, hay, m))


@pytest.mark.parametrize("mode", [1, 3, 4, 5, 6])
def test_clutter_scale_search_sampled_needles(rici, oracle_mod, mode):
    """Full benchmark size: 10,242 needles x 114,892 haystack images, N = 64."""
    Q, H = 10242, 114892
    nd, hay, m = dataset(9, Q, H, 64, clutter_fraction=0.3)
    got = run(rici, nd, hay, m, mode=mode)
    rng = np.random.default_rng(1)
    s = np.unique(np.concatenate([[0, Q - 1], rng.integers(0, Q, 30)]))
    ref = oracle_mod.crss_search(nd[s], hay, m[s])
    assert np.array_equal(got["true_distance"][s], ref["true_distance"])
    assert np.array_equal(got["rank"][s], ref["rank"])
    assert np.array_equal(got["top1"][s], ref["top1"])


def test_auto_form_with_mixed_needles(rici, oracle_mod):
    """RICI_SEARCH_AUTO on needles of both kinds: sparse needles (about 3 changes per row) go to
    the sparse-needle form, dense ones (about 40 per row) to the tensor cores.  The needle order
    puts a first tensor-core tile (128 needles) entirely on the sparse side, so that tile is
    skipped, and mixes the kinds in the other tiles; heavy-tailed haystack plateaus reach the
    dense middle pass and the int64 pass.  Every output equals the oracle's."""
    N, Hn = 64, 3000
    rng = np.random.default_rng(21)
    sparse = synth.images.rici_like_images(rng, 200, N, changes_per_row=3.0)
    dense = synth.images.rici_like_images(rng, 120, N, changes_per_row=40.0, small=6)
    order = np.concatenate([np.arange(130), 200 + np.arange(60), 130 + np.arange(70),
                            200 + np.arange(60, 120)])
    pool = np.concatenate([sparse, dense])
    hay = synth.images.rici_like_images(rng, Hn, N, changes_per_row=10.0)
    match = rng.choice(Hn, len(order), replace=False).astype(np.int64)
    hay[match] = pool[order]
    nd = pool[order].copy()
    synth.images.add_plateaus(rng, hay, 0.05, 0.05)  # tails: some images leave fp16 and int8
    ref = oracle_mod.crss_search(nd, hay, match)
    check(run(rici, nd, hay, match, mode=6), ref)
    check(run(rici, nd, hay, match, mode=3), ref)
