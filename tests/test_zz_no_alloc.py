"""rici_generate_noalloc, the generation entry point for callers that must not allocate.

Callers such as a service with a device-memory budget fixed at start-up, a plugin host that
owns the GPU allocator, or a latency-critical loop that cannot afford cudaFree's implicit
device-wide synchronisation need a generation call that never allocates.  This test calls
that entry point directly through the C ABI, twice in a row on different meshes (the second
call must not see anything the first left in the shared scratch array), and requires images
identical to those of rici_generate, the allocating entry point, and, on sampled origins, to
the FP64 oracle.  It also calls it once at its largest accepted mesh (262,144 triangles) and
checks that a larger one is rejected with an error text.  It runs last so that a failure here
does not hide failures elsewhere, and it passes alone in a fresh process too.
"""
import ctypes

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


def _dev(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _noalloc(rici, v, n, t, o, R, N):
    import torch

    lib = rici.load_library()
    out = torch.empty((len(o), N, N), dtype=torch.uint16, device="cuda")
    vd, nd, td, od = _dev(v), _dev(n), _dev(t.astype(np.int32)), _dev(np.asarray(o, np.int32))
    ptr = lambda x: ctypes.c_void_p(x.data_ptr())  # noqa: E731
    rc = lib.rici_generate_noalloc(ptr(vd), ptr(nd), vd.shape[0], ptr(td), td.shape[0], ptr(od),
                                   od.numel(), R, N, ptr(out),
                                   ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0
    assert rici.sync_status() == 0
    return out.cpu().numpy()


def _reference(rici, v, n, t, o, R, N):
    out = rici.rici_generate(_dev(v), _dev(n), _dev(t.astype(np.int32)),
                             _dev(np.asarray(o, np.int32)), R, N)
    assert rici.sync_status() == 0
    return out.cpu().numpy()


def test_noalloc_matches_rici_generate_twice(rici, oracle_mod):
    big = synth.clutter_scene()
    o_big = np.arange(0, big.num_vertices, 97)
    small = synth.tiny_scene(3)
    o_small = np.arange(small.num_vertices)
    # first call: the 230k-triangle clutter scene, second call: a 320-triangle mesh
    got1 = _noalloc(rici, big.vertices, big.normals, big.triangles, o_big, 0.3, 64)
    got2 = _noalloc(rici, small.vertices, small.normals, small.triangles, o_small, 0.3, 32)
    ref1 = _reference(rici, big.vertices, big.normals, big.triangles, o_big, 0.3, 64)
    ref2 = _reference(rici, small.vertices, small.normals, small.triangles, o_small, 0.3, 32)
    assert np.array_equal(got1, ref1)
    assert np.array_equal(got2, ref2)
    assert got1.any() and got2.any()
    # and the FP64 definition itself on sampled origins of both meshes
    pick = np.array([0, 7, len(o_big) - 1])
    assert np.array_equal(got1[pick], oracle_mod.rici_fp64(big.vertices, big.normals,
                                                           big.triangles, o_big[pick], 0.3, 64))
    assert np.array_equal(got2, oracle_mod.rici_fp64(small.vertices, small.normals,
                                                     small.triangles, o_small, 0.3, 32))


def test_noalloc_at_its_largest_mesh(rici, oracle_mod):
    # exactly 262,144 triangles: the clutter scene's 229,756 plus a repeat of its first 32,388
    big = synth.clutter_scene()
    limit = 262144
    t = np.concatenate([big.triangles, big.triangles[: limit - big.num_triangles]])
    assert t.shape[0] == limit
    o = np.arange(0, big.num_vertices, 1013)
    got = _noalloc(rici, big.vertices, big.normals, t, o, 0.3, 64)
    assert np.array_equal(got, _reference(rici, big.vertices, big.normals, t, o, 0.3, 64))
    pick = np.array([0, len(o) // 2, len(o) - 1])
    assert np.array_equal(got[pick], oracle_mod.rici_fp64(big.vertices, big.normals, t, o[pick],
                                                          0.3, 64))
    assert got.any()


def test_noalloc_rejects_meshes_beyond_its_scratch(rici):
    lib = rici.load_library()
    d = ctypes.c_void_p(16)
    assert lib.rici_generate_noalloc(d, d, 3, d, 262145, d, 1, 0.3, 64, d, None) == \
        rici.binding.ERR_OUT_TOO_LARGE
    assert b"262144" in lib.rici_last_error_string()
    # the argument checks of rici_generate apply, with their error text
    assert lib.rici_generate_noalloc(d, d, 3, d, 1, d, 1, float("inf"), 64, d, None) == \
        rici.binding.ERR_INVALID_ARGUMENT
    assert b"support_radius" in lib.rici_last_error_string()
