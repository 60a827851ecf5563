"""GPU spin images (Section 2.1) against the oracle.

Both sides form every sample position, projection and bilinear weight in FP32 with the same
explicit roundings (the projection is the generation kernel's FP32 stage, bit-exact against the
oracle's FP32 mode) and sum the weights exactly as integers in units of 2^-24, so the images
agree bit for bit whatever order the samples are added in.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

R = float(np.float32(0.3))


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


def gpu_spin(rici, s, o, N, m):
    out = rici.spin_images(dev(s.vertices), dev(s.normals), dev(s.triangles),
                           dev(np.asarray(o, np.int32)), R, N, m)
    assert rici.sync_status() == 0
    return out.cpu().numpy()


def bit_exact(got, ref):
    assert np.array_equal(got.view(np.uint32), ref.view(np.uint32)), np.abs(got - ref).max()


@pytest.mark.parametrize("N,m", [(32, 3), (8, 1), (16, 5), (64, 2), (128, 3)])
def test_tiny_scene_all_vertices(rici, oracle_mod, N, m):
    s = synth.tiny_scene()
    o = np.arange(s.num_vertices, dtype=np.int32)
    got = gpu_spin(rici, s, o, N, m)
    ref = oracle_mod.spin_images(s.vertices, s.normals, s.triangles, o, R, N, m)
    assert ref.sum() > 0
    bit_exact(got, ref)


def test_clutter_scene_sampled_origins(rici, oracle_mod):
    s = synth.scenes.clutter_scene(seed=6, target_subdivisions=4, n_clutter=5, tri_lo=1000,
                                   tri_hi=20000)
    rng = np.random.default_rng(2)
    o = np.unique(np.r_[0, s.num_vertices - 1, rng.integers(0, s.num_vertices, 40)]).astype(np.int32)
    got = gpu_spin(rici, s, o, 64, 3)
    ref = oracle_mod.spin_images(s.vertices, s.normals, s.triangles, o, R, 64, 3)
    bit_exact(got, ref)


def test_invalid_origin_gives_a_zero_image_and_status(rici):
    s = synth.tiny_scene()
    out = rici.spin_images(dev(s.vertices), dev(s.normals), dev(s.triangles),
                           dev(np.array([0, s.num_vertices], np.int32)), R, 16, 2)
    assert rici.sync_status() & rici.binding.ERR_INDEX_OUT_OF_RANGE
    assert out[1].abs().sum().item() == 0.0 and out[0].sum().item() > 0
