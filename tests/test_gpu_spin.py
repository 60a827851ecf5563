"""GPU spin images (Section 2.1) against the oracle.

Primary check: the FP64 definition (sample positions, projection and bilinear weights in double,
summed in double).  The kernel works in single precision, so every bin must lie within the
oracle's per-bin bound on a single-precision evaluation: the FP32 rounding of each sample
position, of the projection (10 u (|dx| + |dy| + |dz|) plus the position error), of alpha, u
and v, the rounding of each weight to a multiple of 2^-24, and samples that may fall on either
side of the volume boundary.

Second check: the oracle's single-precision same-operation-order mode forms every quantity with
the kernel's roundings and sums the weights as integers in units of 2^-24, so the two agree bit
for bit whatever order the samples are added in.
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


def within_fp64_bound(oracle_mod, s, o, N, m, got):
    ref, bound = oracle_mod.spin_images(s.vertices, s.normals, s.triangles, o, R, N, m,
                                        return_bound=True)
    dev = np.abs(got.astype(np.float64) - ref.astype(np.float64))
    worst = np.unravel_index(np.argmax(dev - bound), dev.shape)
    assert (dev <= bound).all(), (worst, dev[worst], bound[worst], ref[worst], got[worst])
    assert ref.sum() > 0


@pytest.mark.parametrize("N,m", [(32, 3), (8, 1), (16, 5), (64, 2), (128, 3)])
def test_tiny_scene_all_vertices(rici, oracle_mod, N, m):
    s = synth.tiny_scene()
    o = np.arange(s.num_vertices, dtype=np.int32)
    got = gpu_spin(rici, s, o, N, m)
    within_fp64_bound(oracle_mod, s, o, N, m, got)
    bit_exact(got, oracle_mod.spin_images_fp32(s.vertices, s.normals, s.triangles, o, R, N, m))


def test_clutter_scene_sampled_origins(rici, oracle_mod):
    s = synth.scenes.clutter_scene(seed=6, target_subdivisions=4, n_clutter=5, tri_lo=1000,
                                   tri_hi=20000)
    rng = np.random.default_rng(2)
    o = np.unique(np.r_[0, s.num_vertices - 1, rng.integers(0, s.num_vertices, 40)]).astype(np.int32)
    got = gpu_spin(rici, s, o, 64, 3)
    within_fp64_bound(oracle_mod, s, o, 64, 3, got)
    bit_exact(got, oracle_mod.spin_images_fp32(s.vertices, s.normals, s.triangles, o, R, 64, 3))


def test_invalid_origin_gives_a_zero_image_and_status(rici):
    s = synth.tiny_scene()
    out = rici.spin_images(dev(s.vertices), dev(s.normals), dev(s.triangles),
                           dev(np.array([0, s.num_vertices], np.int32)), R, 16, 2)
    assert rici.sync_status() & rici.binding.ERR_INDEX_OUT_OF_RANGE
    assert out[1].abs().sum().item() == 0.0 and out[0].sum().item() > 0
