"""The GPU's FP32 projection stage against the oracle's FP32 same-order mode, bit for bit, and a
near tie that single precision alone decides wrongly but the GPU decides like the FP64 definition.
"""
import numpy as np
import pytest

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


NORMALS = [(0, 0, 1), (0, 0, -1), (1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 0), (3, 4, 12),
           (1e-30, 0, 1), (0.3, -0.7, 0.1)]


@pytest.mark.parametrize("normal", NORMALS)
def test_projection_bit_exact(rici, oracle_mod, normal):
    import torch

    rng = np.random.default_rng(abs(hash(normal)) % 1000)
    s = rng.uniform(-1, 1, 3).astype(np.float32)
    n = np.array(normal, np.float32)
    pts = (s + rng.uniform(-0.6, 0.6, (4096, 3))).astype(np.float32)
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    got = rici.binding.project_fp32(d(pts), d(s), d(n)).cpu().numpy()
    want = oracle_mod.project_fp32(pts, s, n)
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))


def test_near_tie_follows_fp64(rici, oracle_mod):
    import torch

    from synth import fixtures as F

    v, n, t, c = F.radius_tie_scene()
    o = np.array([0], np.int32)
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    img = rici.rici_generate(d(v), d(n), d(t), d(o), 0.3, 64)
    assert rici.sync_status() == 0
    got = img.view(torch.int16).cpu().numpy().view(np.uint16)
    want = oracle_mod.rici_fp64(v, n, t, o, 0.3, 64)
    fp32, _ = oracle_mod.rici_fp32(v, n, t, o, 0.3, 64)
    assert np.array_equal(got, want)
    assert not np.array_equal(got, fp32)
