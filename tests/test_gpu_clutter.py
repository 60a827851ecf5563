"""GPU clutter measure (Eq. clutter, Section 4.1) against the oracle and closed forms.

Both sides evaluate the same closed form in FP64 (slab clip, then the disk area of the
projection over the cosine of the plane's tilt) with different operation orders.  Rounding moves
clipped vertices by a few ulps of R, and a triangle that only touches the volume along a boundary
(a vertex on the slab plane or on the cylinder) may then add a sliver of ~1e-15..1e-11 on one
side only, so both areas of an oriented point are compared to 1e-9 of that point's total area
(clutter fractions then agree to 1e-9).
"""
import math

import numpy as np
import pytest

import synth
from synth import fixtures as F

pytestmark = pytest.mark.gpu

R = float(np.float32(0.3))
RTOL = 1e-9


def close(got, ref, total):
    assert np.all(np.abs(got - ref) <= RTOL * total + 1e-15), np.max(np.abs(got - ref) / total)


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


def gpu_areas(rici, v, n, t, o, object_vertices):
    a, b = rici.clutter_areas(dev(v), dev(n), dev(t), dev(np.asarray(o, np.int32)), R,
                              object_vertices)
    assert rici.sync_status() == 0
    return a.cpu().numpy(), b.cpu().numpy()


def plane(fn, nu=41, nv=29):
    p, t = F.grid_surface(lambda u, v: fn((2 * u - 1) + 0.0137, (2 * v - 1) - 0.0071), nu, nv)
    return F._with_origin(p, t)


def test_closed_forms(rici):
    cases = [
        (plane(lambda a, b: np.stack([a, b, np.full_like(a, 0.0625)], -1)), math.pi * R * R),
        (F.vertical_plane(0.125, half_width=1.0, half_height=0.4),
         2.0 * math.sqrt(R * R - 0.125 ** 2) * R),
        (plane(lambda a, b: np.stack([a, b, np.full_like(a, 0.1875)], -1)), 0.0),
        (F.vertical_plane(0.3125), 0.0),
    ]
    for (v, n, t, o), want in cases:
        a, b = gpu_areas(rici, v, n, t, [o], v.shape[0])
        assert a[0] == pytest.approx(want, rel=1e-12, abs=1e-15)
        assert b[0] == a[0]


@pytest.mark.parametrize("object_share", [0, 1, 2])
def test_small_clutter_scene_against_the_oracle(rici, oracle_mod, object_share):
    s = synth.scenes.clutter_scene(seed=6, target_subdivisions=3, n_clutter=4, tri_lo=300,
                                   tri_hi=4000)
    obj = [0, s.target_vertices, s.num_vertices][object_share]
    o = np.arange(0, s.num_vertices, 7, dtype=np.int32)
    ga, gb = gpu_areas(rici, s.vertices, s.normals, s.triangles, o, obj)
    ra, rb = oracle_mod.clutter_areas(s.vertices, s.normals, s.triangles, o, R, obj)
    assert (ra > 0).all()
    close(ga, ra, ra)
    close(gb, rb, ra)


def test_benchmark_scene_sampled_origins(rici, oracle_mod):
    """The benchmark's clutter scene (about 230k triangles): clutter of every target vertex,
    sampled origins checked against the oracle."""
    s = synth.clutter_scene(seed=2)
    o = np.arange(s.target_vertices, dtype=np.int32)
    ga, gb = gpu_areas(rici, s.vertices, s.normals, s.triangles, o, s.target_vertices)
    rng = np.random.default_rng(3)
    pick = np.unique(np.r_[0, s.target_vertices - 1, rng.integers(0, s.target_vertices, 22)])
    ra, rb = oracle_mod.clutter_areas(s.vertices, s.normals, s.triangles, o[pick], R,
                                      s.target_vertices)
    close(ga[pick], ra, ra)
    close(gb[pick], rb, ra)
    assert (gb <= ga * (1 + 1e-12)).all() and (ga > 0).all()


def test_zero_normal_and_no_triangles(rici, oracle_mod):
    v, n, t, o = plane(lambda a, b: np.stack([a, b, np.full_like(a, -0.05)], -1))
    n = n.copy()
    n[o] = 0.0  # identity rotations: the same frame as normal +z
    a, _ = gpu_areas(rici, v, n, t, [o], 0)
    assert a[0] == pytest.approx(math.pi * R * R, rel=1e-12)
    a, b = gpu_areas(rici, v, n, t[:0], [o, 0], 0)
    assert (a == 0).all() and (b == 0).all()


def test_invalid_origin_sets_status(rici):
    import torch

    v, n, t, o = F.vertical_plane(0.125)
    a, b = rici.clutter_areas(dev(v), dev(n), dev(t), dev(np.array([o, v.shape[0]], np.int32)), R,
                              0)
    assert rici.sync_status() & rici.binding.ERR_INDEX_OUT_OF_RANGE
    assert torch.isnan(a[1]).item() and torch.isnan(b[1]).item()
    assert a[0].item() == pytest.approx(2.0 * math.sqrt(R * R - 0.125 ** 2) * R, rel=1e-12)
