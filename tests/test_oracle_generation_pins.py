"""Pins for the oracle's RICI generation (CPU only).

Each test ties the FP64 oracle to something outside itself: closed-form geometry, an
exact-rational evaluation, an independent world-frame circle/triangle intersection count,
or an invariance the paper's construction guarantees.  A dropped term, a wrong sign, a
swapped operand or an off-by-one bin in the oracle fails at least one of them.
"""
import math

import numpy as np
import pytest

import synth
from synth import fixtures as F
from tests import _geom

R = 0.3


def bin_alpha(N, R=R):
    return R * (2 * np.arange(N) + 1) / (2 * N)


def bin_beta(N, R=R):
    return R * (2 * np.arange(N) + 1 - N) / (2 * N)


# ---------------------------------------------------------------- projection (Section 3.1.1)

def test_projection_matches_cylindrical_closed_form(oracle_mod):
    rng = np.random.default_rng(11)
    for _ in range(20):
        S = rng.uniform(-1, 1, 3).astype(np.float32)
        n = rng.normal(size=3).astype(np.float32)
        P = rng.uniform(-1, 1, (50, 3)).astype(np.float32)
        T = oracle_mod.project_fp64(P, S, n)
        d = P.astype(np.float64) - S.astype(np.float64)
        nh = n.astype(np.float64) / np.linalg.norm(n.astype(np.float64))
        beta = d @ nh
        alpha2 = (d * d).sum(1) - beta ** 2
        scale = (d * d).sum(1) + 1e-30
        assert np.allclose(T[:, 2], beta, rtol=0, atol=1e-13)
        assert np.allclose(T[:, 0] ** 2 + T[:, 1] ** 2, alpha2, rtol=0, atol=1e-12 * scale.max())


@pytest.mark.parametrize("normal,perm", [
    ((0, 0, 1), lambda d: (d[:, 0], d[:, 1], d[:, 2])),     # identity rule: both pairs
    ((0, 0, -1), lambda d: (-d[:, 0], d[:, 1], -d[:, 2])),
    ((0, 1, 0), lambda d: (-d[:, 2], -d[:, 0], d[:, 1])),    # pins the second normalisation
    ((1, 0, 0), lambda d: (-d[:, 2], d[:, 1], d[:, 0])),
    ((0, 2, 0), lambda d: (-d[:, 2], -d[:, 0], d[:, 1])),    # normal length does not matter
])
def test_projection_axis_aligned_normals_exact(oracle_mod, normal, perm):
    rng = np.random.default_rng(3)
    S = rng.uniform(-1, 1, 3).astype(np.float32)
    P = rng.uniform(-1, 1, (40, 3)).astype(np.float32)
    T = oracle_mod.project_fp64(P, S, np.array(normal, np.float32))
    d = P.astype(np.float64) - S.astype(np.float64)
    ex, ey, ez = perm(d)
    assert np.array_equal(T[:, 0], ex) and np.array_equal(T[:, 1], ey) and np.array_equal(T[:, 2], ez)


def test_zero_normal_uses_identity_rotations(oracle_mod):
    P = np.array([[0.25, -0.5, 0.125]], np.float32)
    T = oracle_mod.project_fp64(P, np.zeros(3, np.float32), np.zeros(3, np.float32))
    assert T.tolist() == [[0.25, -0.5, 0.125]]


# ---------------------------------------------------------------- closed-form images

@pytest.mark.parametrize("d", [0.0731, 0.1513, 0.2777])
def test_vertical_plane_two_crossings_beyond_distance(oracle_mod, d):
    N = 32
    v, n, t, o = F.vertical_plane(d)
    img = oracle_mod.rici_fp64(v, n, t, [o], R, N)[0].astype(np.int64)
    expect = np.where(bin_alpha(N) > d, 2, 0)[None, :].repeat(N, 0)
    assert np.array_equal(img, expect)


@pytest.mark.parametrize("c,rho", [(0.12, 0.05), (0.05, 0.12), (0.2, 0.2)])
def test_vertical_cylinder_annulus_rule(oracle_mod, c, rho):
    N = 32
    n_around = 1440
    v, n, t, o = F.vertical_cylinder(c, rho, n_around=n_around)
    img = oracle_mod.rici_fp64(v, n, t, [o], R, N)[0].astype(np.int64)
    a = bin_alpha(N)
    rin = F.polygon_inradius(rho, n_around)
    lo, hi = abs(c - rho), c + rho
    expect = np.where((a > lo) & (a < hi), 2, 0)
    tol = (rho - rin) + 1e-9
    ok = (np.abs(a - lo) > tol) & (np.abs(a - hi) > tol)
    assert ok.sum() > N // 3
    for r in range(N):
        assert np.array_equal(img[r, ok], expect[ok]), r


def test_off_axis_sphere_annulus_rule(oracle_mod):
    N = 32
    c, zc, rs, k = 0.13, 0.02, 0.09, 6
    v, n, t, o = F.off_axis_sphere(c, zc, rs, subdivisions=k)
    img = oracle_mod.rici_fp64(v, n, t, [o], R, N)[0].astype(np.int64)
    a = bin_alpha(N)
    dev = F.icosphere_deviation(rs, k)
    checked = 0
    for r, b in enumerate(bin_beta(N)):
        h = abs(b - zc)
        if h >= rs - 4 * dev:
            if h > rs + 1e-9:
                assert not img[r].any()
            continue
        rho_out = math.sqrt(rs * rs - h * h)
        # the polygonal slice lies between the true circle and a circle shrunk by the
        # deviation converted to a slice radius change
        rho_in = math.sqrt(max(0.0, (rs - dev) ** 2 - h * h))
        tol = (rho_out - rho_in) + 1e-9
        lo_o, hi_o = abs(c - rho_out), c + rho_out
        expect = np.where((a > lo_o) & (a < hi_o), 2, 0)
        ok = (np.abs(a - lo_o) > tol) & (np.abs(a - hi_o) > tol)
        assert np.array_equal(img[r, ok], expect[ok]), r
        checked += int(ok.sum())
    assert checked > 100


# ---------------------------------------------------------------- exact and independent counts

def _dyadic_case(seed, n_tris=6, n_verts=7):
    rng = np.random.default_rng(seed)
    v, t = F.dyadic_mesh(rng, n_tris, n_verts)
    normals = np.array(F.PYTHAGOREAN_NORMALS, np.float32)
    origins_n = normals[rng.choice(len(normals), 3, replace=False)]
    origins_v = (rng.integers(-8, 9, size=(3, 3)) / 32.0).astype(np.float32)
    V = np.concatenate([v, origins_v]).astype(np.float32)
    Nr = np.concatenate([np.zeros_like(v), origins_n]).astype(np.float32)
    origins = list(range(len(v), len(v) + 3))
    return V, Nr, t, origins


@pytest.mark.parametrize("seed", range(6))
def test_fp64_matches_exact_rational_away_from_ties(oracle_mod, seed):
    from oracle import exact

    N = 8
    V, Nr, t, origins = _dyadic_case(seed)
    ex, margin = exact.rici_exact(V, Nr, t, origins, 0.5, N)
    got = oracle_mod.rici_fp64(V, Nr, t, origins, 0.5, N).astype(np.int64)
    ok = margin > 1e-9
    # dyadic vertices often sit exactly on a layer plane (ties); those bins are excluded
    assert ok.mean() > 0.7
    assert np.array_equal(got[ok], ex[ok])
    assert ex.sum() > 0


@pytest.mark.parametrize("seed", range(4))
def test_matches_world_frame_circle_triangle_count(oracle_mod, seed):
    rng = np.random.default_rng(100 + seed)
    m = synth.meshes.displaced_icosphere(rng, 2)
    V = (m.vertices * 0.2).astype(np.float32)
    t = m.triangles.astype(np.int32)
    S = rng.uniform(-0.05, 0.05, 3)
    nrm = rng.normal(size=3)
    V = np.concatenate([V, S[None, :].astype(np.float32)])
    Nr = np.zeros_like(V)
    Nr[-1] = nrm.astype(np.float32)
    N = 16
    img = oracle_mod.rici_fp64(V, Nr, t, [len(V) - 1], R, N)[0].astype(np.int64)
    ref, mg = _geom.circle_counts(V.astype(np.float64), Nr[-1].astype(np.float64),
                                  V[-1].astype(np.float64), t, R, N)
    ok = mg > 1e-6
    assert ok.mean() > 0.8
    assert np.array_equal(img[ok], ref[ok])
    assert ref.sum() > 50


# ---------------------------------------------------------------- invariances

def test_watertight_meshes_give_even_counts(oracle_mod):
    s = synth.tiny_scene(7)
    img = oracle_mod.rici_fp64(s.vertices, s.normals, s.triangles, np.arange(s.num_vertices), R, 32)
    assert img.sum() > 0 and not (img % 2).any()
    rng = np.random.default_rng(5)
    tor = synth.meshes.displaced_torus(rng, 800)
    V = tor.vertices.astype(np.float32)
    Nn = synth.meshes.area_weighted_normals(tor.vertices, tor.triangles).astype(np.float32)
    img = oracle_mod.rici_fp64(V, Nn, tor.triangles, np.arange(0, len(V), 7), 0.6, 32)
    assert img.sum() > 0 and not (img % 2).any()


def test_triangle_order_and_vertex_rotation_invariance(oracle_mod):
    s = synth.tiny_scene(3)
    o = np.arange(0, s.num_vertices, 5)
    base = oracle_mod.rici_fp64(s.vertices, s.normals, s.triangles, o, R, 32)
    rng = np.random.default_rng(0)
    t = s.triangles[rng.permutation(s.num_triangles)]
    t = np.stack([np.roll(row, int(k)) for row, k in zip(t, rng.integers(0, 3, len(t)))])
    t[::2] = t[::2][:, [0, 2, 1]]  # flip the winding of every other triangle
    other = oracle_mod.rici_fp64(s.vertices, s.normals, t, o, R, 32)
    assert np.array_equal(base, other)


def test_mirror_and_dyadic_translation_invariance(oracle_mod):
    s = synth.tiny_scene(4)
    o = np.arange(0, s.num_vertices, 3)
    base = oracle_mod.rici_fp64(s.vertices, s.normals, s.triangles, o, R, 32)
    mv = s.vertices * np.array([1, -1, 1], np.float32)
    mn = s.normals * np.array([1, -1, 1], np.float32)
    assert np.array_equal(base, oracle_mod.rici_fp64(mv, mn, s.triangles, o, R, 32))
    # on a 2^-16 grid, shifting by 4 keeps every FP32 coordinate (and so every P - S) exact
    qv = (np.round(s.vertices.astype(np.float64) * 65536.0) / 65536.0).astype(np.float32)
    qbase = oracle_mod.rici_fp64(qv, s.normals, s.triangles, o, R, 32)
    tv = (qv.astype(np.float64) + np.array([4.0, -4.0, 4.0])).astype(np.float32)
    assert np.array_equal((tv.astype(np.float64) - qv.astype(np.float64)),
                          np.broadcast_to(np.array([4.0, -4.0, 4.0]), tv.shape))
    assert np.array_equal(qbase, oracle_mod.rici_fp64(tv, s.normals, s.triangles, o, R, 32))


def test_normal_scale_invariance(oracle_mod):
    s = synth.tiny_scene(5)
    o = np.arange(0, s.num_vertices, 4)
    base = oracle_mod.rici_fp64(s.vertices, s.normals, s.triangles, o, R, 32)
    for k in (0.5, 2.0, 8.0):
        other = oracle_mod.rici_fp64(s.vertices, s.normals * np.float32(k), s.triangles, o, R, 32)
        assert np.array_equal(base, other)


def test_counts_saturate_at_uint16_max(oracle_mod):
    v, n, t, o = F.vertical_plane(0.1, nu=1, nv=1)
    reps = 32769  # 2 crossings per copy -> 65538 > 65535
    T = np.tile(t, (reps, 1))
    img = oracle_mod.rici_fp64(v, n, T, [o], R, 8)[0]
    a = bin_alpha(8)
    assert np.all(img[:, a > 0.1] == 65535) and np.all(img[:, a < 0.1] == 0)


def test_support_volume_bounds(oracle_mod):
    """Nothing outside alpha <= R and |beta| <= R/2 is counted; rows follow beta ascending."""
    # a small horizontal-ish triangle crossing only the top layer, far left of the axis
    N = 8
    bt = bin_beta(N)
    z0, z1 = bt[-1] - 0.001, bt[-1] + 0.001
    v = np.array([[0.05, -0.1, z0], [0.05, 0.1, z0], [0.05, 0.0, z1], [0, 0, 0]], np.float32)
    n = np.zeros_like(v)
    n[3] = (0, 0, 1)
    img = oracle_mod.rici_fp64(v, n, [[0, 1, 2]], [3], R, N)[0]
    assert img[:-1].sum() == 0 and img[-1].sum() > 0
    far = v.copy()
    far[:3, 0] = R * 1.01
    assert oracle_mod.rici_fp64(far, n, [[0, 1, 2]], [3], R, N).sum() == 0
    high = v.copy()
    high[:3, 2] += R
    assert oracle_mod.rici_fp64(high, n, [[0, 1, 2]], [3], R, N).sum() == 0
