"""Pins of the oracle's clutter measure (Eq. clutter, Section 4.1) against closed forms.

The oriented point of every fixture sits at the world origin with normal +z (the identity frame,
so Tx, Ty, Tz are world x, y, z).  Its support volume is x^2 + y^2 <= R^2, |z| <= R/2.

* plane z = z0 with |z0| < R/2 covering the disk: area pi R^2; above the slab: 0;
* plane x = d parallel to the axis: a rectangle 2 sqrt(R^2 - d^2) wide and R high;
* plane x = d + t z: 2 sqrt(1 + t^2) / t * (F(d + t R/2) - F(d - t R/2)) with
  F(u) = (u sqrt(R^2 - u^2) + R^2 asin(u / R)) / 2, the integral of the chord length;
* a closed mesh wholly inside: its own area; split between object and clutter by vertex index;
* rigid motions of scene and oriented point together leave both areas unchanged;
* random triangles: Monte Carlo over points sampled uniformly on the triangle.
"""
import math

import numpy as np
import pytest

import synth
from synth import fixtures as F
from synth import meshes as M

R = float(np.float32(0.3))  # the oracle takes the support radius as float32


def plane_fixture(fn, half=1.0, nu=41, nv=29):
    p, t = F.grid_surface(lambda u, v: fn((2 * u - 1) * half + 0.0137, (2 * v - 1) * half - 0.0071),
                          nu, nv)
    return F._with_origin(p, t)


def areas(fx, object_vertices=None):
    import oracle

    v, n, t, o = fx
    return oracle.clutter_areas(v, n, t, [o], R, v.shape[0] if object_vertices is None
                                else object_vertices)


def chord_integral(u):
    return 0.5 * (u * math.sqrt(R * R - u * u) + R * R * math.asin(u / R))


@pytest.mark.parametrize("z0", [0.0, 0.0625, -0.1])
def test_horizontal_plane_inside_the_slab_is_the_full_disk(z0):
    fx = plane_fixture(lambda a, b: np.stack([a, b, np.full_like(a, z0)], -1))
    a_all, a_obj = areas(fx)
    assert a_all[0] == pytest.approx(math.pi * R * R, rel=1e-12)
    assert a_obj[0] == a_all[0]


def test_horizontal_plane_above_the_slab_adds_nothing():
    fx = plane_fixture(lambda a, b: np.stack([a, b, np.full_like(a, 0.1875)], -1))
    assert areas(fx)[0][0] == 0.0


@pytest.mark.parametrize("d", [0.0, 0.125, -0.25, 0.296875])
def test_plane_parallel_to_the_axis(d):
    v, n, t, o = F.vertical_plane(d, half_width=1.0, half_height=0.4)
    a_all, _ = areas((v, n, t, o))
    assert a_all[0] == pytest.approx(2.0 * math.sqrt(R * R - d * d) * R, rel=1e-12)


def test_plane_parallel_to_the_axis_outside_the_cylinder():
    assert areas(F.vertical_plane(0.3125))[0][0] == 0.0


@pytest.mark.parametrize("d,t", [(0.1, 0.5), (-0.05, 0.8), (0.0, 0.2), (0.2, -0.4)])
def test_tilted_plane(d, t):
    fx = plane_fixture(lambda a, b: np.stack([d + t * b * 0.4, a, b * 0.4], -1))
    want = 2.0 * math.sqrt(1.0 + t * t) / abs(t) * abs(
        chord_integral(d + t * R / 2) - chord_integral(d - t * R / 2))
    # the fixture's float32 vertices move the plane by ~1e-8
    assert areas(fx)[0][0] == pytest.approx(want, rel=1e-6)


def test_nearly_parallel_plane_agrees_with_the_parallel_rectangle():
    d, t = 0.125, 2e-9
    fx = plane_fixture(lambda a, b: np.stack([d + t * b * 0.4, a, b * 0.4], -1))
    assert areas(fx)[0][0] == pytest.approx(2.0 * math.sqrt(R * R - d * d) * R, rel=1e-6)


def mesh_area(v, t):
    p = v.astype(np.float64)[t]
    return 0.5 * np.linalg.norm(np.cross(p[:, 1] - p[:, 0], p[:, 2] - p[:, 0]), axis=1).sum()


def small_sphere(rng, radius, centre):
    m = M.displaced_icosphere(rng, 3)
    return m.vertices * radius + np.asarray(centre), m.triangles


def test_closed_mesh_inside_counts_whole_and_splits_by_object():
    rng = np.random.default_rng(4)
    sv, st = small_sphere(rng, 0.12, (0.05, -0.02, 0.0))
    # clutter: a horizontal plane through the slab, after the object's vertices
    pv, pt = F.grid_surface(lambda u, v: np.stack([(2 * u - 1) + 0.013, (2 * v - 1) - 0.007,
                                                   np.full_like(u, 0.03)], -1), 31, 27)
    v = np.concatenate([sv, pv.reshape(-1, 3)])
    t = np.concatenate([st, pt + sv.shape[0]])
    fx = F._with_origin(v, t)
    a_all, a_obj = areas(fx, object_vertices=sv.shape[0])
    sphere = mesh_area(fx[0], fx[2][: st.shape[0]])
    assert a_obj[0] == pytest.approx(sphere, rel=1e-12)
    # both surfaces inside the volume count: the sphere whole, the plane as the full disk
    assert a_all[0] == pytest.approx(sphere + math.pi * R * R, rel=1e-12)
    import oracle

    c = oracle.clutter(fx[0], fx[1], fx[2], [fx[3]], R, sv.shape[0])[0]
    assert c == pytest.approx(math.pi * R * R / (sphere + math.pi * R * R), rel=1e-12)


def test_rigid_motion_of_scene_and_oriented_point():
    import oracle

    s = synth.scenes.clutter_scene(seed=3, target_subdivisions=3, n_clutter=3, tri_lo=500,
                                   tri_hi=3000)
    o = np.arange(0, s.num_vertices, 97, dtype=np.int32)
    a0, b0 = oracle.clutter_areas(s.vertices, s.normals, s.triangles, o, R, s.target_vertices)
    rng = np.random.default_rng(8)
    rot = M.random_rotation(rng)
    v1 = (s.vertices.astype(np.float64) @ rot.T + np.array([0.3, -0.2, 0.1])).astype(np.float32)
    n1 = (s.normals.astype(np.float64) @ rot.T).astype(np.float32)
    a1, b1 = oracle.clutter_areas(v1, n1, s.triangles, o, R, s.target_vertices)
    assert (a0 > 0).all()
    np.testing.assert_allclose(a1, a0, rtol=2e-5, atol=1e-9)
    np.testing.assert_allclose(b1, b0, rtol=2e-5, atol=1e-9)
    assert (b0 <= a0 * (1 + 1e-12)).all()


@pytest.mark.parametrize("seed", range(6))
def test_random_triangles_against_monte_carlo(seed):
    import oracle

    rng = np.random.default_rng(100 + seed)
    tri = rng.uniform(-0.45, 0.45, size=(3, 3))
    if seed == 5:
        tri[:, 0] = 0.1 + 0.02 * tri[:, 2]  # steep, nearly parallel to the axis
    fx = F._with_origin(tri, [[0, 1, 2]])
    v = fx[0].astype(np.float64)
    got = oracle.clutter_areas(fx[0], fx[1], fx[2], [fx[3]], R, 3)[0][0]
    # uniform points on the triangle
    n = 400_000
    r1, r2 = rng.random(n), rng.random(n)
    s1 = np.sqrt(r1)
    p = (1 - s1)[:, None] * v[0] + (s1 * (1 - r2))[:, None] * v[1] + (s1 * r2)[:, None] * v[2]
    inside = (p[:, 0] ** 2 + p[:, 1] ** 2 <= R * R) & (np.abs(p[:, 2]) <= R / 2)
    area = 0.5 * np.linalg.norm(np.cross(v[1] - v[0], v[2] - v[0]))
    f = inside.mean()
    sigma = area * math.sqrt(max(f * (1 - f), 1.0 / n) / n)
    assert abs(got - area * f) <= 5 * sigma + 1e-12
