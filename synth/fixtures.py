"""Small geometric inputs with known answers (inputs only).

Every fixture returns FP32 ``vertices``, FP32 ``normals`` and int32 ``triangles`` plus the
index of one extra vertex that serves as the oriented point: the spin vertex at the world
origin with spin normal +z (so the central axis is the z axis and beta = z).  That vertex is
not referenced by any triangle.  The shapes are chosen so the RICI of that oriented point has
a closed form:

* ``vertical_plane``: the plane x = d; every circle of radius alpha > d crosses it twice,
  every circle with alpha < d misses it.
* ``vertical_cylinder``: a cylinder parallel to the axis, centre distance c, radius rho; in
  every layer a circle of radius alpha crosses it twice exactly when |c - rho| < alpha < c + rho.
* ``off_axis_sphere``: the same rule with the slice radius rho(beta) = sqrt(rs^2 - (beta-zc)^2).
"""
from __future__ import annotations

import math

import numpy as np

from . import meshes as M


def _with_origin(v, t, normal=(0.0, 0.0, 1.0), origin=(0.0, 0.0, 0.0)):
    v = np.concatenate([np.asarray(v, np.float64), np.asarray([origin], np.float64)], 0)
    n = np.zeros_like(v)
    n[-1] = normal
    return (np.ascontiguousarray(v.astype(np.float32)), np.ascontiguousarray(n.astype(np.float32)),
            np.ascontiguousarray(np.asarray(t, np.int64).astype(np.int32)), int(v.shape[0] - 1))


def grid_surface(pts_fn, nu: int, nv: int, wrap_u: bool = False):
    """Triangulate a parametric grid: pts_fn(u, v) -> xyz with u in [0,1], v in [0,1]."""
    us = np.arange(nu) / nu if wrap_u else np.linspace(0.0, 1.0, nu + 1)
    vs = np.linspace(0.0, 1.0, nv + 1)
    uu, vv = np.meshgrid(us, vs, indexing="ij")
    p = pts_fn(uu, vv).reshape(-1, 3)
    nuu = us.size
    i = np.arange(nuu if wrap_u else nuu - 1)[:, None]
    j = np.arange(nv)[None, :]
    i1 = (i + 1) % nuu
    p00 = i * (nv + 1) + j
    p10 = i1 * (nv + 1) + j
    p01 = i * (nv + 1) + j + 1
    p11 = i1 * (nv + 1) + j + 1
    t = np.concatenate([np.stack([p00, p10, p11], -1).reshape(-1, 3),
                        np.stack([p00, p11, p01], -1).reshape(-1, 3)], 0)
    return p, t


def vertical_plane(d: float, half_width: float = 1.0, half_height: float = 0.4,
                   nu: int = 37, nv: int = 23):
    """Plane x = d, y in [-hw, hw], z in [-hh, hh], tessellated (nu x nv quads)."""
    def f(u, v):
        return np.stack([np.full_like(u, d), (2 * u - 1) * half_width, (2 * v - 1) * half_height], -1)
    p, t = grid_surface(f, nu, nv)
    return _with_origin(p, t)


def vertical_cylinder(c: float, rho: float, half_height: float = 0.4, n_around: int = 1440,
                      nv: int = 7):
    """Open cylinder around the vertical line (c, 0, z), tessellated as an n_around-gon prism."""
    def f(u, v):
        a = 2 * math.pi * u
        return np.stack([c + rho * np.cos(a), rho * np.sin(a), (2 * v - 1) * half_height], -1)
    p, t = grid_surface(f, n_around, nv, wrap_u=True)
    return _with_origin(p, t)


def polygon_inradius(rho: float, n_around: int) -> float:
    """Distance from the prism axis to the middle of a polygon edge."""
    return rho * math.cos(math.pi / n_around)


def off_axis_sphere(c: float, zc: float, rs: float, subdivisions: int = 6):
    m = M.icosphere(subdivisions)
    v = m.vertices * rs + np.array([c, 0.0, zc])[None, :]
    return _with_origin(v, m.triangles)


def icosphere_deviation(rs: float, subdivisions: int) -> float:
    """Upper bound on how far the tessellated sphere's surface lies inside the true sphere."""
    m = M.icosphere(subdivisions)
    e = m.vertices[m.triangles]
    edge = np.sqrt(((e[:, 1] - e[:, 0]) ** 2).sum(-1)).max()
    # a flat triangle with circumradius <= edge/sqrt(3) sits at most r - sqrt(r^2 - R_c^2) inside
    rc = edge / math.sqrt(3.0)
    return rs * (1.0 - math.sqrt(max(0.0, 1.0 - rc * rc)))


PYTHAGOREAN_NORMALS = [
    (0, 0, 1), (0, 0, -1), (1, 0, 0), (0, 1, 0), (-1, 0, 0), (0, -1, 0),
    (3, 4, 12), (4, -3, 12), (-3, -4, -12), (0, 3, 4), (3, 0, -4), (6, 8, 0),
    (12, 5, 84), (-5, 12, -84),
]
"""Spin normals whose frame coefficients are rational: nx^2+ny^2 and nx^2+ny^2+nz^2 are squares."""


def dyadic_mesh(rng: np.random.Generator, n_tris: int, n_verts: int, scale_bits: int = 5,
                extent: float = 0.25):
    """Random triangles over random vertices whose coordinates are multiples of 2^-scale_bits."""
    q = 2.0 ** scale_bits
    lim = int(extent * q)
    v = rng.integers(-lim, lim + 1, size=(n_verts, 3)).astype(np.float64) / q
    t = np.stack([rng.choice(n_verts, 3, replace=False) for _ in range(n_tris)]).astype(np.int32)
    return v.astype(np.float32), t


def radius_tie_scene(R=0.3, N=64):
    """A triangle with a vertical edge at distance x from the axis, where x^2 lies just below
    alpha_c^2 in exact arithmetic but rounds to the same FP32 value as alpha_c^2: the circle of
    column c misses the edge in FP64 and touches it in FP32 (origin at 0 with normal +z, where
    both precisions project every vertex exactly)."""
    R = float(np.float32(R))  # the support radius is passed as an FP32 value
    for c in range(N):
        a2d = ((R * (2 * c + 1)) / (2 * N)) ** 2
        a2f = np.float32(a2d)
        x = np.float32(np.sqrt(a2d))
        for _ in range(64):
            if float(x) ** 2 < a2d and np.float32(float(x) ** 2) == a2f:
                v = np.array([[0, 0, 0], [x, 0, -0.01], [x, 0, 0.01], [x + 0.05, 0.04, 0.0]],
                             np.float32)
                n = np.tile(np.array([0.0, 0.0, 1.0], np.float32), (4, 1))
                return v, n, np.array([[1, 2, 3]], np.int32), c
            x = np.nextafter(x, np.float32(0))
    raise AssertionError("no near-tie found")
