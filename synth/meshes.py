"""Seeded synthetic triangle meshes that stand in for the paper's object collection.

The paper's clutterbox experiment (Section 4.1) draws whole objects from a large mesh
collection, fits each into the unit sphere, and drops them at random orientations and
positions into a box.  That collection is not available here, so closed synthetic meshes of
the same role are generated instead: noise-displaced icospheres and tori.

Nothing in this module computes any part of the RICI method (no frames, projections,
slicing, counting or distances).  It only produces inputs: FP32 vertex positions, FP32
per-vertex normals and int32 triangle indices.  All randomness comes from a caller-supplied
``numpy.random.Generator`` so every mesh is reproducible from one seed.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


@dataclass
class Mesh:
    """A triangle mesh with per-vertex normals.

    vertices:  float64 [V, 3] (kept in float64 until the final FP32 rounding)
    triangles: int64 [T, 3] vertex indices
    """

    vertices: np.ndarray
    triangles: np.ndarray

    @property
    def num_vertices(self) -> int:
        return int(self.vertices.shape[0])

    @property
    def num_triangles(self) -> int:
        return int(self.triangles.shape[0])


# The 12 vertices and 20 faces of a regular icosahedron (golden-ratio construction).
_PHI = (1.0 + math.sqrt(5.0)) / 2.0
_ICO_V = np.array(
    [
        (-1, _PHI, 0), (1, _PHI, 0), (-1, -_PHI, 0), (1, -_PHI, 0),
        (0, -1, _PHI), (0, 1, _PHI), (0, -1, -_PHI), (0, 1, -_PHI),
        (_PHI, 0, -1), (_PHI, 0, 1), (-_PHI, 0, -1), (-_PHI, 0, 1),
    ],
    dtype=np.float64,
)
_ICO_F = np.array(
    [
        (0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11),
        (1, 5, 9), (5, 11, 4), (11, 10, 2), (10, 7, 6), (7, 1, 8),
        (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9),
        (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1),
    ],
    dtype=np.int64,
)


def icosphere(subdivisions: int) -> Mesh:
    """Unit icosphere: 10*4^k + 2 vertices, 20*4^k triangles, outward winding."""
    v = _ICO_V / np.linalg.norm(_ICO_V, axis=1, keepdims=True)
    f = _ICO_F.copy()
    for _ in range(subdivisions):
        nv = v.shape[0]
        e = np.concatenate([f[:, [0, 1]], f[:, [1, 2]], f[:, [2, 0]]], axis=0)
        e.sort(axis=1)
        uniq, inv = np.unique(e, axis=0, return_inverse=True)
        inv = inv.reshape(-1)
        mid = 0.5 * (v[uniq[:, 0]] + v[uniq[:, 1]])
        mid /= np.linalg.norm(mid, axis=1, keepdims=True)
        v = np.concatenate([v, mid], axis=0)
        nf = f.shape[0]
        ab = nv + inv[:nf]
        bc = nv + inv[nf:2 * nf]
        ca = nv + inv[2 * nf:]
        a, b, c = f[:, 0], f[:, 1], f[:, 2]
        f = np.concatenate(
            [
                np.stack([a, ab, ca], 1),
                np.stack([b, bc, ab], 1),
                np.stack([c, ca, bc], 1),
                np.stack([ab, bc, ca], 1),
            ],
            axis=0,
        )
    # make every face wind outward (normal points away from the centre)
    fn = np.cross(v[f[:, 1]] - v[f[:, 0]], v[f[:, 2]] - v[f[:, 0]])
    flip = np.einsum("ij,ij->i", fn, v[f].mean(axis=1)) < 0
    f[flip] = f[flip][:, [0, 2, 1]]
    return Mesh(v, f)


def torus(n_major: int, n_minor: int, minor_radius: float, major_radius: float = 1.0) -> Mesh:
    """Closed torus around the z axis: n_major*n_minor vertices, 2*n_major*n_minor triangles."""
    u = 2.0 * math.pi * np.arange(n_major) / n_major
    w = 2.0 * math.pi * np.arange(n_minor) / n_minor
    uu, ww = np.meshgrid(u, w, indexing="ij")
    ring = major_radius + minor_radius * np.cos(ww)
    v = np.stack([ring * np.cos(uu), ring * np.sin(uu), minor_radius * np.sin(ww)], -1).reshape(-1, 3)
    i = np.arange(n_major)[:, None]
    j = np.arange(n_minor)[None, :]
    p00 = (i * n_minor + j)
    p10 = (((i + 1) % n_major) * n_minor + j)
    p01 = (i * n_minor + (j + 1) % n_minor)
    p11 = (((i + 1) % n_major) * n_minor + (j + 1) % n_minor)
    t1 = np.stack([p00, p10, p11], -1).reshape(-1, 3)
    t2 = np.stack([p00, p11, p01], -1).reshape(-1, 3)
    f = np.concatenate([t1, t2], 0).astype(np.int64)
    return Mesh(v, f)


def displace_radially(mesh: Mesh, rng: np.random.Generator, amplitude: float = 0.1) -> Mesh:
    """Scale every vertex's distance from the mesh centroid by 1 + U(-amplitude, amplitude)."""
    c = mesh.vertices.mean(axis=0)
    s = 1.0 + rng.uniform(-amplitude, amplitude, size=(mesh.num_vertices, 1))
    return Mesh(c + (mesh.vertices - c) * s, mesh.triangles.copy())


def fit_unit_sphere(mesh: Mesh) -> Mesh:
    """Translate the AABB centre to the origin and scale so the farthest vertex is at distance 1."""
    lo = mesh.vertices.min(axis=0)
    hi = mesh.vertices.max(axis=0)
    c = 0.5 * (lo + hi)
    v = mesh.vertices - c
    r = float(np.sqrt((v * v).sum(axis=1)).max())
    return Mesh(v / r, mesh.triangles.copy())


def random_rotation(rng: np.random.Generator) -> np.ndarray:
    """Uniform random rotation matrix from a unit quaternion (Shoemake's method)."""
    u1, u2, u3 = rng.random(3)
    a = math.sqrt(1.0 - u1)
    b = math.sqrt(u1)
    qx, qy, qz, qw = a * math.sin(2 * math.pi * u2), a * math.cos(2 * math.pi * u2), \
        b * math.sin(2 * math.pi * u3), b * math.cos(2 * math.pi * u3)
    return np.array(
        [
            [1 - 2 * (qy * qy + qz * qz), 2 * (qx * qy - qz * qw), 2 * (qx * qz + qy * qw)],
            [2 * (qx * qy + qz * qw), 1 - 2 * (qx * qx + qz * qz), 2 * (qy * qz - qx * qw)],
            [2 * (qx * qz - qy * qw), 2 * (qy * qz + qx * qw), 1 - 2 * (qx * qx + qy * qy)],
        ]
    )


def transform(mesh: Mesh, rotation: np.ndarray, translation) -> Mesh:
    v = mesh.vertices @ rotation.T + np.asarray(translation, dtype=np.float64)[None, :]
    return Mesh(v, mesh.triangles.copy())


def area_weighted_normals(vertices: np.ndarray, triangles: np.ndarray) -> np.ndarray:
    """Per-vertex normals: sum of incident face cross products (area weighted), normalised, FP64."""
    v = np.asarray(vertices, dtype=np.float64)
    t = np.asarray(triangles, dtype=np.int64)
    fn = np.cross(v[t[:, 1]] - v[t[:, 0]], v[t[:, 2]] - v[t[:, 0]])
    n = np.zeros_like(v)
    for k in range(3):
        np.add.at(n, t[:, k], fn)
    ln = np.sqrt((n * n).sum(axis=1, keepdims=True))
    ln[ln == 0] = 1.0
    return n / ln


def displaced_icosphere(rng: np.random.Generator, subdivisions: int, amplitude: float = 0.1) -> Mesh:
    return fit_unit_sphere(displace_radially(icosphere(subdivisions), rng, amplitude))


def displaced_torus(rng: np.random.Generator, target_triangles: int, amplitude: float = 0.1) -> Mesh:
    minor = float(rng.uniform(0.2, 0.5))
    quads = max(12, int(round(target_triangles / 2)))
    # aspect of the parameter grid follows the ratio of the two circumferences
    n_major = max(6, int(round(math.sqrt(quads / minor))))
    n_minor = max(3, int(round(quads / n_major)))
    return fit_unit_sphere(displace_radially(torus(n_major, n_minor, minor), rng, amplitude))
