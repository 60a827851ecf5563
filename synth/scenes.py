"""Seeded clutter scenes (inputs only).

A scene is the combined mesh of a clutterbox run (Section 4.1): the target object first,
then clutter objects, each fitted to the unit sphere and placed at a uniform random
orientation and a uniform random centre.  Because the target comes first, its vertices keep
the indices 0..V_t-1 in the combined mesh, so the true match of needle i (the target's
vertex i, imaged with the target alone) is haystack image i.

Workload recipes (sizes and distributions follow the paper's clutterbox scenes; the
collection itself is replaced by displaced icospheres and tori):

* ``tiny_scene``    one displaced icosphere, 2 subdivisions (162 vertices, 320 triangles).
* ``clutter_scene`` a subdivision-5 target (20,480 triangles) plus 9 clutter meshes of
  5k-50k triangles (log-uniform), centres uniform in [-1,1]^3 (box side 2).
* ``large_scene``   a subdivision-7 target plus meshes up to ~5M triangles in total (about 40
  meshes), box side 4 with every bounding sphere inside the box (centres in [-1,1]^3).
* ``clutterbox``    the levels of one clutterbox run (Section 4.1): n objects drawn from the
  synthetic collection, each fitted to the unit sphere and placed in a box of side s with its
  bounding sphere inside the box; level k is the combined mesh of the first k objects, the
  reference object first.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import meshes as M


@dataclass
class Scene:
    vertices: np.ndarray          # float32 [V, 3]
    normals: np.ndarray           # float32 [V, 3]
    triangles: np.ndarray         # int32 [T, 3]
    target_vertices: int          # the first target_vertices vertices belong to the target
    target_triangles: int         # the first target_triangles triangles belong to the target
    mesh_vertex_offsets: list = field(default_factory=list)
    mesh_triangle_offsets: list = field(default_factory=list)

    @property
    def num_vertices(self) -> int:
        return int(self.vertices.shape[0])

    @property
    def num_triangles(self) -> int:
        return int(self.triangles.shape[0])

    def target_only(self) -> "Scene":
        """The target mesh alone, with the same vertex arrays (so indices are unchanged)."""
        return Scene(self.vertices, self.normals, self.triangles[: self.target_triangles],
                     self.target_vertices, self.target_triangles, [0], [0])


def assemble(meshes_world) -> Scene:
    """Concatenate placed meshes (float64) into one FP32 scene with per-mesh normals."""
    vs, ns, ts, voff, toff = [], [], [], [], []
    nv = 0
    nt = 0
    for m in meshes_world:
        vs.append(m.vertices)
        ns.append(M.area_weighted_normals(m.vertices, m.triangles))
        ts.append(m.triangles + nv)
        voff.append(nv)
        toff.append(nt)
        nv += m.num_vertices
        nt += m.num_triangles
    v = np.concatenate(vs).astype(np.float32)
    n = np.concatenate(ns).astype(np.float32)
    t = np.concatenate(ts).astype(np.int32)
    return Scene(np.ascontiguousarray(v), np.ascontiguousarray(n), np.ascontiguousarray(t),
                 meshes_world[0].num_vertices, meshes_world[0].num_triangles, voff, toff)


def _place(rng, mesh, half_box: float):
    rot = M.random_rotation(rng)
    centre = rng.uniform(-half_box, half_box, size=3)
    return M.transform(mesh, rot, centre)


def _clutter_mesh(rng, tri_lo: int, tri_hi: int) -> M.Mesh:
    want = math.exp(rng.uniform(math.log(tri_lo), math.log(tri_hi)))
    if rng.random() < 0.5:
        # icosphere with the subdivision level closest (in log scale) to the drawn size
        k = int(np.clip(round(math.log(want / 20.0, 4)), 1, 7))
        return M.displaced_icosphere(rng, k)
    return M.displaced_torus(rng, int(want))


def tiny_scene(seed: int = 1) -> Scene:
    """One noise-displaced icosphere (subdivision 2), fitted to the unit sphere."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return assemble([M.displaced_icosphere(rng, 2)])


def clutter_scene(seed: int = 2, target_subdivisions: int = 5, n_clutter: int = 9,
                  tri_lo: int = 5000, tri_hi: int = 50000, half_box: float = 1.0) -> Scene:
    """Target icosphere plus clutter meshes, centres uniform in [-half_box, half_box]^3."""
    rng = np.random.Generator(np.random.PCG64(seed))
    placed = [_place(rng, M.displaced_icosphere(rng, target_subdivisions), half_box)]
    for _ in range(n_clutter):
        placed.append(_place(rng, _clutter_mesh(rng, tri_lo, tri_hi), half_box))
    return assemble(placed)


def large_scene(seed: int = 5, total_triangles: int = 5_000_000, n_meshes: int = 40,
                half_box: float = 1.0) -> Scene:
    """~total_triangles over about n_meshes meshes: a subdivision-7 target (163,842 vertices),
    then displaced icospheres (subdivision 6) and tori of the remaining average size."""
    rng = np.random.Generator(np.random.PCG64(seed))
    placed = [_place(rng, M.displaced_icosphere(rng, 7), half_box)]
    total = placed[0].num_triangles
    while total < total_triangles:
        left = max(1, n_meshes - len(placed))
        per = max(20_000, (total_triangles - total) // left)
        if rng.random() < 0.5 and per < 2 * 81920:
            m = M.displaced_icosphere(rng, 6)
        else:
            m = M.displaced_torus(rng, int(per))
        placed.append(_place(rng, m, half_box))
        total += m.num_triangles
    return assemble(placed)


def scene_batch(seed: int, n_scenes: int, tri_lo: int = 2000, tri_hi: int = 200_000,
                clutter_lo: int = 1, clutter_hi: int = 15, total_lo: int = 10_000,
                total_hi: int = 2_000_000, half_box: float = 1.0):
    """Scenes of uneven size: a target plus 1-15 clutter meshes, totals clipped to a range."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for _ in range(n_scenes):
        placed = [_place(rng, _clutter_mesh(rng, tri_lo, tri_hi), half_box)]
        total = placed[0].num_triangles
        for _ in range(int(rng.integers(clutter_lo, clutter_hi + 1))):
            m = _clutter_mesh(rng, tri_lo, tri_hi)
            if total + m.num_triangles > total_hi:
                break
            placed.append(_place(rng, m, half_box))
            total += m.num_triangles
        while total < total_lo:
            m = _clutter_mesh(rng, tri_lo, tri_hi)
            placed.append(_place(rng, m, half_box))
            total += m.num_triangles
        out.append(assemble(placed))
    return out


def clutterbox(seed: int, n: int = 10, box_side: float = 3.0, tri_lo: int = 2000,
               tri_hi: int = 50_000):
    """Levels 1..n of one clutterbox run (Section 4.1, steps 1-6a).

    The n objects come from the synthetic collection (displaced icospheres and tori of
    tri_lo..tri_hi triangles, log-uniform), each fitted to the unit sphere (step 3).  The
    reference object is one of them chosen at random (step 4) and is placed first; then the
    others follow in random order (step 6).  Every object gets a uniform random orientation and
    a centre uniform in [-(s/2 - 1), s/2 - 1]^3, so its bounding sphere lies inside the box
    (step 6a).  Returns [level_1, ..., level_n]; level k is the combined mesh of the first k
    placed objects, so the reference object's vertex i is vertex i of every level, and level 1
    (the reference alone) gives the reference descriptor set.
    """
    if box_side < 2.0:
        raise ValueError("a unit sphere fits in the clutterbox only when its side is at least 2")
    rng = np.random.Generator(np.random.PCG64(seed))
    objects = [_clutter_mesh(rng, tri_lo, tri_hi) for _ in range(n)]
    ref = int(rng.integers(n))
    order = [ref] + [int(i) for i in rng.permutation([i for i in range(n) if i != ref])]
    half = box_side / 2.0 - 1.0
    placed = [_place(rng, objects[i], half) for i in order]
    return [assemble(placed[:k]) for k in range(1, n + 1)]


def precision_form_scenes(seed: int = 31, n_scenes: int = 6473):
    """The base meshes of the precision-form image set: n_scenes single displaced icospheres
    (subdivision 2, 162 vertices each, as ``tiny_scene``), each with its own seed; their RICI
    images in scene order, first 2^20 kept, make the haystack pool."""
    return [tiny_scene(seed * 100_000 + k) for k in range(n_scenes)]


def scene_batch_pooled(seed: int, n_scenes: int = 256, pool_size: int = 96, tri_lo: int = 2000,
                       tri_hi: int = 200_000, clutter_lo: int = 1, clutter_hi: int = 15,
                       total_lo: int = 10_000, total_hi: int = 2_000_000, half_box: float = 1.0):
    """The batched workload at scale: n_scenes scenes of a target plus clutter_lo..clutter_hi
    clutter meshes (2k-200k triangles, log-uniform), totals clipped to [total_lo, total_hi], with
    every mesh drawn from a seeded pool of ``pool_size`` meshes of the synthetic collection (as
    the clutterbox draws from a fixed object collection) and placed at its own uniform random
    orientation and centre in [-half_box, half_box]^3.  Normals are the pool mesh's area-weighted
    normals (FP64) turned with it.  Building a few hundred scenes of up to 2M triangles from
    scratch would take minutes; placing pooled meshes takes seconds."""
    rng = np.random.Generator(np.random.PCG64(seed))
    pool = [_clutter_mesh(rng, tri_lo, tri_hi) for _ in range(pool_size)]
    pool_n = [M.area_weighted_normals(m.vertices, m.triangles) for m in pool]
    out = []
    for _ in range(n_scenes):
        picks = [int(rng.integers(pool_size))]
        total = pool[picks[0]].num_triangles
        for _ in range(int(rng.integers(clutter_lo, clutter_hi + 1))):
            k = int(rng.integers(pool_size))
            if total + pool[k].num_triangles > total_hi:
                break
            picks.append(k)
            total += pool[k].num_triangles
        while total < total_lo:
            k = int(rng.integers(pool_size))
            picks.append(k)
            total += pool[k].num_triangles
        vs, ns, ts, voff, toff = [], [], [], [], []
        nv = nt = 0
        for k in picks:
            rot = M.random_rotation(rng)
            centre = rng.uniform(-half_box, half_box, size=3)
            vs.append(pool[k].vertices @ rot.T + centre[None, :])
            ns.append(pool_n[k] @ rot.T)
            ts.append(pool[k].triangles + nv)
            voff.append(nv)
            toff.append(nt)
            nv += pool[k].num_vertices
            nt += pool[k].num_triangles
        out.append(Scene(np.ascontiguousarray(np.concatenate(vs).astype(np.float32)),
                         np.ascontiguousarray(np.concatenate(ns).astype(np.float32)),
                         np.ascontiguousarray(np.concatenate(ts).astype(np.int32)),
                         pool[picks[0]].num_vertices, pool[picks[0]].num_triangles, voff, toff))
    return out
