"""Clutterbox experiment driver (Section 4.1) over the batched GPU path.

A run is a sequence of clutter levels: level 1 holds the reference object alone, level k the
combined mesh of the first k objects (reference first, so the reference object's vertex i is
vertex i of every level).  The reference descriptor set {RD} is the images of the reference
object's vertices at level 1 (step 5); the cluttered set {CD} of level k is the images of every
vertex of that level (step 6b).  Each reference descriptor is searched against {CD} with the
clutter-resistant distance and the rank of its own vertex's image is kept (step 6c); a histogram
of those ranks per level is the experiment's output (step 6d), summarised by the fraction of
results at rank 0 (Section 4.2).

All levels of all runs are imaged by one batched generation call and searched by one batched
search call; everything on the way runs in the library's kernels.  Optionally the clutter of
Eq. clutter is measured around every reference vertex of every level (``rici_clutter``: the
share of the surface area inside its support volume that does not belong to the reference
object), which gives the clutter-versus-rank heatmap of Section 4.2.  Input meshes come from
``synth.scenes.clutterbox`` or any objects with the same fields.
"""
from __future__ import annotations

import numpy as np
import torch

from . import binding as B


def prepare(runs, device="cuda"):
    """Copy every level of every run to the device (inputs of ``run_prepared``).

    runs: list of runs, each a list of level scenes with ``vertices`` float32 [V,3], ``normals``
    float32 [V,3] and ``triangles`` int32 [T,3], level 1 first.
    """
    def dv(a):
        return torch.from_numpy(np.ascontiguousarray(a)).to(device)

    gen, sizes = [], []
    for levels in runs:
        if not levels:
            raise ValueError("a clutterbox run needs at least one level")
        sizes.append([int(sc.vertices.shape[0]) for sc in levels])
        for sc in levels:
            v = int(sc.vertices.shape[0])
            gen.append({"vertices": dv(sc.vertices), "normals": dv(sc.normals),
                        "triangles": dv(sc.triangles),
                        "origins": torch.arange(v, dtype=torch.int32, device=device)})
    return {"gen": gen, "sizes": sizes, "device": device}


def run_prepared(prep, support_radius: float = 0.3, resolution: int = 64,
                 mode: int = B.SEARCH_TENSOR, stream=None):
    """Image every level and search each run's reference descriptors against each of its
    levels.  Returns the per-(run, level) search results (device tensors)."""
    imgs = B.rici_generate_batch(prep["gen"], support_radius, resolution, stream=stream)
    search, k = [], 0
    for sizes in prep["sizes"]:
        rd = imgs[k]  # level 1: the reference object alone
        match = torch.arange(sizes[0], dtype=torch.int64, device=rd.device)
        for j in range(len(sizes)):
            search.append({"needles": rd, "haystack": imgs[k + j], "true_match": match})
        k += len(sizes)
    return B.crss_search_batch(search, resolution, mode=mode, stream=stream)


def clutter_prepared(prep, support_radius: float = 0.3, stream=None):
    """Eq. clutter around every reference vertex of every level: per (run, level) the device
    tensors (A_all, A_object, clutter), the object being the reference object (level 1's
    vertices); the library computes clutter = (A_all - A_object) / A_all."""
    out, k = [], 0
    for sizes in prep["sizes"]:
        ref = torch.arange(sizes[0], dtype=torch.int32, device=prep["gen"][k]["vertices"].device)
        for j in range(len(sizes)):
            g = prep["gen"][k + j]
            out.append(B.clutter_areas(g["vertices"], g["normals"], g["triangles"], ref,
                                       support_radius, sizes[0], with_clutter=True,
                                       stream=stream))
        k += len(sizes)
    return out


RANK_EDGES = np.array([0, 1, 2, 5, 10, 20, 50, 100, 1000, np.iinfo(np.int64).max])


def histograms(prep, results, areas=None, clutter_bins: int = 10):
    """Per run: ranks, rank histograms (bin i = results at rank i, |CD| bins) and the fraction
    of results at rank 0, one entry per level.  With ``areas`` (from ``clutter_prepared``) also
    the clutter of every reference vertex (Eq. clutter, from the library; 0 where the volume
    holds no surface) and a heatmap per level:
    counts of results by clutter (``clutter_bins`` equal bins of [0, 1]) and rank (bins with the
    edges of RANK_EDGES: rank 0, 1, 2-4, 5-9, ...)."""
    out, k = [], 0
    for sizes in prep["sizes"]:
        ranks, hists, frac, clut, heat = [], [], [], [], []
        for j, v in enumerate(sizes):
            r = results[k + j]["rank"].cpu().numpy()
            h = np.bincount(r, minlength=v).astype(np.int64)
            ranks.append(r)
            hists.append(h)
            frac.append(float(h[0]) / r.size if r.size else float("nan"))
            if areas is not None:
                c = np.nan_to_num(areas[k + j][2].cpu().numpy(), nan=0.0)
                clut.append(c)
                ci = np.minimum((c * clutter_bins).astype(np.int64), clutter_bins - 1)
                ri = np.searchsorted(RANK_EDGES, r, side="right") - 1
                hm = np.zeros((clutter_bins, RANK_EDGES.size - 1), np.int64)
                np.add.at(hm, (ci, ri), 1)
                heat.append(hm)
        entry = {"ranks": ranks, "histograms": hists, "rank0_fraction": frac}
        if areas is not None:
            entry["clutter"] = clut
            entry["heatmap"] = heat
        out.append(entry)
        k += len(sizes)
    return out


def run(runs, support_radius: float = 0.3, resolution: int = 64, mode: int = B.SEARCH_TENSOR,
        device="cuda", clutter: bool = False):
    """The whole experiment for a list of runs (see ``prepare`` and ``histograms``)."""
    prep = prepare(runs, device)
    res = run_prepared(prep, support_radius, resolution, mode)
    areas = clutter_prepared(prep, support_radius) if clutter else None
    st = B.sync_status()
    if st:
        raise B.RiciError(st, "device status in the clutterbox run")
    return histograms(prep, res, areas)
