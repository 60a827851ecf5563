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
search call; everything on the way runs in the library's kernels.  Input meshes come from
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


def histograms(prep, results):
    """Per run: ranks, rank histograms (bin i = results at rank i, |CD| bins) and the fraction
    of results at rank 0, one entry per level."""
    out, k = [], 0
    for sizes in prep["sizes"]:
        ranks, hists, frac = [], [], []
        for j, v in enumerate(sizes):
            r = results[k + j]["rank"].cpu().numpy()
            h = np.bincount(r, minlength=v).astype(np.int64)
            ranks.append(r)
            hists.append(h)
            frac.append(float(h[0]) / r.size if r.size else float("nan"))
        out.append({"ranks": ranks, "histograms": hists, "rank0_fraction": frac})
        k += len(sizes)
    return out


def run(runs, support_radius: float = 0.3, resolution: int = 64, mode: int = B.SEARCH_TENSOR,
        device="cuda"):
    """The whole experiment for a list of runs (see ``prepare`` and ``histograms``)."""
    prep = prepare(runs, device)
    res = run_prepared(prep, support_radius, resolution, mode)
    st = B.sync_status()
    if st:
        raise B.RiciError(f"device status {st} in the clutterbox run")
    return histograms(prep, res)
