"""Autotuned launch shapes for the batched run, cached per GPU, resolution and workload class.

The library's autotuners (``rici_autotune_generate_batch`` / ``rici_autotune_search_batch``) time
every candidate launch tuning on real inputs with CUDA events; this module decides what to time
them on and remembers the answer.  A cache entry is keyed by the GPU's name, the resolution and a
workload class (the order of magnitude of the per-scene triangle or image counts), so one
measurement serves every later batch of the same shape.  Tunings never change results, only
speed, so a stale or foreign cache entry can cost time but not correctness.

The cache is a JSON file: ``$RICI_TUNING_CACHE`` if set, else ``_build/tuning.json`` beside the
library.
"""
from __future__ import annotations

import json
import math
import os
import tempfile

from . import binding
from . import build as _build


def cache_path() -> str:
    return os.environ.get("RICI_TUNING_CACHE") or os.path.join(_build.BUILD, "tuning.json")


def _mag(x: float) -> int:
    """Order of magnitude in powers of two (0 for empty)."""
    return int(round(math.log2(x))) if x > 0 else 0


def generation_class(scenes, resolution: int) -> str:
    tris = [int(sc["triangles"].shape[0]) for sc in scenes] or [0]
    origins = [int(sc["origins"].numel()) for sc in scenes] or [0]
    return (f"generate|N={int(resolution)}|tri=2^{_mag(sum(tris) / len(tris))}"
            f"|origins=2^{_mag(sum(origins) / len(origins))}")


def search_class(scenes, resolution: int) -> str:
    q = [int(sc["needles"].shape[0]) for sc in scenes] or [0]
    h = [int(sc["haystack"].shape[0]) for sc in scenes] or [0]
    return (f"search|N={int(resolution)}|needles=2^{_mag(sum(q) / len(q))}"
            f"|haystack=2^{_mag(sum(h) / len(h))}")


def load_cache(path: str | None = None) -> dict:
    path = path or cache_path()
    try:
        with open(path) as f:
            data = json.load(f)
        return data if isinstance(data, dict) else {}
    except (OSError, ValueError):
        return {}


def store_cache(cache: dict, path: str | None = None) -> None:
    path = path or cache_path()
    d = os.path.dirname(os.path.abspath(path))
    os.makedirs(d, exist_ok=True)
    fd, tmp = tempfile.mkstemp(dir=d, prefix=".tuning.", suffix=".json")
    with os.fdopen(fd, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def _valid(t) -> bool:
    return isinstance(t, dict) and all(k in t for k in binding.TUNING_FIELDS)


def tune_batch(gen_scenes, search_scenes, support_radius: float, resolution: int, *,
               gpu_name: str, sample: int = 4, repeats: int = 1, path: str | None = None,
               gen_tuner=None, search_tuner=None) -> dict:
    """Tuning for a batched run: cached entries where present, otherwise measured and stored.

    gen_scenes / search_scenes: the batch as passed to rici_generate_batch / crss_search_batch
    (either may be empty).  The autotuners run on the first ``sample`` scenes.  Returns the merged
    tuning (generation fields from the generation entry, tc_group_m from the search entry) and
    applies it with ``binding.set_tuning``.  gen_tuner / search_tuner replace the library's
    autotuners (same signatures; used to test the cache logic without a GPU).
    """
    gen_tuner = gen_tuner or binding.autotune_generate_batch
    search_tuner = search_tuner or binding.autotune_search_batch
    cache = load_cache(path)
    tuning = binding.get_tuning()
    changed = False
    if gen_scenes:
        key = f"{gpu_name}|{generation_class(gen_scenes, resolution)}"
        entry = cache.get(key)
        if not (isinstance(entry, dict) and _valid(entry.get("tuning"))):
            best, ms = gen_tuner(list(gen_scenes)[:sample], support_radius, resolution,
                                 repeats=repeats)
            entry = {"tuning": best, "ms": ms, "scenes_timed": min(sample, len(gen_scenes))}
            cache[key] = entry
            changed = True
        for f in ("gen_cells_per_reach", "gen_big_radius", "gen_warps"):
            tuning[f] = entry["tuning"][f]
    if search_scenes:
        key = f"{gpu_name}|{search_class(search_scenes, resolution)}"
        entry = cache.get(key)
        if not (isinstance(entry, dict) and _valid(entry.get("tuning"))):
            best, ms = search_tuner(list(search_scenes)[:sample], resolution, repeats=repeats)
            entry = {"tuning": best, "ms": ms, "scenes_timed": min(sample, len(search_scenes))}
            cache[key] = entry
            changed = True
        tuning["tc_group_m"] = entry["tuning"]["tc_group_m"]
    if changed:
        store_cache(cache, path)
    binding.set_tuning(tuning)
    return tuning
