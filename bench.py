#!/usr/bin/env python
"""Benchmark of the RICI hot path on the large scene (one JSON line on stdout).

Workload (the largest single-GPU configuration): 41 seeded displaced meshes (a subdivision-7
icosphere target, subdivision-6 icospheres and tori) with 5,019,510 triangles and 2,509,797
vertices, centres in [-1,1]^3 (box of side 4, every bounding sphere inside).  One step is the
whole hot path over that scene:
  1. RICI 64x64 images of every vertex at support radii 0.15, 0.3 and 0.6 (7,529,391 images),
  2. RICI images (R = 0.3) of 100,000 seeded target vertices with the target alone (needles),
  3. clutter-resistant search of every needle against all 2,509,797 R = 0.3 images
     (2.5e11 comparisons): rank of its true match (the same vertex), true distance, top-1.
value = images generated per second of the whole step (7,629,391 images / step time); the
breakdown gives every part and comparisons/s.  Inputs are resident in HBM (all images are
larger than L2) and L2 is flushed by a 512 MB write before every timed step.  e2e repeats the
step through the same public API from pinned host buffers with the copies timed.

Beside the step (outside its timed region): the other exact search forms on a needle sample of
the same images (int8 tensor cores, CUDA-core dense, sparse-needle), and the comparison
workloads: the clutter scene, the precision-form image set at full size, the batched run of
256 scenes at full size, a synthetic clutterbox experiment, the clutter measure and spin images.

--impl reference times the CPU oracle (FP64 brute force / int64 distances) on bounded samples
of the same workload: each step is one sample, its measured time is the line's ms_per_step, and
the rate is the samples' rate extrapolated to the full step's mix of generation and search.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "RICI images/s; CRSS comparisons/s (int8-TC vs CUDA-core), ranks exact vs oracle"
N_RES = 64
RADII = (0.15, 0.3, 0.6)
R_SEARCH = 0.3
SEED = 5
NEEDLES = 100_000
WORKLOAD = ("large scene: 41 displaced meshes (icosphere target of subdivision 7, icospheres of "
            "subdivision 6 and tori), 5,019,510 triangles, 2,509,797 vertices, box side 4; RICI "
            "64x64 uint16 of every vertex at R = 0.15, 0.3, 0.6, then 100,000 seeded target "
            "vertices imaged with the target alone (R = 0.3) searched against all 2,509,797 "
            "R = 0.3 images (tensor-core CRSS): rank, true distance, top-1")

# FP32 operations of the definition (Section 3.1.2), counted from its formulas:
#  F_PROJ per projected vertex: P' = P - S (3 subtractions), P''x, P''y, Tx, Tz (2 products and
#    a sum each: 12) = 15;
#  F_LAYER per (triangle, layer) crossing: per crossed edge lambda = (beta - z_u) / (z_v - z_u)
#    (2 subtractions, 1 division) and E = T_u + lambda (T_v - T_u) in x and y (2 x 3) = 9, two
#    edges = 18; |E0|^2, |E1|^2, E0.D, E1.D, E0 x D, |D|^2 (3 each = 18) and D (2) = 20; = 38;
#  F_COL per crossing: the interval boundaries, min/max of |E|^2 (1), h^2 = (E0 x D)^2 / |D|^2
#    (2), the two sign tests d0 < 0 < d1 (2) and the comparisons that place the single and double
#    intervals against the bin radii (3) = 8.
# Work is counted only where it can change an image: pairs and crossings whose segment comes
# within the largest circle (the oracle's contributing counters); culled work is not counted.
F_PROJ = 15
F_LAYER = 38
F_COL = 8
# int8 multiply-adds per masked squared difference in the expanded form m(a-b)^2 =
# a^2 - 2ab + (mb)^2 with sum a^2 per row precomputed: one for a*b and one for (mb)*(mb)
MACS_PER_TERM = 2
DP4A_PER_SM_CLK = 64
# DRAM bytes (read + write) per full-size launch from one-pass ncu captures (commands in
# profiles/); None where the kernel changed since it was captured
# (k_generate at R = 0.6: 235.9 GB read + 32.2 GB written on the first 131,072 origins, in a
# run whose tuner chose 8 warps per point, scaled to the full launch by 2,509,797 / 131,072
# origins)
TRAFFIC = {"k_generate_R0.6": (235.93e9 + 32.17e9) * 2509797 / 131072,
           "k_tc_rank_clutter": 21.483e9 + 3.71e5, "k_dense_clutter": 1.895e9 + 5.57e6}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--search-mode", type=int, default=3,
                    help="search form of the step (3 tensor cores, 1 CUDA cores, 4 sparse, "
                         "5 int8 tensor cores)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default launch tuning instead of autotuning each radius")
    ap.add_argument("--forms-needles", type=int, default=10_000,
                    help="needle sample for the other search forms on the step's images")
    ap.add_argument("--cpu-origins", type=int, default=256,
                    help="oracle sample: oriented points per radius (scene brute force)")
    ap.add_argument("--cpu-needle-origins", type=int, default=64)
    ap.add_argument("--cpu-needles", type=int, default=32)
    ap.add_argument("--cpu-haystack", type=int, default=100_000)
    ap.add_argument("--clutter-compare", type=int, default=1,
                    help="the clutter scene (10 meshes, 229,756 triangles): generation and search")
    ap.add_argument("--precision-compare", type=int, default=1,
                    help="the precision-form set at full size (2^20 RICI images, 65,536 needles)")
    ap.add_argument("--batched-compare", type=int, default=1,
                    help="the batched run at full size (256 scenes, 1,024 needles each)")
    ap.add_argument("--clutterbox-compare", type=int, default=1,
                    help="a synthetic clutterbox experiment (Section 4.1) with the clutter measure")
    ap.add_argument("--spin-compare", type=int, default=1,
                    help="spin images (Section 2.1) of the clutter scene")
    ap.add_argument("--origin-limit", type=int, default=0,
                    help="image only the first V scene vertices (small profiling case)")
    ap.add_argument("--needle-limit", type=int, default=0,
                    help="use only the first Q needles (small profiling case)")
    ap.add_argument("--radii", type=str, default="",
                    help="comma-separated subset of the support radii (small profiling case)")
    ap.add_argument("--budget-s", type=float, default=1400.0,
                    help="wall-time budget of the run: a comparison workload that would start "
                         "after it is skipped (the step, its warm-up, e2e and the CPU baseline "
                         "always run)")
    return ap.parse_args()


def input_digest(scene) -> str:
    """First 16 hex digits of the SHA-256 of the scene's vertex, normal and triangle arrays."""
    h = hashlib.sha256()
    for a in (scene.vertices, scene.normals, scene.triangles):
        h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()[:16]


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x: float, device) -> float:
    """The largest value over all ranks (a job's step time is its slowest rank's); x itself when
    no process group is running or it has one rank."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, ms: float, world: int) -> float:
    """Whole-job throughput: every rank processes units_per_rank in ms (the max over ranks)."""
    return world * units_per_rank / (ms / 1e3)


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for name, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(name)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


class Timer:
    """CUDA events on the launching stream around named parts of a step."""

    def __init__(self, torch, stream):
        self.torch, self.stream, self.marks = torch, stream, []

    def mark(self, name):
        e = self.torch.cuda.Event(enable_timing=True)
        e.record(self.stream)
        self.marks.append((name, e))

    def parts(self):
        self.torch.cuda.synchronize()
        return {self.marks[k + 1][0]: self.marks[k][1].elapsed_time(self.marks[k + 1][1])
                for k in range(len(self.marks) - 1)}


def timed_ms(torch, stream, fn, reps=1, flush=None):
    """Mean CUDA-event time of fn over reps runs (after one warm-up run)."""
    out = fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        if flush is not None:
            flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return statistics.mean(ts), out


def release(p, torch):
    p.binding.release_workspaces()
    torch.cuda.empty_cache()


def run_comparisons(todo, t_start: float, budget_s: float, after=None, clock=time.time) -> dict:
    """Runs the enabled workloads of todo = [(name, enabled, run)] in order; one whose start would
    come more than budget_s seconds after t_start is reported as skipped instead.  after() runs
    after each workload that ran."""
    out = {}
    for name, enabled, run in todo:
        if not enabled:
            continue
        if clock() - t_start > budget_s:
            out[name] = {"skipped": f"the run's wall-time budget ({budget_s:.0f} s) was spent "
                                    "before it started"}
            continue
        out[name] = run()
        if after:
            after()
    return out


def build_workload():
    import synth

    return synth.large_scene(seed=SEED)


def needle_origins(scene, limit=0):
    rng = np.random.default_rng(SEED)
    q = min(NEEDLES, scene.target_vertices)
    on = np.sort(rng.choice(scene.target_vertices, q, replace=False)).astype(np.int32)
    return on[:limit] if limit else on


def cpu_baseline(scene, args, steps: int = 1):
    """Oracle on bounded samples of the step; per step the seconds extrapolated to the whole
    step and the seconds the samples took, threads, sample text and the oracle's per-origin work
    counters at each radius."""
    import oracle
    import synth

    oracle.build()
    rng = np.random.default_rng(123)
    V, Vt = scene.num_vertices, scene.target_vertices
    Q = len(needle_origins(scene, args.needle_limit))
    if args.origin_limit:
        V = min(V, args.origin_limit)
    tgt = scene.target_only()
    og = {R: rng.choice(scene.num_vertices, args.cpu_origins, replace=False) for R in RADII}
    on = rng.choice(Vt, args.cpu_needle_origins, replace=False)
    ims_rng = np.random.default_rng(7)
    nd = synth.images.rici_like_images(ims_rng, args.cpu_needles, N_RES)
    hay = synth.images.rici_like_images(ims_rng, args.cpu_haystack, N_RES)
    threads = oracle.max_threads()
    est, wall, work = [], [], {}
    for _ in range(steps):
        total = 0.0
        w0 = time.perf_counter()
        for R in RADII:
            t0 = time.perf_counter()
            _, c = oracle.rici_fp64(scene.vertices, scene.normals, scene.triangles, og[R], R, N_RES,
                                    return_counters=True)
            total += (time.perf_counter() - t0) / len(og[R]) * V
            work[R] = {k: v / len(og[R]) for k, v in c.items()}
        t0 = time.perf_counter()
        oracle.rici_fp64(tgt.vertices, tgt.normals, tgt.triangles, on, R_SEARCH, N_RES)
        total += (time.perf_counter() - t0) / len(on) * Q
        t0 = time.perf_counter()
        oracle.crss_search(nd, hay, np.zeros(len(nd), np.int64))
        total += (time.perf_counter() - t0) / (len(nd) * len(hay)) * Q * V
        est.append(total)
        wall.append(time.perf_counter() - w0)
    sample = (f"{args.cpu_origins} scene-vertex images per radius at R = 0.15 / 0.3 / 0.6 and "
              f"{len(on)} target-alone images (FP64 brute force over all {scene.num_triangles} "
              f"triangles), {len(nd)} needles x {len(hay)} haystack images (int64 distances) per "
              f"step, extrapolated to {3 * V + Q} images and {Q * V} comparisons")
    return est, wall, threads, sample, work


def generation_work(work, F=None):
    """Definition FP32 operations per oriented point from the oracle's contributing counters."""
    return (F_PROJ * 3 * work["pairs_contributing"] +
            (F_LAYER + F_COL) * work["crossings_contributing"])


def search_forms(p, torch, stream, nd, hay, match, q, ref):
    """The other exact forms on the first q needles of the step's search (same images)."""
    out = {"needles": q, "haystack": int(hay.shape[0]), "comparisons": q * int(hay.shape[0])}
    ndq, mq = nd[:q], match[:q]
    for name, mode in (("tensor_core", p.SEARCH_TENSOR), ("int8_tensor_core", p.SEARCH_INT8_TC),
                       ("cuda_core_dense", p.SEARCH_CUDA_CORE), ("sparse_needle", p.SEARCH_SPARSE),
                       ("auto", p.SEARCH_AUTO)):
        cnt = torch.zeros(4, dtype=torch.int64, device=nd.device)
        p.crss_search(ndq, hay, mq, mode=mode, counters=cnt)  # warm-up, with the work counters
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = p.crss_search(ndq, hay, mq, mode=mode)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        same = all(bool(torch.equal(r[k], ref[k][:q])) for k in ("rank", "true_distance", "top1"))
        out[name] = {"ms": ms, "comparisons_per_s": q * int(hay.shape[0]) / (ms / 1e3),
                     "same_as_step": same, "counters": [int(x) for x in cnt.cpu()],
                     "status": p.sync_status()}
        del r
    return out


def clutter_scene_comparison(p, torch, dev, stream, flush, steps=3):
    """The clutter scene (target icosphere of subdivision 5 + 9 clutter meshes, 229,756
    triangles): needle and haystack images and the CUDA-core search, as one step; the same search
    in the tensor-core form; the dense kernel's roofline (dp4a issue)."""
    import synth

    s = synth.clutter_scene(seed=2)
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
    v, n, t = d(s.vertices), d(s.normals), d(s.triangles)
    on = d(np.arange(s.target_vertices, dtype=np.int32))
    oh = d(np.arange(s.num_vertices, dtype=np.int32))
    m = torch.arange(s.target_vertices, dtype=torch.int64, device=dev)
    Vt, V = s.target_vertices, s.num_vertices
    nd = p.rici_generate(v, n, t[: s.target_triangles], on, R_SEARCH, N_RES)
    hy = p.rici_generate(v, n, t, oh, R_SEARCH, N_RES)
    res = {}
    for _ in range(2):
        p.crss_search(nd, hy, m, mode=p.SEARCH_CUDA_CORE)
    torch.cuda.synchronize()
    parts = []
    for _ in range(steps):
        flush.zero_()
        torch.cuda.nvtx.range_push("clutter_step")  # selects these launches for ncu
        tm = Timer(torch, stream)
        tm.mark("start")
        p.rici_generate(v, n, t[: s.target_triangles], on, R_SEARCH, N_RES, out=nd)
        tm.mark("needles")
        p.rici_generate(v, n, t, oh, R_SEARCH, N_RES, out=hy)
        tm.mark("haystack")
        r = p.crss_search(nd, hy, m, mode=p.SEARCH_CUDA_CORE)
        tm.mark("search")
        torch.cuda.nvtx.range_pop()
        parts.append(tm.parts())
    torch.cuda.nvtx.range_push("clutter_sparse")
    p.crss_search(nd, hy, m, mode=p.SEARCH_SPARSE)
    torch.cuda.nvtx.range_pop()
    ms = {k: statistics.mean(x[k] for x in parts) for k in parts[0]}
    cnt = torch.zeros(4, dtype=torch.int64, device=dev)
    p.crss_search(nd, hy, m, mode=p.SEARCH_CUDA_CORE, counters=cnt)
    cnt = [int(x) for x in cnt.cpu()]
    torch.cuda.nvtx.range_push("clutter_tc")  # selects these launches for ncu
    tc_ms, rt = timed_ms(torch, stream, lambda: p.crss_search(nd, hy, m, mode=p.SEARCH_TENSOR),
                         reps=steps, flush=flush)
    torch.cuda.nvtx.range_pop()
    same = all(bool(torch.equal(rt[k], r[k])) for k in ("rank", "true_distance", "top1"))
    pairs = V * Vt
    res = {"recipe": "synth.clutter_scene(seed=2): 10 meshes, 229,756 triangles, N = 64, R = 0.3",
           "needles": Vt, "haystack": V, "comparisons": pairs, "step_ms": sum(ms.values()),
           "needle_generation_ms": ms["needles"], "haystack_generation_ms": ms["haystack"],
           "images_per_s": (V + Vt) / (sum(ms.values()) / 1e3),
           "cuda_core_search_ms": ms["search"],
           "cuda_core_comparisons_per_s": pairs / (ms["search"] / 1e3),
           "pair_rows": cnt[0], "lane_utilisation": cnt[0] / cnt[3] if cnt[3] else None,
           "tensor_core_search_ms": tc_ms,
           "tensor_core_comparisons_per_s": pairs / (tc_ms / 1e3),
           "tensor_core_same_ranks": same, "status": p.sync_status()}
    del nd, hy, r, rt
    return res


def precision_form_comparison(p, torch, dev, stream, flush, i8_needles=16384):
    """The precision-form set at full size: 2^20 RICI images (N = 64, R = 0.3) of 6,473 seeded
    subdivision-2 icospheres with heavy-tailed plateaus, 65,536 needles taken before clutter
    plateaus; every exact form of the search (the int8 tensor-core form on a needle sample)."""
    import synth

    H, Q = 1 << 20, 65536
    scenes = synth.scenes.precision_form_scenes(31, 6473)
    tails, match, clutter = synth.images.precision_form_recipe(31, H, Q, N_RES)
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
    total = sum(sc.num_vertices for sc in scenes)
    base = torch.empty((total, N_RES, N_RES), dtype=torch.uint16, device=dev)
    gen, k = [], 0
    for sc in scenes:
        gen.append({"vertices": d(sc.vertices), "normals": d(sc.normals),
                    "triangles": d(sc.triangles),
                    "origins": d(np.arange(sc.num_vertices, dtype=np.int32)),
                    "out": base[k:k + sc.num_vertices]})
        k += sc.num_vertices
    gen_ms, _ = timed_ms(torch, stream, lambda: p.rici_generate_batch(gen, R_SEARCH, N_RES))
    hay = base[:H]
    synth.images.apply_plateaus_torch(hay, tails)
    nd = hay.view(torch.int16)[d(match)].view(torch.uint16)
    synth.images.apply_plateaus_torch(hay, clutter)
    m = d(match)
    out = {"recipe": "6,473 seeded subdivision-2 icospheres (synth.scenes.precision_form_scenes(31)"
                     "), RICI 64x64 at R = 0.3, first 2^20 images; synth.images."
                     "precision_form_recipe(31): heavy-tailed plateaus, 65,536 needles, clutter",
           "generation_ms": gen_ms, "generation_images_per_s": total / (gen_ms / 1e3),
           "scenes": len(scenes), "needles": Q, "haystack": H, "comparisons": Q * H}
    ref = None
    for name, mode, q in (("tensor_core", p.SEARCH_TENSOR, Q), ("cuda_core_dense", p.SEARCH_CUDA_CORE, Q),
                          ("sparse_needle", p.SEARCH_SPARSE, Q), ("auto", p.SEARCH_AUTO, Q),
                          ("int8_tensor_core", p.SEARCH_INT8_TC, i8_needles)):
        ms, r = timed_ms(torch, stream, lambda: p.crss_search(nd[:q], hay, m[:q], mode=mode),
                         flush=flush)
        if ref is None:
            ref = r
        same = all(bool(torch.equal(r[k2], ref[k2][:q])) for k2 in ("rank", "true_distance", "top1"))
        out[name] = {"needles": q, "ms": ms, "comparisons_per_s": q * H / (ms / 1e3),
                     "same_as_tensor_core": same}
        del r
    out["status"] = p.sync_status()
    del gen, base, hay, nd, m, ref
    release(p, torch)
    return out


def batched_full(p, torch, dev, stream, n_scenes=256, needles=1024, seed=44,
                 chunk_images=6_000_000):
    """The batched run at its stated size: 256 scenes of a target plus 1-15 clutter meshes
    (2k-200k triangles each, 10k-2M per scene) from a pooled collection, needle images of up to
    1,024 seeded target vertices per scene (target alone), haystack images of every scene vertex,
    tensor-core search per scene.  The scenes do not fit on the device at once (about 0.45 TB of
    images), so they run in chunks of at most chunk_images haystack images, each chunk one
    rici_batch_run call; against one rici_generate / rici_generate / crss_search sequence per
    scene over the same chunks."""
    import synth

    t0 = time.time()
    scenes = synth.scenes.scene_batch_pooled(seed, n_scenes)
    build_s = time.time() - t0
    rng = np.random.default_rng(3)
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
    chunks, cur, cur_n = [], [], 0
    for s in scenes:
        if cur and cur_n + s.num_vertices > chunk_images:
            chunks.append(cur)
            cur, cur_n = [], 0
        cur.append(s)
        cur_n += s.num_vertices
    if cur:
        chunks.append(cur)

    def prepare(chunk):
        xs = []
        for s in chunk:
            q = min(needles, s.target_vertices)
            on = np.sort(rng.choice(s.target_vertices, q, replace=False)).astype(np.int32)
            xs.append({"vertices": d(s.vertices), "normals": d(s.normals),
                       "triangles": d(s.triangles), "target_triangles": s.target_triangles,
                       "needle_origins": d(on),
                       "haystack_origins": d(np.arange(s.num_vertices, dtype=np.int32)),
                       "true_match": d(on.astype(np.int64))})
        return xs

    t_b = t_p = 0.0
    images = pairs = 0
    same = True
    first = True
    for chunk in chunks:
        xs = prepare(chunk)
        if first:  # warm-up on the first chunk
            p.batch_run(xs, R_SEARCH, N_RES)
            torch.cuda.synchronize()
            release(p, torch)
            first = False
        ms_b, rb = timed_ms(torch, stream, lambda: p.batch_run(xs, R_SEARCH, N_RES), reps=1)
        rb = [{k: r[k].clone() for k in ("rank", "true_distance", "top1")} for r in rb]
        release(p, torch)

        def plain():
            out = []
            for x in xs:
                ni = p.rici_generate(x["vertices"], x["normals"],
                                     x["triangles"][: x["target_triangles"]], x["needle_origins"],
                                     R_SEARCH, N_RES)
                hi = p.rici_generate(x["vertices"], x["normals"], x["triangles"],
                                     x["haystack_origins"], R_SEARCH, N_RES)
                out.append(p.crss_search(ni, hi, x["true_match"], mode=p.SEARCH_TENSOR))
                del ni, hi
            return out

        ms_p, rp = timed_ms(torch, stream, plain, reps=1)
        for a, b in zip(rb, rp):
            same &= all(bool(torch.equal(a[k], b[k])) for k in ("rank", "true_distance", "top1"))
        t_b += ms_b
        t_p += ms_p
        images += sum(int(x["needle_origins"].numel() + x["haystack_origins"].numel()) for x in xs)
        pairs += sum(int(x["needle_origins"].numel()) * int(x["haystack_origins"].numel())
                     for x in xs)
        del xs, rb, rp
        release(p, torch)
    return {"recipe": f"synth.scenes.scene_batch_pooled(seed={seed}, {n_scenes} scenes, pool of "
                      f"96 meshes), up to {needles} needles per scene (target alone) vs every "
                      "scene vertex, N = 64, R = 0.3, tensor-core search",
            "scenes": n_scenes, "triangles": int(sum(s.num_triangles for s in scenes)),
            "chunks": len(chunks), "images": images, "comparisons": pairs,
            "batched_ms": t_b, "per_scene_calls_ms": t_p, "speedup": t_p / t_b,
            "batched_images_per_s": images / (t_b / 1e3),
            "batched_comparisons_per_s": pairs / (t_b / 1e3),
            "same_results": same, "scene_build_s": build_s, "status": p.sync_status()}


def clutterbox_experiment(p, torch, dev, stream, runs=4, n=10, seed=51, tri_lo=2000,
                          tri_hi=20000, steps=3):
    """Synthetic clutterbox runs (Section 4.1): every level of every run imaged by one batched
    generation call and searched by one batched search call (tensor-core form)."""
    import synth
    from paper_2007_02306_gb300 import clutterbox

    levels = [synth.scenes.clutterbox(seed + r, n=n, box_side=3.0, tri_lo=tri_lo, tri_hi=tri_hi)
              for r in range(runs)]
    prep = clutterbox.prepare(levels, dev)
    clutterbox.run_prepared(prep, R_SEARCH, N_RES)
    torch.cuda.synchronize()
    ts = []
    for _ in range(steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res = clutterbox.run_prepared(prep, R_SEARCH, N_RES)
        e1.record(stream)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    # Eq. clutter around every reference vertex of every level (clutter-versus-rank heatmap)
    areas = clutterbox.clutter_prepared(prep, R_SEARCH)
    torch.cuda.synchronize()
    tc = []
    for _ in range(steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        areas = clutterbox.clutter_prepared(prep, R_SEARCH)
        e1.record(stream)
        torch.cuda.synchronize()
        tc.append(e0.elapsed_time(e1))
    st = p.sync_status()
    h = clutterbox.histograms(prep, res, areas)
    lv5 = min(4, n - 1)  # the paper's heatmaps: scenes with 4 added objects
    heat = np.sum([r["heatmap"][lv5] for r in h], axis=0)
    with np.errstate(invalid="ignore", divide="ignore"):
        r0_by_clutter = [float(x) if np.isfinite(x) else None
                         for x in heat[:, 0] / heat.sum(axis=1)]
    clutter_points = sum(sz[0] * len(sz) for sz in prep["sizes"])
    images = sum(sum(sz) for sz in prep["sizes"])
    comparisons = sum(sz[0] * sum(sz) for sz in prep["sizes"])
    t = statistics.mean(ts)
    out = {"runs": runs, "levels": n, "box_side": 3.0, "images": images,
           "comparisons": comparisons, "ms": t, "runs_per_s": runs / (t / 1e3),
           "images_per_s": images / (t / 1e3),
           "rank0_fraction_by_level": [float(x) for x in
                                       np.mean([r["rank0_fraction"] for r in h], axis=0)],
           "clutter_ms": statistics.mean(tc), "clutter_points": clutter_points,
           "clutter_points_per_s": clutter_points / (statistics.mean(tc) / 1e3),
           "heatmap_level": lv5 + 1,
           "heatmap_rank_edges": [int(x) for x in clutterbox.RANK_EDGES[:-1]],
           "heatmap_counts": heat.tolist(),
           "rank0_fraction_by_clutter_decile": r0_by_clutter,
           "status": st,
           "recipe": f"synth.scenes.clutterbox(seed={seed}..{seed + runs - 1}, n={n}, box side 3, "
                     f"objects of {tri_lo}-{tri_hi} triangles), N = {N_RES}, R = {R_SEARCH}"}
    del prep, res, areas
    torch.cuda.empty_cache()
    return out


def spin_comparison(p, torch, dev, stream, flush, steps=3):
    """Spin images (Section 2.1, 9 samples per triangle) of every vertex of the clutter scene,
    beside the RICI images of the same points."""
    import synth

    s = synth.clutter_scene(seed=2)
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
    v, n, t = d(s.vertices), d(s.normals), d(s.triangles)
    oh = d(np.arange(s.num_vertices, dtype=np.int32))
    si = torch.empty((s.num_vertices, N_RES, N_RES), dtype=torch.float32, device=dev)
    torch.cuda.nvtx.range_push("spin_images")
    p.spin_images(v, n, t, oh, R_SEARCH, N_RES, 3, out=si)
    torch.cuda.nvtx.range_pop()
    ms, _ = timed_ms(torch, stream, lambda: p.spin_images(v, n, t, oh, R_SEARCH, N_RES, 3, out=si),
                     reps=steps, flush=flush)
    rms, _ = timed_ms(torch, stream, lambda: p.rici_generate(v, n, t, oh, R_SEARCH, N_RES),
                      reps=steps, flush=flush)
    return {"images": s.num_vertices, "samples_per_triangle": 9, "ms": ms,
            "images_per_s": s.num_vertices / (ms / 1e3), "rici_images_ms": rms,
            "status": p.sync_status()}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    scene = build_workload()
    cpu_baseline(scene, args, steps=max(0, args.warmup))
    est, wall, threads, sample, _ = cpu_baseline(scene, args, steps=args.steps)
    images = 3 * scene.num_vertices + len(needle_origins(scene))
    sec = statistics.mean(est)
    value = images / sec
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "images/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        # a step is one bounded sample of the workload (the samples below); value is the rate
        # those samples give for the whole step's mix of generation and search
        "ms_per_step": statistics.mean(wall) * 1e3,
        "ms_per_step_kind": "measured: one oracle sample step on the host cores",
        "ms_per_full_step_extrapolated": sec * 1e3,
        "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64+i64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "resolution": N_RES, "support_radii": list(RADII),
                   "seed": SEED},
        "cpu_baseline": {"value": value, "unit": "images/s", "cores": threads, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "images/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    t_start = time.time()
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())

    import paper_2007_02306_gb300 as p
    from paper_2007_02306_gb300 import build as libbuild

    if rank == 0:
        libbuild.build()
    if world > 1:
        torch.distributed.barrier()
    p.load_library()

    scene = build_workload()
    global RADII
    if args.radii:
        RADII = tuple(float(x) for x in args.radii.split(","))
        if R_SEARCH not in RADII:
            raise SystemExit("--radii must include the search radius 0.3")
    V = scene.num_vertices if not args.origin_limit else min(scene.num_vertices, args.origin_limit)
    Vt, Tt, T = scene.target_vertices, scene.target_triangles, scene.num_triangles
    on_np = needle_origins(scene, args.needle_limit)
    Q = len(on_np)
    if args.origin_limit or args.needle_limit or args.radii:
        args.no_cpu_baseline = True
    h_vert = torch.from_numpy(scene.vertices).pin_memory()
    h_norm = torch.from_numpy(scene.normals).pin_memory()
    h_tri = torch.from_numpy(scene.triangles).pin_memory()
    h_oh = torch.arange(V, dtype=torch.int32).pin_memory()
    h_on = torch.from_numpy(on_np).pin_memory()
    h_match = torch.from_numpy(on_np.astype(np.int64)).pin_memory()
    vert, norm, tri = h_vert.to(dev), h_norm.to(dev), h_tri.to(dev)
    oh, on, match = h_oh.to(dev), h_on.to(dev), h_match.to(dev)
    imgs = {R: torch.empty((V, N_RES, N_RES), dtype=torch.uint16, device=dev) for R in RADII}
    needles = torch.empty((Q, N_RES, N_RES), dtype=torch.uint16, device=dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    # launch tuning of each radius, measured on three contiguous blocks of oriented points (the
    # order of the full run, so their cache behaviour is the full run's), fresh every run
    tunings, tune_s = {}, 0.0
    t0 = time.time()
    blk = min(4096, V)
    sub = torch.cat([oh[:blk], oh[V // 2: V // 2 + blk], oh[V - blk:]]).contiguous()
    subout = torch.empty((sub.numel(), N_RES, N_RES), dtype=torch.uint16, device=dev)
    for R in RADII:
        if args.no_autotune:
            tunings[R] = p.get_tuning()
        else:
            tunings[R], _ = p.autotune_generate_batch(
                [{"vertices": vert, "normals": norm, "triangles": tri, "origins": sub,
                  "out": subout}], R, N_RES, repeats=2)
    tune_s = time.time() - t0
    del sub, subout

    def step(vv, nn, tt, ohh, onn, mm, tm=None, gcnt=None, scnt=None):
        for R in RADII:
            p.set_tuning(tunings[R])
            p.rici_generate(vv, nn, tt, ohh, R, N_RES, out=imgs[R],
                            counters=None if gcnt is None else gcnt[R])
            if tm:
                tm.mark(f"generation_R{R}")
        p.set_tuning(tunings[R_SEARCH])
        p.rici_generate(vv, nn, tt[:Tt], onn, R_SEARCH, N_RES, out=needles)
        if tm:
            tm.mark("needle_generation")
        r = p.crss_search(needles, imgs[R_SEARCH], mm, mode=args.search_mode, counters=scnt)
        if tm:
            tm.mark("search")
        return r

    gcnt = {R: torch.zeros(4, dtype=torch.int64, device=dev) for R in RADII}
    scnt = torch.zeros(4, dtype=torch.int64, device=dev)
    for k in range(args.warmup):
        last = k == args.warmup - 1
        step(vert, norm, tri, oh, on, match, gcnt=gcnt if last else None,
             scnt=scnt if last else None)
    torch.cuda.synchronize()
    st = p.sync_status()
    if st != 0:
        raise RuntimeError(f"device status {st} during warm-up")
    gcnt = {R: [int(x) for x in c.cpu()] for R, c in gcnt.items()}
    scnt = [int(x) for x in scnt.cpu()]

    clocks = ClockSampler(dev.index if world == 1 else local)
    launches0 = p.binding.kernel_launches()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    parts = []
    for k in range(args.steps):
        flush.zero_()
        torch.cuda.nvtx.range_push("timed_step")  # selects the step's launches for ncu
        tm = Timer(torch, stream)
        tm.mark("start")
        res = step(vert, norm, tri, oh, on, match, tm=tm)
        parts.append(tm)
        torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    clk = clocks.stop()
    launches = p.binding.kernel_launches() - launches0
    if world > 1:
        torch.distributed.barrier()
    st = p.sync_status()
    if st != 0:
        raise RuntimeError(f"device status {st} in the timed region")
    parts = [tm.parts() for tm in parts]
    pms = {k: statistics.mean(x[k] for x in parts) for k in parts[0]}
    ms_step = max_over_ranks(statistics.mean(sum(x.values()) for x in parts), dev)
    images = len(RADII) * V + Q
    pairs = Q * V
    value = job_rate(images, ms_step, world)
    rk = res["rank"].cpu().numpy()

    # the other exact forms of the same search on a needle sample of the step's images
    forms = None
    if rank == 0 and args.forms_needles:
        forms = search_forms(p, torch, stream, needles, imgs[R_SEARCH], match,
                             min(args.forms_needles, Q), res)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    dp4a_rate = p.binding.measure_dp4a_rate()
    mma_rate = p.binding.measure_mma_s8_rate()

    # e2e: the same step from pinned host buffers, host<->device copies inside the timed region
    e2e = None
    if not args.no_e2e:
        h_rank = torch.empty(Q, dtype=torch.int32).pin_memory()
        h_top1 = torch.empty(Q, dtype=torch.int32).pin_memory()
        h_dt = torch.empty(Q, dtype=torch.int64).pin_memory()
        e2e_ms = []
        # one untimed pass warms the copy path, then up to two timed passes (the step is long)
        for k in range(min(args.steps, 2) + 1):
            flush.zero_()
            a0 = torch.cuda.Event(enable_timing=True)
            a1 = torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            dv = h_vert.to(dev, non_blocking=True)
            dn = h_norm.to(dev, non_blocking=True)
            dtri = h_tri.to(dev, non_blocking=True)
            doh = h_oh.to(dev, non_blocking=True)
            don = h_on.to(dev, non_blocking=True)
            dm = h_match.to(dev, non_blocking=True)
            r = step(dv, dn, dtri, doh, don, dm)
            h_rank.copy_(r["rank"], non_blocking=True)
            h_top1.copy_(r["top1"], non_blocking=True)
            h_dt.copy_(r["true_distance"], non_blocking=True)
            a1.record(stream)
            torch.cuda.synchronize()
            if k > 0:  # the first pass warms the copy path
                e2e_ms.append(a0.elapsed_time(a1))
            del dv, dn, dtri, doh, don, dm, r
        e_ms = max_over_ranks(statistics.mean(e2e_ms), dev)
        h2d = sum(x.numel() * x.element_size() for x in (h_vert, h_norm, h_tri, h_oh, h_on, h_match))
        d2h = Q * (4 + 4 + 8)
        e2e = {"value": job_rate(images, e_ms, world), "unit": "images/s",
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": e_ms}
    st = p.sync_status()

    # free the step's buffers before the comparison workloads
    del imgs, needles, res, vert, norm, tri, oh, on, match
    p.set_tuning(None)
    release(p, torch)

    cmp = {}
    if rank == 0:
        # comparison workloads in order, each only if the run's wall-time budget is not spent
        todo = [("clutter_scene", args.clutter_compare,
                 lambda: clutter_scene_comparison(p, torch, dev, stream, flush)),
                ("precision_form", args.precision_compare,
                 lambda: precision_form_comparison(p, torch, dev, stream, flush)),
                ("batched_run", args.batched_compare, lambda: batched_full(p, torch, dev, stream)),
                ("clutterbox", args.clutterbox_compare,
                 lambda: clutterbox_experiment(p, torch, dev, stream)),
                ("spin_images", args.spin_compare,
                 lambda: spin_comparison(p, torch, dev, stream, flush))]
        cmp = run_comparisons(todo, t_start, args.budget_s, after=lambda: release(p, torch))

    # oracle on the host cores: the CPU baseline, and the definition's work counts per radius
    cpu, work = None, None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        est, _, threads, sample, work = cpu_baseline(scene, args)
        cpu = {"value": images / est[0], "unit": "images/s", "cores": threads, "kind": "oracle",
               "sample": sample}
    elif rank == 0:
        import oracle

        rng = np.random.default_rng(123)
        work = {}
        for R in RADII:
            og = rng.choice(scene.num_vertices, 8, replace=False)
            _, c = oracle.rici_fp64(scene.vertices, scene.normals, scene.triangles, og, R, N_RES,
                                    return_counters=True)
            work[R] = {k: v / len(og) for k, v in c.items()}

    pk, pk_kind = peaks()
    clk_mhz = (clk or {}).get("sm_mhz") or pk.get("sm_max_mhz", 2070.0)
    lane_peak = sms * 128 * clk_mhz * 1e6 / 1e9  # FP32 lane operations, G/s
    dp4a_peak = sms * DP4A_PER_SM_CLK * 4 * clk_mhz * 1e6 / 1e9  # int8 MACs via dp4a, G/s
    rooflines = {}
    if work is not None:
        for R in RADII:
            ops = generation_work(work[R]) * V
            rooflines[f"generation_R{R}"] = {
                "bound": "alu", "unit": "Gop/s",
                "achieved": ops / (pms[f"generation_R{R}"] / 1e3) / 1e9, "peak": lane_peak,
                "work": (f"{F_PROJ} FP32 ops x 3 vertices per contributing (origin, triangle) pair "
                         f"+ {F_LAYER + F_COL} per contributing (origin, triangle, layer) "
                         "crossing (segment within the largest circle), counted by the oracle "
                         f"on sampled origins: {work[R]['pairs_contributing']:.0f} pairs and "
                         f"{work[R]['crossings_contributing']:.0f} crossings per origin, x {V} "
                         "origins"),
                "traffic": TRAFFIC["k_generate_R0.6"] if R == 0.6 else None,
                "peak_kind": f"derived: {sms} SMs x 128 FP32 lanes x {clk_mhz:.0f} MHz "
                             "(median SM clock)"}
    if forms is not None:
        f = forms
        n8 = f["int8_tensor_core"]
        i8_pairs = f["comparisons"] - n8["counters"][1]  # pairs outside the int8 class: int64
        rooflines["search_int8_tensor_core"] = {
            "bound": "tensor", "unit": "G int8-MAC/s",
            "achieved": 3 * N_RES * N_RES * i8_pairs / (n8["ms"] / 1e3) / 1e9,
            "peak": mma_rate / 1e9,
            "work": f"{i8_pairs} int8-class pairs x 3 GEMM terms x {N_RES * N_RES} int8 MACs",
            "traffic": None,
            "peak_kind": "measured: mma.sync m16n8k32 s8 issue rate of the whole GPU"}
        dn = f["cuda_core_dense"]
        rooflines["search_cuda_core_dense"] = {
            "bound": "alu", "unit": "G int8-MAC/s",
            "achieved": MACS_PER_TERM * dn["counters"][0] * (N_RES - 1) / (dn["ms"] / 1e3) / 1e9,
            "peak": dp4a_peak,
            "work": f"{dn['counters'][0]} (pair, row) evaluations x {N_RES - 1} x "
                    f"{MACS_PER_TERM} int8 MACs",
            "traffic": None,
            "peak_kind": f"derived: {sms} SMs x {DP4A_PER_SM_CLK} dp4a per clock x 4 MACs x "
                         f"{clk_mhz:.0f} MHz; measured {dp4a_rate / sms / (clk_mhz * 1e6):.1f} "
                         "dp4a per SM per clock"}
    if "clutter_scene" in cmp and "skipped" not in cmp["clutter_scene"]:
        c = cmp["clutter_scene"]
        kt = 2 * N_RES * N_RES
        rooflines["search_tensor_core_clutter_scene"] = {
            "bound": "tensor", "unit": "TFLOP/s",
            "achieved": 2.0 * kt * c["comparisons"] / (c["tensor_core_search_ms"] / 1e3) / 1e12,
            "peak": pk.get("bf16_tflops", 1900.0),
            "work": f"{c['comparisons']} pairs x 2 x {kt} fp16 multiply-adds (dense, K = 2 N^2; "
                    "every image of the clutter scene is in the fp16 class)",
            "traffic": TRAFFIC["k_tc_rank_clutter"],
            "peak_kind": f"{pk_kind} bf16 dense burst (fp16 runs at the bf16 rate)"}
        rooflines["search_cuda_core_clutter_scene"] = {
            "bound": "alu", "unit": "G int8-MAC/s",
            "achieved": MACS_PER_TERM * c["pair_rows"] * (N_RES - 1) /
            (c["cuda_core_search_ms"] / 1e3) / 1e9,
            "peak": dp4a_peak,
            "work": f"{c['pair_rows']} (pair, row) evaluations x {N_RES - 1} x {MACS_PER_TERM} "
                    "int8 MACs",
            "traffic": TRAFFIC["k_dense_clutter"],
            "peak_kind": f"derived: {sms} SMs x {DP4A_PER_SM_CLK} dp4a per clock x 4 MACs x "
                         f"{clk_mhz:.0f} MHz (median SM clock)"}
    for r in rooflines.values():
        r["frac"] = r["achieved"] / r["peak"]
    gen_parts = {R: pms[f"generation_R{R}"] for R in RADII}
    dom_R = max(gen_parts, key=gen_parts.get)
    dominant = (f"generation_R{dom_R}" if gen_parts[dom_R] >= pms["search"] or
                f"generation_R{dom_R}" not in rooflines else None)
    roof = dict(rooflines[dominant]) if dominant in rooflines else None
    if roof is not None:
        roof["kernel"] = f"k_generate (R = {dom_R})"

    line = {
        "metric": METRIC, "value": value, "unit": "images/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f16+i32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "resolution": N_RES, "support_radii": list(RADII),
                   "triangles": T, "vertices": V, "needles": Q, "haystack": V, "comparisons": pairs,
                   "images_per_step": images, "seed": SEED, "search_mode": args.search_mode,
                   "input_sha256": input_digest(scene),
                   "l2": "inputs larger than L2; also flushed by a 512 MB device write before "
                         "every timed step",
                   "parallelism": f"replicas x{world}"},
        "breakdown": {
            **{f"{k}_ms": v for k, v in pms.items()},
            **{f"generation_R{R}_images_per_s": V / (pms[f'generation_R{R}'] / 1e3) for R in RADII},
            "search_comparisons_per_s": pairs / (pms["search"] / 1e3),
            "rank0_fraction": float((rk == 0).mean()),
            "generation_counters": {
                str(R): {"pairs_processed": c[0], "layer_items": c[1], "fp64_band_items": c[2],
                         "cull_candidates": c[3], "fp64_band_rate": c[2] / c[1] if c[1] else None}
                for R, c in gcnt.items()},
            "search_counters": {"dense_pair_rows": scnt[0], "int64_pairs": scnt[1],
                                "int64_terms": scnt[2], "dense_lane_slots": scnt[3]},
            "oracle_work_per_origin": work,
            "search_forms_on_step_images": forms,
            "tuning": {str(R): t for R, t in tunings.items()}, "autotune_s": tune_s,
            **cmp,
        },
        "roofline": roof,
        "rooflines": rooflines,
        "peaks": {"kind": pk_kind, "hbm_gbs": pk.get("hbm_gbs"),
                  "bf16_tflops": pk.get("bf16_tflops"),
                  "mma_s8_gmacs_measured": mma_rate / 1e9,
                  "dp4a_g_per_s_measured": dp4a_rate / 1e9},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "clocks": clk,
        "gpu_launches": launches,
        "status": st,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
