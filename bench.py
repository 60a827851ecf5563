#!/usr/bin/env python
"""Benchmark of the RICI hot path on one clutter scene (one JSON line on stdout).

Workload: a displaced-icosphere target (20,480 triangles) plus 9 clutter meshes of
5k-50k triangles in a box of side 2 (229,756 triangles, 114,892 vertices, seed 2).
One step is the whole hot path over that scene:
  1. RICI 64x64 images (R = 0.3) of the target's 10,242 vertices with the target alone
     (the needles),
  2. RICI images of all 114,892 scene vertices (the haystack),
  3. CUDA-core clutter-resistant search of every needle against every haystack image
     (1.18e9 comparisons): rank of its true match, true distance, top-1.
value = (needle + haystack images) / step time, whole job.  Inputs are resident in HBM and
L2 is flushed (512 MB write) before every timed step.  e2e repeats the step through the
same public API starting from pinned host buffers, with the host<->device copies timed.

--impl reference times the CPU oracle (FP64 brute force / int64 Listing 1) on bounded
samples of the same workload and extrapolates to the full step.
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
R_SUP = 0.3
SEED = 2
WORKLOAD = ("clutter scene: displaced icosphere target (subdivision 5, 20,480 triangles) + 9 "
            "clutter meshes (5k-50k triangles, displaced icospheres/tori), box side 2; RICI 64x64 "
            "uint16 at R=0.3 for the 10,242 target vertices (target alone) and all 114,892 scene "
            "vertices; CUDA-core CRSS search of every needle against every haystack image, ranks")

# FP32-pipe operations of the definition per unit of generation work: the projection of one
# vertex (Eqs. relativeLocation, firstRotation, secondRotation: 3 subtractions and 6 multiply-adds
# with their roundings, counted as 15 operations) for each vertex of an (origin, triangle) pair
# that crosses a layer, and per (origin, triangle, layer) crossing the slicing of two edges, the
# segment quantities |E0|^2, |E1|^2, E0.D, E1.D, E0 x D, |D|^2 and the interval boundaries of
# Section 3.1.2 (counted as 40 operations)
F_PROJ = 15
F_LAYER = 40
# int8 multiply-adds per masked squared difference in the expanded form m(a-b)^2 =
# a^2 - 2ab + (mb)^2 with sum a^2 per row precomputed: one for a*b and one for (mb)*(mb); dp4a
# performs four of them per instruction.
MACS_PER_TERM = 2
# dp4a instructions per SM per clock: half the 128 FP32 lanes (a microbenchmark of independent
# dp4a chains measured 61.3 per SM per clock at 2070 MHz; FFMA measured 117.3)
DP4A_PER_SM_CLK = 64
# DRAM bytes (read + write) per launch from one-pass ncu captures (dram__bytes_read and
# dram__bytes_write; commands in profiles/) of the current kernels at the full clutter-scene
# size: k_dense (the search) and k_generate (the haystack images; its traffic is the 8 KB image
# of each origin plus a small read of triangle records, so it is the same for every launch
# tuning).  Set to None when a kernel changes until it is captured again.
TRAFFIC_DENSE_FULL = 1.90e9 + 5.01e6
TRAFFIC_GEN_FULL = 63.63e6 + 901.22e6


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--search-mode", type=int, default=1)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default launch tuning instead of autotuning the generation")
    ap.add_argument("--cpu-origins", type=int, default=96)
    ap.add_argument("--cpu-needle-origins", type=int, default=48)
    ap.add_argument("--cpu-needles", type=int, default=12)
    ap.add_argument("--cpu-haystack", type=int, default=24000)
    ap.add_argument("--tc-compare", type=int, default=1,
                    help="also time the tensor-core search on the same images (breakdown)")
    ap.add_argument("--sparse-compare", type=int, default=1,
                    help="also time the sparse-needle CUDA-core search on the same images")
    ap.add_argument("--precision-compare", type=int, default=1,
                    help="also time the three search forms on a precision-form image set sample")
    ap.add_argument("--spin-compare", type=int, default=1,
                    help="also time spin-image generation (Section 2.1) for the haystack points")
    ap.add_argument("--clutterbox-compare", type=int, default=1,
                    help="also time a synthetic clutterbox experiment (Section 4.1) on the GPU path")
    ap.add_argument("--batched-compare", type=int, default=1,
                    help="also time the batched multi-scene run (CUDA graph) against per-scene calls")
    ap.add_argument("--haystack-limit", type=int, default=0,
                    help="image only the first H scene vertices (small profiling case)")
    ap.add_argument("--needle-limit", type=int, default=0,
                    help="use only the first Q target vertices as needles (small profiling case)")
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


def build_workload():
    import synth

    return synth.clutter_scene(seed=SEED)


def cpu_baseline(scene, args, steps: int = 1):
    """Oracle on bounded samples of the step; returns per-step extrapolated seconds and info."""
    import oracle
    import synth

    oracle.build()
    rng = np.random.default_rng(123)
    V, Vt = scene.num_vertices, scene.target_vertices
    tgt = scene.target_only()
    og = rng.choice(V, args.cpu_origins, replace=False)
    on = rng.choice(Vt, args.cpu_needle_origins, replace=False)
    ims_rng = np.random.default_rng(7)
    nd = synth.images.rici_like_images(ims_rng, args.cpu_needles, N_RES)
    hay = synth.images.rici_like_images(ims_rng, args.cpu_haystack, N_RES)
    threads = oracle.max_threads()
    est = []
    for _ in range(steps):
        t0 = time.perf_counter()
        oracle.rici_fp64(scene.vertices, scene.normals, scene.triangles, og, R_SUP, N_RES)
        t1 = time.perf_counter()
        oracle.rici_fp64(tgt.vertices, tgt.normals, tgt.triangles, on, R_SUP, N_RES)
        t2 = time.perf_counter()
        oracle.crss_search(nd, hay, np.zeros(len(nd), np.int64))
        t3 = time.perf_counter()
        per_o = (t1 - t0) / len(og)
        per_n = (t2 - t1) / len(on)
        per_pair = (t3 - t2) / (len(nd) * len(hay))
        est.append(per_o * V + per_n * Vt + per_pair * Vt * V)
    sample = (f"{len(og)} scene-vertex images + {len(on)} target-alone images (FP64 brute force "
              f"over all triangles) and {len(nd)} needles x {len(hay)} haystack images (int64 "
              f"Listing 1) per step, extrapolated to {Vt + V} images and {Vt * V} comparisons")
    return est, threads, sample


def precision_form_comparison(p, torch, dev, stream, Q=16384, H=262144, seed=31, steps=3):
    """The three exact search forms on a sample of the precision-form image set (heavy-tailed
    RICI-like rows, needles copied before clutter is added to 30 % of the haystack)."""
    import synth

    nd, hay, m = synth.images.needle_haystack_set_torch(seed, Q, H, N_RES, dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    out = {"recipe": f"synth.images.needle_haystack_set_torch(seed={seed}), {Q} needles x {H} "
                     f"haystack images, N = {N_RES}", "comparisons": Q * H}
    ref = None
    for name, mode in (("tensor_core", p.SEARCH_TENSOR), ("cuda_core", p.SEARCH_CUDA_CORE),
                       ("sparse_needle", p.SEARCH_SPARSE)):
        r = p.crss_search(nd, hay, m, mode=mode)
        torch.cuda.synchronize()
        ts = []
        for _ in range(steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r = p.crss_search(nd, hay, m, mode=mode)
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        same = None if ref is None else all(bool(torch.equal(r[k], ref[k]))
                                            for k in ("rank", "true_distance", "top1"))
        if ref is None:
            ref = r
        t = statistics.mean(ts)
        out[name] = {"ms": t, "comparisons_per_s": Q * H / (t / 1e3),
                     "same_ranks_as_tensor_core": same}
    out["status"] = p.sync_status()
    del nd, hay, m, ref, r, flush
    torch.cuda.empty_cache()
    return out


def clutterbox_experiment(p, torch, dev, stream, runs=4, n=10, seed=51, tri_lo=2000,
                          tri_hi=20000, steps=3):
    """Synthetic clutterbox runs (Section 4.1): every level of every run imaged by one batched
    generation call and searched by one batched search call (tensor-core form)."""
    import synth
    from paper_2007_02306_gb300 import clutterbox

    levels = [synth.scenes.clutterbox(seed + r, n=n, box_side=3.0, tri_lo=tri_lo, tri_hi=tri_hi)
              for r in range(runs)]
    prep = clutterbox.prepare(levels, dev)
    clutterbox.run_prepared(prep, R_SUP, N_RES)
    torch.cuda.synchronize()
    ts = []
    for _ in range(steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res = clutterbox.run_prepared(prep, R_SUP, N_RES)
        e1.record(stream)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    # Eq. clutter around every reference vertex of every level (clutter-versus-rank heatmap)
    areas = clutterbox.clutter_prepared(prep, R_SUP)
    torch.cuda.synchronize()
    tc = []
    for _ in range(steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        areas = clutterbox.clutter_prepared(prep, R_SUP)
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
                     f"objects of {tri_lo}-{tri_hi} triangles), N = {N_RES}, R = {R_SUP}"}
    del prep, res, areas
    torch.cuda.empty_cache()
    return out


def batched_comparison(p, torch, dev, stream, args, n_scenes=24, needles=256, seed=41,
                       tri_lo=2000, tri_hi=60_000, total_lo=10_000, total_hi=300_000):
    """Batched run of many uneven scenes (one set of launches, replayed from a CUDA graph)
    against one plain generate/generate/search call sequence per scene."""
    import synth

    scenes = synth.scene_batch(seed=seed, n_scenes=n_scenes, tri_lo=tri_lo, tri_hi=tri_hi,
                               total_lo=total_lo, total_hi=total_hi)
    rng = np.random.default_rng(2)
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
    xs = []
    for s in scenes:
        q = min(needles, s.target_vertices)
        on = np.sort(rng.choice(s.target_vertices, q, replace=False)).astype(np.int32)
        xs.append({"V": d(s.vertices), "Nrm": d(s.normals), "T": d(s.triangles),
                   "Tt": d(s.triangles[: s.target_triangles]), "on": d(on),
                   "oh": d(np.arange(s.num_vertices, dtype=np.int32)), "m": d(on.astype(np.int64))})
    gen = []
    for x in xs:
        gen.append({"vertices": x["V"], "normals": x["Nrm"], "triangles": x["Tt"], "origins": x["on"]})
        gen.append({"vertices": x["V"], "normals": x["Nrm"], "triangles": x["T"], "origins": x["oh"]})
    outs = [torch.empty((g["origins"].numel(), N_RES, N_RES), dtype=torch.uint16, device=dev)
            for g in gen]
    for g, o in zip(gen, outs):
        g["out"] = o
    srch = [{"needles": outs[2 * i], "haystack": outs[2 * i + 1], "true_match": x["m"]}
            for i, x in enumerate(xs)]
    res = [{"rank": torch.empty(x["on"].numel(), dtype=torch.int32, device=dev),
            "true_distance": torch.empty(x["on"].numel(), dtype=torch.int64, device=dev),
            "top1": torch.empty(x["on"].numel(), dtype=torch.int32, device=dev)} for x in xs]
    wg = torch.empty(p.binding.generate_batch_workspace_bytes(gen, N_RES) + 512, dtype=torch.uint8,
                     device=dev)
    wsr = torch.empty(p.binding.search_batch_workspace_bytes(srch, N_RES) + 512, dtype=torch.uint8,
                      device=dev)
    wg = wg[(-wg.data_ptr()) % 256:]
    wsr = wsr[(-wsr.data_ptr()) % 256:]

    def run_batched():
        p.rici_generate_batch(gen, R_SUP, N_RES, workspace_tensor=wg)
        p.crss_search_batch(srch, N_RES, workspace_tensor=wsr, outputs=res)

    def run_plain():
        for x, g0, g1 in zip(xs, gen[0::2], gen[1::2]):
            p.rici_generate(x["V"], x["Nrm"], x["Tt"], x["on"], R_SUP, N_RES, out=g0["out"])
            p.rici_generate(x["V"], x["Nrm"], x["T"], x["oh"], R_SUP, N_RES, out=g1["out"])
            p.crss_search(g0["out"], g1["out"], x["m"], mode=p.SEARCH_TENSOR)

    def capture():
        cs = torch.cuda.Stream(device=dev)
        cs.wait_stream(stream)
        with torch.cuda.stream(cs):
            run_batched()
        stream.wait_stream(cs)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            run_batched()
        return g

    # a graph replays the launch shapes in force when it was captured: one with the default
    # tuning, one with the autotuned tuning (measured on the first scenes, fresh cache)
    from paper_2007_02306_gb300 import autotune

    prev_tuning = p.get_tuning()
    p.set_tuning(None)
    graph_default = capture()
    t_tune = time.time()
    with tempfile.TemporaryDirectory() as td:
        tuning = autotune.tune_batch(gen, srch, R_SUP, N_RES, gpu_name=torch.cuda.get_device_name(dev),
                                     sample=4, path=os.path.join(td, "tuning.json"))
    t_tune = time.time() - t_tune
    graph = capture()
    for _ in range(2):
        graph.replay()
        run_plain()
        graph_default.replay()
    torch.cuda.synchronize()
    reps = max(3, args.steps)
    t_b, t_p, t_d = [], [], []
    for _ in range(reps):
        e0, e1, e2, e3 = (torch.cuda.Event(enable_timing=True) for _ in range(4))
        e0.record(stream)
        graph.replay()
        e1.record(stream)
        run_plain()
        e2.record(stream)
        graph_default.replay()
        e3.record(stream)
        torch.cuda.synchronize()
        t_b.append(e0.elapsed_time(e1))
        t_p.append(e1.elapsed_time(e2))
        t_d.append(e2.elapsed_time(e3))
    st = p.sync_status()
    p.set_tuning(prev_tuning)
    images = sum(g["origins"].numel() for g in gen)
    pairs = sum(x["on"].numel() * x["oh"].numel() for x in xs)
    return {"scenes": n_scenes, "triangles": int(sum(s.num_triangles for s in scenes)),
            "images": int(images), "comparisons": int(pairs),
            "batched_graph_ms": statistics.mean(t_b), "per_scene_calls_ms": statistics.mean(t_p),
            "speedup": statistics.mean(t_p) / statistics.mean(t_b),
            "batched_graph_default_tuning_ms": statistics.mean(t_d),
            "autotuned": tuning, "autotune_s": t_tune,
            "batched_images_per_s": images / (statistics.mean(t_b) / 1e3), "status": st,
            "recipe": f"synth.scene_batch(seed={seed}, {n_scenes} scenes, {total_lo}-{total_hi} "
                      f"triangles each), {needles} needles per scene (target alone) vs all scene "
                      "vertices, tensor-core search"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    scene = build_workload()
    cpu_baseline(scene, args, steps=max(0, args.warmup))
    est, threads, sample = cpu_baseline(scene, args, steps=args.steps)
    images = scene.num_vertices + scene.target_vertices
    sec = statistics.mean(est)
    value = images / sec
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "images/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": sec * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64+i64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "resolution": N_RES, "support_radius": R_SUP,
                   "seed": SEED},
        "cpu_baseline": {"value": value, "unit": "images/s", "cores": threads, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "images/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
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
    V, T, Vt, Tt = scene.num_vertices, scene.num_triangles, scene.target_vertices, scene.target_triangles
    if args.needle_limit:
        Vt = min(Vt, args.needle_limit)
    if args.haystack_limit:
        V = max(Vt, min(V, args.haystack_limit))
    h_vert = torch.from_numpy(scene.vertices).pin_memory()
    h_norm = torch.from_numpy(scene.normals).pin_memory()
    h_tri = torch.from_numpy(scene.triangles).pin_memory()
    h_oh = torch.arange(V, dtype=torch.int32).pin_memory()
    h_on = torch.arange(Vt, dtype=torch.int32).pin_memory()
    h_match = torch.arange(Vt, dtype=torch.int64).pin_memory()

    vert, norm, tri = h_vert.to(dev), h_norm.to(dev), h_tri.to(dev)
    if args.needle_limit or args.haystack_limit:
        args.no_cpu_baseline = True
    tri_t = tri[:Tt]
    oh, on, match = h_oh.to(dev), h_on.to(dev), h_match.to(dev)
    needles = torch.empty((Vt, N_RES, N_RES), dtype=torch.uint16, device=dev)
    hay = torch.empty((V, N_RES, N_RES), dtype=torch.uint16, device=dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        p.rici_generate(vert, norm, tri_t, on, R_SUP, N_RES, out=needles)
        p.rici_generate(vert, norm, tri, oh, R_SUP, N_RES, out=hay)
        return p.crss_search(needles, hay, match, mode=args.search_mode)

    # launch tuning of the generation kernels, measured on this workload (fresh cache)
    tune_s = 0.0
    if not args.no_autotune:
        from paper_2007_02306_gb300 import autotune

        t0 = time.time()
        with tempfile.TemporaryDirectory() as td:
            autotune.tune_batch(
                [{"vertices": vert, "normals": norm, "triangles": tri_t, "origins": on, "out": needles},
                 {"vertices": vert, "normals": norm, "triangles": tri, "origins": oh, "out": hay}],
                [], R_SUP, N_RES, gpu_name=torch.cuda.get_device_name(dev), sample=2, repeats=2,
                path=os.path.join(td, "tuning.json"))
        tune_s = time.time() - t0
    step_tuning = p.get_tuning()

    for _ in range(args.warmup):
        step()
    st = p.sync_status()
    if st != 0:
        raise RuntimeError(f"device status {st} during warm-up")

    # untimed: work counters for the roofline
    gcnt = torch.zeros(4, dtype=torch.int64, device=dev)
    scnt = torch.zeros(4, dtype=torch.int64, device=dev)
    p.rici_generate(vert, norm, tri, oh, R_SUP, N_RES, out=hay, counters=gcnt)
    p.crss_search(needles, hay, match, mode=args.search_mode, counters=scnt)
    torch.cuda.synchronize()
    gcnt, scnt = gcnt.cpu().tolist(), scnt.cpu().tolist()

    clocks = ClockSampler(dev.index if world == 1 else local)
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    launches0 = p.binding.kernel_launches()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    for k in range(args.steps):
        flush.zero_()
        e = ev[k]
        e[0].record(stream)
        p.rici_generate(vert, norm, tri_t, on, R_SUP, N_RES, out=needles)
        e[1].record(stream)
        p.rici_generate(vert, norm, tri, oh, R_SUP, N_RES, out=hay)
        e[2].record(stream)
        res = p.crss_search(needles, hay, match, mode=args.search_mode)
        e[3].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    launches = p.binding.kernel_launches() - launches0
    if world > 1:
        torch.distributed.barrier()
    st = p.sync_status()
    if st != 0:
        raise RuntimeError(f"device status {st} in the timed region")
    t_nd = [ev[k][0].elapsed_time(ev[k][1]) for k in range(args.steps)]
    t_hy = [ev[k][1].elapsed_time(ev[k][2]) for k in range(args.steps)]
    t_se = [ev[k][2].elapsed_time(ev[k][3]) for k in range(args.steps)]
    ms = [a + b + c for a, b, c in zip(t_nd, t_hy, t_se)]
    ms_step = max_over_ranks(statistics.mean(ms), dev)
    images = V + Vt
    pairs = V * Vt
    value = job_rate(images, ms_step, world)

    # tensor-core form of the same search (exact fp16 tcgen05 GEMM), timed separately
    tc = None
    if args.tc_compare:
        for _ in range(2):
            p.crss_search(needles, hay, match, mode=p.SEARCH_TENSOR)
        torch.cuda.synchronize()
        tc_ms = []
        for k in range(args.steps):
            flush.zero_()
            b0 = torch.cuda.Event(enable_timing=True)
            b1 = torch.cuda.Event(enable_timing=True)
            b0.record(stream)
            rt = p.crss_search(needles, hay, match, mode=p.SEARCH_TENSOR)
            b1.record(stream)
            torch.cuda.synchronize()
            tc_ms.append(b0.elapsed_time(b1))
        same = all(bool(torch.equal(rt[k2], res[k2])) for k2 in ("rank", "true_distance", "top1"))
        st = p.sync_status()
        tc = {"ms": statistics.mean(tc_ms), "comparisons_per_s": pairs / (statistics.mean(tc_ms) / 1e3),
              "same_ranks_as_cuda_core": same, "status": st}

    # sparse-needle form of the same search (CUDA cores, the needles' non-zero words only)
    sp = None
    if args.sparse_compare:
        for _ in range(2):
            p.crss_search(needles, hay, match, mode=p.SEARCH_SPARSE)
        torch.cuda.synchronize()
        sp_ms = []
        for k in range(args.steps):
            flush.zero_()
            b0 = torch.cuda.Event(enable_timing=True)
            b1 = torch.cuda.Event(enable_timing=True)
            b0.record(stream)
            rs = p.crss_search(needles, hay, match, mode=p.SEARCH_SPARSE)
            b1.record(stream)
            torch.cuda.synchronize()
            sp_ms.append(b0.elapsed_time(b1))
        same = all(bool(torch.equal(rs[k2], res[k2])) for k2 in ("rank", "true_distance", "top1"))
        spc = torch.zeros(4, dtype=torch.int64, device=dev)
        p.crss_search(needles, hay, match, mode=p.SEARCH_SPARSE, counters=spc)
        spc = [int(x) for x in spc.cpu()]
        st = p.sync_status()
        sp = {"ms": statistics.mean(sp_ms),
              "comparisons_per_s": pairs / (statistics.mean(sp_ms) / 1e3),
              "same_ranks_as_cuda_core": same, "status": st,
              "pair_words": spc[0], "lane_slots": spc[3],
              "lane_utilisation": spc[0] / spc[3] if spc[3] else None}
    precision = None
    if args.precision_compare and rank == 0:
        precision = precision_form_comparison(p, torch, dev, stream)

    spin = None
    if args.spin_compare:
        # spin images of every haystack point from 9 samples per triangle (the paper used 10)
        si = torch.empty((V, N_RES, N_RES), dtype=torch.float32, device=dev)
        for _ in range(2):
            p.spin_images(vert, norm, tri, oh, R_SUP, N_RES, 3, out=si)
        torch.cuda.synchronize()
        sm = []
        for _ in range(args.steps):
            flush.zero_()
            s0 = torch.cuda.Event(enable_timing=True)
            s1 = torch.cuda.Event(enable_timing=True)
            s0.record(stream)
            p.spin_images(vert, norm, tri, oh, R_SUP, N_RES, 3, out=si)
            s1.record(stream)
            torch.cuda.synchronize()
            sm.append(s0.elapsed_time(s1))
        spin = {"images": V, "samples_per_triangle": 9, "ms": statistics.mean(sm),
                "images_per_s": V / (statistics.mean(sm) / 1e3),
                "rici_haystack_generation_ms": statistics.mean(t_hy), "status": p.sync_status()}
        del si

    cbox = None
    if args.clutterbox_compare and rank == 0:
        cbox = clutterbox_experiment(p, torch, dev, stream)
        # Eq. clutter around every needle's vertex of the step's scene (object = the target)
        for _ in range(2):
            p.clutter_areas(vert, norm, tri, on, R_SUP, Vt)
        torch.cuda.synchronize()
        cm = []
        for _ in range(args.steps):
            c0 = torch.cuda.Event(enable_timing=True)
            c1 = torch.cuda.Event(enable_timing=True)
            c0.record(stream)
            ca, co = p.clutter_areas(vert, norm, tri, on, R_SUP, Vt)
            c1.record(stream)
            torch.cuda.synchronize()
            cm.append(c0.elapsed_time(c1))
        cf = ((ca - co) / ca).cpu().numpy()
        cbox["clutter_scene_measure"] = {
            "points": Vt, "triangles": T, "ms": statistics.mean(cm),
            "points_per_s": Vt / (statistics.mean(cm) / 1e3),
            "clutter_mean": float(cf.mean()), "clutter_quartiles": [
                float(x) for x in np.quantile(cf, [0.25, 0.5, 0.75])],
            "status": p.sync_status()}

    batched = batched_small = None
    if args.batched_compare and rank == 0:
        batched = batched_comparison(p, torch, dev, stream, args)
        # many small scenes: where one set of launches per batch matters most
        batched_small = batched_comparison(p, torch, dev, stream, args, n_scenes=256, needles=64,
                                           seed=42, tri_lo=500, tri_hi=5000, total_lo=2000,
                                           total_hi=12_000)

    # e2e: same step from pinned host buffers, host<->device copies inside the timed region
    e2e = None
    if not args.no_e2e:
        h_rank = torch.empty(Vt, dtype=torch.int32).pin_memory()
        h_top1 = torch.empty(Vt, dtype=torch.int32).pin_memory()
        h_dt = torch.empty(Vt, dtype=torch.int64).pin_memory()
        e2e_ms = []
        for k in range(args.steps + 1):
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
            p.rici_generate(dv, dn, dtri[:Tt], don, R_SUP, N_RES, out=needles)
            p.rici_generate(dv, dn, dtri, doh, R_SUP, N_RES, out=hay)
            r = p.crss_search(needles, hay, dm, mode=args.search_mode)
            h_rank.copy_(r["rank"], non_blocking=True)
            h_top1.copy_(r["top1"], non_blocking=True)
            h_dt.copy_(r["true_distance"], non_blocking=True)
            a1.record(stream)
            torch.cuda.synchronize()
            if k > 0:  # first pass warms the copy path
                e2e_ms.append(a0.elapsed_time(a1))
        e_ms = max_over_ranks(statistics.mean(e2e_ms), dev)
        h2d = sum(x.numel() * x.element_size() for x in (h_vert, h_norm, h_tri, h_oh, h_on, h_match))
        d2h = Vt * (4 + 4 + 8)
        e2e = {"value": job_rate(images, e_ms, world), "unit": "images/s",
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": e_ms}

    pk, pk_kind = peaks()
    clk_mhz = (clk or {}).get("sm_mhz") or pk.get("sm_max_mhz", 2070.0)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    alu_peak_gops = sms * 128 * clk_mhz * 1e6 / 1e9  # 32-bit lane operations per second
    mac_peak_gops = sms * DP4A_PER_SM_CLK * 4 * clk_mhz * 1e6 / 1e9  # int8 MACs via dp4a
    dp4a_rate = p.binding.measure_dp4a_rate()  # after the timed regions

    gen_ms = statistics.mean(t_hy)
    se_ms = statistics.mean(t_se)
    cpu = None
    cpu_ops = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        est, threads, sample = cpu_baseline(scene, args)
        cpu = {"value": images / est[0], "unit": "images/s", "cores": threads, "kind": "oracle",
               "sample": sample}
        import oracle

        rng = np.random.default_rng(5)
        og = rng.choice(V, 32, replace=False)
        _, cc = oracle.rici_fp64(scene.vertices, scene.normals, scene.triangles, og, R_SUP, N_RES,
                                 return_counters=True)
        cpu_ops = cc
    # roofline of the dominant kernel (the larger of haystack generation and search)
    rooflines = {}
    search_terms = scnt[0] * (N_RES - 1)
    rooflines["search"] = {
        "bound": "alu", "unit": "G int8-MAC/s",
        "achieved": MACS_PER_TERM * search_terms / (se_ms / 1e3) / 1e9,
        "peak": mac_peak_gops,
        "work": f"{scnt[0]} (pair, row) evaluations x {N_RES - 1} masked squared differences x "
                f"{MACS_PER_TERM} int8 multiply-adds",
        "traffic": (TRAFFIC_DENSE_FULL if not (args.haystack_limit or args.needle_limit)
                    else None),
        "peak_kind": f"derived: {sms} SMs x {DP4A_PER_SM_CLK} dp4a per clock x 4 MACs x "
                     f"{clk_mhz:.0f} MHz (median SM clock)",
        "measured_dp4a_per_sm_per_clk": dp4a_rate / sms / (clk_mhz * 1e6),
    }
    if cpu_ops is not None:
        per_o = (F_PROJ * 3 * cpu_ops["pairs_crossing"] + F_LAYER * cpu_ops["layer_crossings"]) / 32
        rooflines["generation"] = {
            "bound": "alu", "unit": "Gop/s",
            "achieved": per_o * V / (gen_ms / 1e3) / 1e9, "peak": alu_peak_gops,
            "work": f"{F_PROJ} ops x 3 vertices per crossing (origin, triangle) pair + {F_LAYER} "
                    "ops per (origin, triangle, layer) crossing, counted by the oracle on 32 "
                    "sampled origins and scaled to all haystack origins",
            "traffic": (TRAFFIC_GEN_FULL if not (args.haystack_limit or args.needle_limit)
                        else None),
        }
    for r in rooflines.values():
        r["frac"] = r["achieved"] / r["peak"]
        r.setdefault("peak_kind", f"derived: {sms} SMs x 128 lanes x {clk_mhz:.0f} MHz "
                                  "(median SM clock)")
    if tc is not None:
        kt = 2 * N_RES * N_RES
        rooflines["search_tensor_core"] = {
            "bound": "tensor", "unit": "TFLOP/s",
            "achieved": 2.0 * kt * pairs / (tc["ms"] / 1e3) / 1e12,
            "peak": pk.get("bf16_tflops", 1900.0),
            "work": f"{pairs} pairs x 2 x {kt} fp16 multiply-adds (dense, K = 2 N^2)",
            "traffic": None, "peak_kind": f"{pk_kind} bf16 dense burst (fp16 runs at the bf16 rate)",
        }
        rooflines["search_tensor_core"]["frac"] = (rooflines["search_tensor_core"]["achieved"] /
                                                   rooflines["search_tensor_core"]["peak"])
    if sp is not None:
        rooflines["search_sparse"] = {
            "bound": "alu", "unit": "G int8-MAC/s",
            "achieved": sp["pair_words"] * 4 * MACS_PER_TERM / (sp["ms"] / 1e3) / 1e9,
            "peak": rooflines["search"]["peak"],
            "work": f"{sp['pair_words']} (pair, needle word) evaluations x 4 masked squared "
                    "differences x 2 int8 multiply-adds",
            "traffic": None, "peak_kind": rooflines["search"]["peak_kind"],
        }
        rooflines["search_sparse"]["frac"] = (rooflines["search_sparse"]["achieved"] /
                                              rooflines["search_sparse"]["peak"])
    dom = "search" if se_ms >= gen_ms or "generation" not in rooflines else "generation"
    roof = dict(rooflines[dom])
    roof["kernel"] = "k_dense (CUDA-core CRSS)" if dom == "search" else "k_generate"

    line = {
        "metric": METRIC, "value": value, "unit": "images/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+i32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "resolution": N_RES, "support_radius": R_SUP,
                   "triangles": T, "needles": Vt, "haystack": V, "comparisons": pairs, "seed": SEED,
                   "search_mode": args.search_mode,
                   "input_sha256": input_digest(scene),
                   "l2": "flushed by a 512 MB device write before every timed step",
                   "parallelism": f"replicas x{world}"},
        "breakdown": {
            "needle_generation_ms": statistics.mean(t_nd),
            "haystack_generation_ms": gen_ms,
            "search_ms": se_ms,
            "generation_images_per_s": images / ((statistics.mean(t_nd) + gen_ms) / 1e3),
            "search_comparisons_per_s": pairs / (se_ms / 1e3),
            "generation_counters": {"triangles_processed": gcnt[0], "layer_items": gcnt[1],
                                    "fp64_band_items": gcnt[2], "cull_candidates": gcnt[3],
                                    "fp64_band_rate": gcnt[2] / gcnt[1] if gcnt[1] else None},
            "search_counters": {"pair_rows": scnt[0], "wide_pairs": scnt[1],
                                "wide_terms": scnt[2], "lane_slots": scnt[3],
                                "lane_utilisation": scnt[0] / scnt[3] if scnt[3] else None},
            "search_tensor_core": tc,
            "search_sparse_needle": sp,
            "precision_form_sample": precision,
            "clutterbox": cbox,
            "spin_images": spin,
            "batched_run": batched,
            "batched_run_small_scenes": batched_small,
            "tuning": step_tuning,
            "autotune_s": tune_s,
        },
        "roofline": roof,
        "rooflines": rooflines,
        "peaks": {"kind": pk_kind, "hbm_gbs": pk.get("hbm_gbs")},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "clocks": clk,
        "gpu_launches": launches,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
