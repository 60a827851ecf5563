"""The benchmark's multi-rank host logic on two CPU ranks (gloo, no GPU).

Under torchrun every rank runs one replica of the step and the job's step time is the slowest
rank's; the whole-job rate is world x units per rank / that time.  Two spawned gloo ranks with
different times must both see the maximum, and the rate must follow from it.  The scene digest
the benchmark records must depend on the seed only.
"""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def rank_main(rank, world, port, out_dir):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        assert bench.dist_env() == (rank, world, rank)
        mine = 100.0 + 25.0 * rank  # rank 1 is the slow one
        ms = bench.max_over_ranks(mine, "cpu")
        rate = bench.job_rate(1000.0, ms, world)
        with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as f:
            f.write(f"{ms} {rate}")
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_time(tmp_path):
    import torch.multiprocessing as mp

    world = 2
    mp.start_processes(rank_main, args=(world, free_port(), str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    for r in range(world):
        ms, rate = map(float, (tmp_path / f"rank{r}.txt").read_text().split())
        assert ms == pytest.approx(125.0)
        assert rate == pytest.approx(2 * 1000.0 / 0.125)


def test_single_process_passes_values_through():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(3.5, "cpu") == 3.5
    assert bench.job_rate(500.0, 250.0, 1) == pytest.approx(2000.0)


def test_input_digest_is_deterministic():
    sys.path.insert(0, ROOT)
    import bench
    import synth

    a = bench.input_digest(synth.tiny_scene(seed=1))
    assert a == bench.input_digest(synth.tiny_scene(seed=1))
    assert a != bench.input_digest(synth.tiny_scene(seed=2))
    assert len(a) == 16


def test_comparisons_stop_starting_once_the_budget_is_spent():
    sys.path.insert(0, ROOT)
    import bench

    now = [0.0]
    ran = []

    def work(name, seconds):
        def run():
            ran.append(name)
            now[0] += seconds
            return {"ms": seconds * 1e3}
        return run

    todo = [("a", 1, work("a", 50)), ("off", 0, work("off", 1)), ("b", 1, work("b", 80)),
            ("c", 1, work("c", 5)), ("d", 1, work("d", 5))]
    after = []
    out = bench.run_comparisons(todo, 0.0, 100.0, after=lambda: after.append(1),
                                clock=lambda: now[0])
    # a starts at 0 and b at 50 (inside the budget); c would start at 130 and d as well
    assert ran == ["a", "b"] and len(after) == 2
    assert out["a"] == {"ms": 50e3} and out["b"] == {"ms": 80e3}
    assert "skipped" in out["c"] and "skipped" in out["d"] and "off" not in out
