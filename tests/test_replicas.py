"""The N > 1 path of the benchmark on the CPU: two gloo ranks run the replica helpers of bench.py.

Under torchrun every rank solves its own problems of the same recipe (seeds offset by rank), the ranks meet
only at barriers and in one MAX reduction of the timings, and rank 0 prints. This checks those pieces with
a real two-process group (gloo, 127.0.0.1), without a GPU.
"""
import json
import os
import socket
import tempfile

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, loc = bench.replica_env()
        top = bench.max_over_ranks(10.0 + 5.0 * rank, dist, "cpu")
        low = -bench.max_over_ranks(-(10.0 + 5.0 * rank), dist, "cpu")
        cases, ps = bench.batched_cases(3, r)
        dist.barrier()
        with open(os.path.join(out_dir, f"{rank}.json"), "w") as f:
            json.dump({"world": w, "rank": r, "local": loc, "max": top, "min": low,
                       "seed": bench.replica_seed(1, r), "orders": [c.n for c in cases], "ps": ps,
                       "first": float(cases[0].A[0, 0])}, f)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_run_independent_replicas():
    with tempfile.TemporaryDirectory() as d:
        mp.spawn(_rank_main, args=(2, _free_port(), d), nprocs=2, join=True)
        r0, r1 = (json.load(open(os.path.join(d, f"{k}.json"))) for k in (0, 1))
    assert (r0["world"], r0["rank"], r0["local"]) == (2, 0, 0) and (r1["world"], r1["rank"], r1["local"]) == (2, 1, 1)
    # The timing every rank reports is the slowest rank's.
    assert r0["max"] == r1["max"] == 15.0 and r0["min"] == r1["min"] == 10.0
    # Independent inputs per replica; rank 0's are the single-GPU benchmark's.
    assert r0["seed"] != r1["seed"]
    assert (r0["orders"], r0["first"]) != (r1["orders"], r1["first"])
    import bench
    cases, ps = bench.batched_cases(3)
    assert r0["orders"] == [c.n for c in cases] and r0["ps"] == ps
    assert r0["first"] == float(cases[0].A[0, 0])


def test_max_over_ranks_without_a_group():
    import bench
    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5
    assert bench.max_over_ranks(3.5, dist, "cpu") == 3.5  # no process group initialised
    assert np.isfinite(bench.replica_seed(7, 3)) and bench.replica_seed(7, 0) == 7
