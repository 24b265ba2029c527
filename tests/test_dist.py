"""The multi-rank plumbing of bench.py on CPU (gloo, world size 2): the timing barrier and the
max-over-ranks reduction, with no collective on the data path."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench.barrier(world)
        # each rank reports its own elapsed time; every rank must receive the maximum
        t = bench.max_over_ranks(1.0 + rank, world)
        out[rank] = t
        # whole-job throughput: units of all ranks over the slowest rank's time
        units = world * 10
        out[world + rank] = units / t
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_weak_scaling_value():
    world = 2
    ctx = mp.get_context("spawn")
    out = ctx.Array("d", 2 * world)
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert list(out[:world]) == [2.0, 2.0]
    assert list(out[world:]) == [10.0, 10.0]


def _reference_worker(rank, world, port, path):
    import contextlib
    import sys
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.argv = ["bench.py", "--impl", "reference", "--gpus", str(world), "--steps", "1", "--warmup", "1"]
    import bench
    with open(f"{path}.{rank}", "w") as f, contextlib.redirect_stdout(f):
        bench.main()


def test_reference_arm_under_two_ranks(tmp_path):
    """`bench.py --impl reference` launched as two ranks (gloo, as torchrun would): rank 0 alone
    times the oracle and prints one JSON line for the whole job; rank 1 exits without work."""
    import json
    world = 2
    ctx = mp.get_context("spawn")
    port = _free_port()
    path = str(tmp_path / "out")
    procs = [ctx.Process(target=_reference_worker, args=(r, world, port, path)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(600)
        assert p.exitcode == 0
    lines = [ln for ln in open(f"{path}.0").read().splitlines() if ln.startswith("{")]
    assert len(lines) == 1 and open(f"{path}.1").read().strip() == ""
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == world and d["steps"] == 1 and d["warmup"] == 1
    assert d["value"] > 0 and d["unit"] == "target-evals/s" and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
