"""The multi-rank plumbing of bench.py on CPU (gloo, world size 2): the timing barrier, the
max-over-ranks reduction, the split of the targets into Morton-order slices (one per GPU, no
collective on the data path) and the one gather that restores the target order."""
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


def test_target_shards_partition_in_morton_order():
    """The N > 1 split of bench.py: the slices are disjoint, cover every target once, differ in size
    by at most one, and are contiguous runs of the targets' Morton order."""
    import numpy as np

    import bench
    rng = np.random.default_rng(0)
    y = rng.uniform(-1.2, 1.2, (10007, 3))
    keys = bench.morton_keys(y, 1 / 16)
    for world in (1, 2, 3, 8):
        sl = bench.shard_indices(y, 1 / 16, world)
        allidx = np.concatenate(sl)
        assert len(sl) == world and np.array_equal(np.sort(allidx), np.arange(len(y)))
        sizes = [len(s) for s in sl]
        assert max(sizes) - min(sizes) <= 1
        assert np.all(np.diff(keys[allidx]) >= 0)  # the concatenated slices are in Morton order
    # Morton order of cells: the 8 cells of a 2 x 2 x 2 block get keys 0..7 with x the lowest bit
    c = np.array([[i, j, k] for k in range(2) for j in range(2) for i in range(2)], dtype=float) + 0.5
    assert list(bench.morton_keys(c, 1.0)) == list(range(8))


def _gather_worker(rank, world, port, out):
    import numpy as np
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        rng = np.random.default_rng(1)
        y = rng.uniform(-1, 1, (1001, 3))
        idx = bench.shard_indices(y, 0.1, world)[rank]
        # each rank "evaluates" its slice: a value that identifies the target
        local = torch.from_numpy(y[idx] * 2.0 + 1.0)
        full = bench.gather_rows(local, idx, len(y), world)
        ok = np.array_equal(full.numpy(), y * 2.0 + 1.0)
        # per-rank relative differences and counts reduce to the whole job's
        a = np.ones((len(idx), 3)) * (1.0 + rank)
        r = bench.rel_max(a, np.ones_like(a), world)
        n = bench.sum_over_ranks([len(idx), 1], world)
        out[rank] = float(ok and abs(r - 1.0) < 1e-15 and n == [len(y), world])
    finally:
        dist.destroy_process_group()


def test_gather_restores_target_order_on_every_rank():
    world = 2
    ctx = mp.get_context("spawn")
    out = ctx.Array("d", world)
    port = _free_port()
    procs = [ctx.Process(target=_gather_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert list(out) == [1.0, 1.0]
