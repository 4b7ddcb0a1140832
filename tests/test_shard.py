"""Cells of the batched workload across ranks (paper_2607_26082_b300.shard): the
longest-processing-time partition and the gather of the ranks' reports, with two gloo
ranks on the CPU."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_2607_26082_b300 import shard  # noqa: E402
import workloads as wl  # noqa: E402


@pytest.mark.parametrize("nranks", [1, 2, 3, 8])
def test_lpt_partition_covers_every_cell_once_and_balances(nranks):
    cells = wl.batch_cells(64, seed0=1000)
    costs = [int(np.prod(c["nvox"])) for c in cells]
    parts = shard.lpt_partition(costs, nranks)
    assert len(parts) == nranks
    flat = sorted(i for p in parts for i in p)
    assert flat == list(range(len(costs)))
    loads = [sum(costs[i] for i in p) for p in parts]
    # longest-first greedy: the spread of the loads is at most one cell's cost
    assert max(loads) - min(loads) <= max(costs)
    assert shard.lpt_partition(costs, nranks) == parts          # deterministic


def test_lpt_partition_small_cases():
    assert shard.lpt_partition([5, 4, 3, 3, 3], 2) == [[0, 3], [1, 2, 4]]
    assert shard.lpt_partition([], 3) == [[], [], []]
    assert shard.lpt_partition([7], 2) == [[0], []]
    with pytest.raises(ValueError):
        shard.lpt_partition([1], 0)


def test_merge_reports():
    a = {"cells": [0, 2], "voxels": 10, "voxel_iters": 100, "batch_s": 2.0, "cell_iterations": [4, 6], "failed": []}
    b = {"cells": [1], "voxels": 8, "voxel_iters": 80, "batch_s": 4.0, "cell_iterations": [10], "failed": [1]}
    m = shard.merge_reports([a, b])
    assert m["cells"] == 3 and m["voxel_iters"] == 180 and m["batch_s"] == 4.0
    assert m["voxel_iters_per_s"] == 45.0
    assert m["iterations"] == {"min": 4, "max": 10, "mean": 20 / 3}
    assert m["failed"] == [1]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2607_26082_b300 import shard as sh
        costs = [9, 7, 5, 4, 3, 2, 1]
        mine = sh.lpt_partition(costs, world)[rank]
        # a stand-in for the solve: iterations = cost, time = rank + 1
        part = {"cells": mine, "voxels": sum(costs[i] for i in mine),
                "voxel_iters": sum(costs[i] * costs[i] for i in mine), "batch_s": float(rank + 1),
                "cell_iterations": [costs[i] for i in mine], "failed": []}
        got = sh.gather_to_root(part, rank, world)
        out[rank] = got
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_gather_on_root():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    assert res[1] is None
    per_rank = res[0]
    assert [r["cells"] for r in per_rank] == shard.lpt_partition([9, 7, 5, 4, 3, 2, 1], 2)
    merged = shard.merge_reports(per_rank)
    assert merged["cells"] == 7
    assert merged["voxel_iters"] == sum(c * c for c in [9, 7, 5, 4, 3, 2, 1])
    assert merged["batch_s"] == 2.0
    assert sorted(merged["rank_voxels"]) == [15, 16]
