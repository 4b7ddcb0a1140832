"""Batched cells across ranks: each rank solves a share of the cells with its own GPU and
its own dtt_batch_solve, and only the per-cell reports are gathered on rank 0 at the end
(no collective on the data path; one solve never spans GPUs).

lpt_partition assigns cells to ranks by the longest-processing-time-first rule, with the
voxel count as a cell's cost: cells in decreasing order of cost, each to the rank with the
smallest load so far (ties: the lower rank).  The largest rank load then exceeds the
smallest by at most one cell's cost.
"""
import json
import os


def lpt_partition(costs, nranks):
    """List of nranks lists of cell indices (each in increasing order)."""
    if nranks < 1:
        raise ValueError("nranks must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    loads = [0] * nranks
    parts = [[] for _ in range(nranks)]
    for i in order:
        r = min(range(nranks), key=lambda q: (loads[q], q))
        parts[r].append(i)
        loads[r] += costs[i]
    return [sorted(p) for p in parts]


def rank_world():
    """(rank, world size, local rank) from the launcher's environment (1 process: 0, 1, 0)."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def gather_to_root(obj, rank, world):
    """Every rank's obj, in rank order, on rank 0 (None elsewhere); a plain list on one rank."""
    if world == 1:
        return [obj]
    import torch.distributed as dist
    out = [None] * world if rank == 0 else None
    dist.gather_object(json.dumps(obj), out, dst=0)
    return [json.loads(s) for s in out] if rank == 0 else None


def merge_reports(per_rank):
    """Whole-job summary from the ranks' reports: all cells' voxel-iterations over the
    slowest rank's time."""
    vi = sum(r["voxel_iters"] for r in per_rank)
    t = max(r["batch_s"] for r in per_rank)
    its = [i for r in per_rank for i in r["cell_iterations"]]
    return {"ranks": len(per_rank), "cells": sum(len(r["cells"]) for r in per_rank), "voxel_iters": vi,
            "batch_s": t, "voxel_iters_per_s": vi / t if t > 0 else 0.0,
            "rank_voxels": [r["voxels"] for r in per_rank],
            "iterations": {"min": min(its), "max": max(its), "mean": sum(its) / len(its)} if its else None,
            "failed": [c for r in per_rank for c in r["failed"]]}
