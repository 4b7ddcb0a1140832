"""Work across ranks, one GPU per rank.

Batched cells: each rank solves a share of the cells with its own GPU and its own
dtt_batch_solve, and only the per-cell reports are gathered on rank 0 at the end (no
collective on the data path; one solve never spans GPUs).

Warm-start training (train_data_parallel): each rank holds its own training items, and
every step sums the ranks' gradients with one all-reduce before all ranks take the same
optimiser step.

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


class RankFailure(RuntimeError):
    """A collective of the training loop failed: another rank left (crashed, raised, or
    stopped answering until the process group's timeout).  Carries where it happened."""

    def __init__(self, epoch, step, cause):
        super().__init__("data-parallel training: collective failed at epoch %d, step %d (another rank left?): %s"
                         % (epoch, step, cause))
        self.epoch, self.step = epoch, step


def _all_reduce(dist, t, group, epoch, step):
    try:
        dist.all_reduce(t, group=group)
    except RuntimeError as e:    # gloo and NCCL report a lost peer or a timeout this way
        raise RankFailure(epoch, step, e) from e


def local_order(seed, epoch, rank, n):
    """The order in which a rank visits its n items in an epoch (a permutation of its own)."""
    import numpy as np
    return [int(j) for j in np.random.default_rng((int(seed), int(epoch), int(rank))).permutation(n)]


def step_contributors(counts):
    """Per step of an epoch, how many ranks hold an item for it: every rank runs
    max(counts) steps, and a rank past its own items adds a zero gradient."""
    return [sum(1 for c in counts if c > t) for t in range(max(counts, default=0))]


def train_data_parallel(n_local, grad_fn, apply_fn, grad, epochs, lr_at, seed=0, group=None, log=None):
    """Data-parallel training with one gradient all-reduce per step.

    n_local: this rank's item count; grad_fn(j, grad) writes the gradient of the rank's item
    j into grad (a float32 tensor on the rank's device) and returns its loss; apply_fn(grad,
    scale, lr) takes the optimiser step with the gradient scale * grad; lr_at(epoch) the step
    size.  Per epoch every rank visits its items in local_order; at step t a rank with a
    t-th item computes its gradient (otherwise zeroes grad), the ranks sum grad with one
    all-reduce, and every rank applies the sum with scale 1 / (ranks that contributed), the
    mean gradient of the step.  All ranks apply the same values, so their parameters stay
    the same.  Without an initialised process group this is the single-rank loop.  Returns
    the mean loss over all ranks' items per epoch (one small all-reduce per epoch).

    A rank that fails leaves the others blocked in their next all-reduce until the backend
    reports the lost peer or the process group's timeout ends it; they then raise
    RankFailure with the epoch and step (step -1: the start; step = the epoch's step count:
    its loss reduction).  Ranks enter each all-reduce only between optimiser steps, with no
    kernel of theirs in flight.
    """
    import torch
    import torch.distributed as dist
    on = dist.is_available() and dist.is_initialized()
    world = dist.get_world_size(group) if on else 1
    rank = dist.get_rank(group) if on else 0
    counts = [int(n_local)]
    if world > 1:
        cnt = torch.zeros(world, dtype=torch.int64, device=grad.device)
        cnt[rank] = int(n_local)
        _all_reduce(dist, cnt, group, -1, -1)
        counts = [int(c) for c in cnt.tolist()]
    contrib = step_contributors(counts)
    hist = []
    for ep in range(epochs):
        order = local_order(seed, ep, rank, n_local)
        lr = lr_at(ep)
        loss_sum = 0.0
        for t, m in enumerate(contrib):
            if t < n_local:
                loss_sum += float(grad_fn(order[t], grad))
            else:
                grad.zero_()
            if world > 1:
                _all_reduce(dist, grad, group, ep, t)
            apply_fn(grad, 1.0 / m, lr)
        tot = torch.tensor([loss_sum, float(n_local)], dtype=torch.float64, device=grad.device)
        if world > 1:
            _all_reduce(dist, tot, group, ep, len(contrib))
        hist.append(float(tot[0] / tot[1]) if float(tot[1]) > 0 else 0.0)
        if log:
            log(ep, hist[-1])
    return hist
