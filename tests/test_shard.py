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


# ---- data-parallel training: one gradient all-reduce per step ------------------------------
# A stand-in model (least squares, float32, plain gradient steps) exercises the host loop of
# shard.train_data_parallel; the network's own gradient and Adam entry points are checked on
# the GPU (tests/test_gpu_net_dp.py).
def _ls_items(rank, n, dim=6, seed=40):
    rng = np.random.default_rng((seed, rank))
    return [(rng.standard_normal((4, dim)).astype(np.float32), rng.standard_normal(4).astype(np.float32))
            for _ in range(n)]


def _ls_grad(item, w):
    A, b = item
    r = A @ w - b
    return (2.0 * (A.T @ r)).astype(np.float32), float(r @ r)


def _ls_expected(counts, epochs, lr, seed, dim=6):
    """The same training written out on one process: at step t the gradients of the ranks
    that hold a t-th item, summed in rank order, times 1 / their number."""
    items = [_ls_items(r, n, dim) for r, n in enumerate(counts)]
    w = np.zeros(dim, np.float32)
    hist = []
    for ep in range(epochs):
        orders = [shard.local_order(seed, ep, r, n) for r, n in enumerate(counts)]
        losses = []
        for t in range(max(counts)):
            tot, m = np.zeros(dim, np.float32), 0
            for r, n in enumerate(counts):
                if t < n:
                    g, loss = _ls_grad(items[r][orders[r][t]], w)
                    tot = tot + g
                    losses.append(loss)
                    m += 1
            w = w - np.float32(lr) * (np.float32(1.0 / m) * tot)
        hist.append(float(np.mean(losses)))
    return w, hist


def _ls_train(rank, n, epochs, lr, seed):
    import torch
    items = _ls_items(rank, n)
    w = torch.zeros(6, dtype=torch.float32)
    grad = torch.zeros(6, dtype=torch.float32)

    def grad_fn(j, g):
        gv, loss = _ls_grad(items[j], w.numpy())
        g.copy_(torch.from_numpy(gv))
        return loss

    def apply_fn(g, scale, lr_):
        w.copy_(w - np.float32(lr_) * (np.float32(scale) * g))

    hist = shard.train_data_parallel(n, grad_fn, apply_fn, grad, epochs, lambda ep: lr, seed=seed)
    return w.numpy().copy(), hist


def test_step_contributors_and_local_order():
    assert shard.step_contributors([3, 5]) == [2, 2, 2, 1, 1]
    assert shard.step_contributors([2, 0, 2]) == [2, 2]
    assert shard.step_contributors([]) == []
    o = shard.local_order(7, 2, 1, 9)
    assert sorted(o) == list(range(9)) and o == shard.local_order(7, 2, 1, 9)
    assert o != shard.local_order(7, 3, 1, 9) or o != shard.local_order(7, 2, 0, 9)


def test_data_parallel_single_rank_is_the_plain_loop():
    pytest.importorskip("torch")
    w, hist = _ls_train(0, 5, 3, 0.05, 11)
    w_ref, h_ref = _ls_expected([5], 3, 0.05, 11)
    np.testing.assert_array_equal(w, w_ref)
    np.testing.assert_allclose(hist, h_ref, rtol=1e-12)


def _dp_rank(rank, world, port, counts, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    calls = []
    real = dist.all_reduce

    def counted(t, *a, **k):
        calls.append(t.numel())
        return real(t, *a, **k)

    dist.all_reduce = counted
    try:
        w, hist = _ls_train(rank, counts[rank], 3, 0.05, 11)
        out[rank] = (w.tolist(), hist, calls)
    finally:
        dist.all_reduce = real
        dist.destroy_process_group()


@pytest.mark.parametrize("counts", [(4, 4), (3, 5), (2, 5, 0)])
def test_data_parallel_gloo_ranks(counts):
    """Two or three gloo ranks with their own items (equal and unequal counts, one rank
    without any): the parameters agree on every rank bit for bit, equal the single-process
    computation of the mean gradient per step, and each step makes exactly one all-reduce
    of the gradient (besides one of the item counts at the start and one of the loss per
    epoch)."""
    pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        world = len(counts)
        procs = [ctx.Process(target=_dp_rank, args=(r, world, port, list(counts), out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    w0, h0, c0 = res[0]
    for r in range(1, len(counts)):
        assert res[r] == res[0]
    w_ref, h_ref = _ls_expected(list(counts), 3, 0.05, 11)
    np.testing.assert_allclose(np.array(w0, np.float32), w_ref, rtol=1e-6, atol=1e-7)
    np.testing.assert_allclose(h0, h_ref, rtol=1e-6)
    steps = max(counts)
    assert c0 == [len(counts)] + ([6] * steps + [2]) * 3


def _dp_failing_rank(rank, world, port, out):
    import datetime
    import time as _time
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=20))
    from paper_2607_26082_b300 import shard as sh
    items = _ls_items(rank, 4)
    w = torch.zeros(6, dtype=torch.float32)
    grad = torch.zeros(6, dtype=torch.float32)
    seen = []

    def grad_fn(j, g):
        if rank == 1 and len(seen) == 2:
            os._exit(3)                    # rank 1 dies before its third gradient
        seen.append(j)
        gv, loss = _ls_grad(items[j], w.numpy())
        g.copy_(torch.from_numpy(gv))
        return loss

    def apply_fn(g, scale, lr_):
        w.copy_(w - np.float32(lr_) * (np.float32(scale) * g))

    t0 = _time.monotonic()
    try:
        sh.train_data_parallel(4, grad_fn, apply_fn, grad, 2, lambda ep: 0.05, seed=11)
        out[rank] = ("finished",)
    except sh.RankFailure as e:
        out[rank] = ("RankFailure", e.epoch, e.step, _time.monotonic() - t0)


def test_data_parallel_rank_failure_is_reported_not_hung():
    """Failure detection without a GPU: rank 1 exits in the middle of epoch 0 (before its
    third gradient); rank 0 does not hang in the all-reduce of that step but raises
    RankFailure naming epoch 0, step 2, well within the process group's timeout."""
    pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_dp_failing_rank, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
        codes = [p.exitcode for p in procs]
        res = dict(out)
    assert codes == [0, 3]
    kind, epoch, step, secs = res[0]
    assert kind == "RankFailure" and (epoch, step) == (0, 2)
    assert secs < 20.0
