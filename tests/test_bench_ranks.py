"""The multi-rank arithmetic of bench.py on CPU ranks (gloo, world size 2): every rank
gets the slowest rank's time, the whole-job rate is world x units / that time, and the
reference arm runs on rank 0 only."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        t = bench.max_over_ranks(1.0 + 2.0 * rank, world, torch.device("cpu"))
        rate = bench.whole_job_rate(1000.0, t, world)

        class A:
            workload, steps, warmup = "ct", 1, 0
        ref = bench.run_reference(A, rank, world) if rank != 0 else "skipped"
        out[rank] = (t, rate, ref)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
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
    for r in range(2):
        t, rate, _ = res[r]
        assert t == 3.0                       # the slower rank's time, on both ranks
        assert rate == 2 * 1000.0 / 3.0
    assert res[1][2] is None                  # reference arm: no work off rank 0


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(2.5, 1, None) == 2.5
    assert bench.whole_job_rate(10.0, 2.0, 1) == 5.0
