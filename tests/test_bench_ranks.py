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


def test_clock_log_summary():
    """The clock record's summary: median SM clock under load, the largest maximum clock,
    and every throttle reason active in any sample (lines in ClockSampler's field order;
    a malformed or N/A sample is skipped)."""
    sys.path.insert(0, ROOT)
    import bench
    lines = [
        "0, 2032, 2032, 850.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n",
        "0, 1980, 2032, 1099.7, 0x0000000000000004, Not Active, Not Active, Not Active, Active\n",
        "0, 2010, 2032, 990.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n",
        "0, [N/A], 2032, 990.0, 0x0, Not Active, Not Active, Active, Not Active\n",
        "garbage\n",
    ]
    out = bench.parse_clock_log(lines)
    assert out == {"sm_mhz": 2010.0, "sm_max_mhz": 2032.0, "reasons": ["sw_power_cap"], "samples": 3}
    assert bench.parse_clock_log([]) == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
    hot = lines[:1] + ["0, 1500, 2032, 700.0, 0x8, Not Active, Active, Not Active, Not Active\n"]
    assert bench.parse_clock_log(hot)["reasons"] == ["hw_thermal_slowdown"]


def test_clock_sampler_reads_its_file(tmp_path):
    """ClockSampler.stop() summarises the file its nvidia-smi child wrote (a finished
    stand-in process here) and keeps it when a path was given."""
    sys.path.insert(0, ROOT)
    import bench
    path = tmp_path / "clocks.csv"
    cs = bench.ClockSampler(0, str(path))
    cs.fh = open(path, "w")
    cs.fh.write("0, 2032, 2032, 850.1, 0x0, Not Active, Not Active, Not Active, Not Active\n")
    cs.fh.flush()
    cs.proc = __import__("subprocess").Popen([sys.executable, "-c", "pass"])
    cs.proc.wait()
    out = cs.stop()
    assert out["sm_mhz"] == 2032.0 and out["samples"] == 1 and out["reasons"] == []
    assert path.exists()
    assert bench.ClockSampler(0).stop()["reasons"] == ["nvidia-smi unavailable"]
