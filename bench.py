#!/usr/bin/env python3
"""Benchmark: voxel-iterations/s and time to residual 1e-6 of the constrained DTT
solver on one B300, mixed precision against the plain FP64 GPU solver.

Workload (default): the upper half of a compact-tension-like plate in the paper's buffer
device (Section 4.1.2), 128 x 128 x 32 voxels, E = 210, nu = 0.3, TETRA2: a null-stiffness
buffer row behind a u_y-Dirichlet face, ligament nodes held at u_y = 0 (strong rows), a
void notch, one pin disk pulled to u_y = +0.05 (strong rows), u_z Dirichlet on z = 0;
Paux reference (lambda, mu); Anderson on p~ every 2 iterations; tolerance 1e-6 (Eq. 5).
One step = one complete solve from u~ = 0 to the tolerance; every step runs all of the
iteration's kernels.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line.  N > 1 (under torchrun): every rank solves its own replica of the
workload (the solve does not shard); value = all ranks' voxel-iterations / max time.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as wl  # noqa: E402

L2_FLUSH_BYTES = 512 << 20

# DRAM traffic per launch of the dominant kernel on this workload, from one ncu capture
# (profiles/k_residual_f32_ct_128x128x32.md); reported only while the kernel source is the
# one that was profiled.
PROFILED_TRAFFIC = {"residual": {"source": "paper_2607_26082_b300/csrc/k_residual_f32.cu",
                                 "sha256_prefix": "0278c5a438094f6d", "bytes": 48168960}}


def profiled_traffic(group):
    import hashlib
    rec = PROFILED_TRAFFIC.get(group)
    if not rec:
        return None
    try:
        h = hashlib.sha256(open(os.path.join(ROOT, rec["source"]), "rb").read()).hexdigest()
    except OSError:
        return None
    return rec["bytes"] if h.startswith(rec["sha256_prefix"]) else None
FP32_LANES_PER_SM = 128


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="ct", choices=["ct", "indent"])
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--clock-log", default=None,
                    help="keep the raw nvidia-smi samples of the timed region in this CSV file")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload(name):
    if name == "ct":
        return wl.ct_plate(128, 128, 32)
    return wl.indentation(256, 256, 128, R=64.0, steps=10)


def nvox_of(spec):
    return int(np.prod(spec["nvox"]))


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index, path=None):
        self.gpu = gpu_index
        self.proc = None
        self.keep = path is not None
        self.path = path if path else os.path.join(tempfile.gettempdir(), "dtt_bench_clocks_%d.csv" % os.getpid())

    def start(self):
        try:
            if os.path.dirname(self.path):
                os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not self.keep:
            try:
                os.remove(self.path)
            except OSError:
                pass
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ CPU oracle
def oracle_sample(spec, seconds, iters_cap=50):
    """The oracle as it stands (Algorithm 1, float64 numpy, naive trigonometric sums) on
    the full workload, for a bounded number of iterations (~`seconds` of CPU work)."""
    from oracle import constraints as ocs, discrete as odz, solver as osv
    pb = odz.problem_from(spec)
    rows = ocs.rows_from_intents(pb, spec["intents"])
    t0 = time.perf_counter()
    osv.solve_alg1(pb, rows, spec["lam0"], spec["mu0"], 0.0, 1, acv_mod=spec["acv_mod"])
    t1 = time.perf_counter()
    per_it = max(t1 - t0, 1e-6)   # one iteration + set-up, as an estimate
    k = int(max(1, min(iters_cap, seconds / per_it)))
    t0 = time.perf_counter()
    res = osv.solve_alg1(pb, rows, spec["lam0"], spec["mu0"], 0.0, k, acv_mod=spec["acv_mod"])
    dt = time.perf_counter() - t0
    return nvox_of(spec) * res.iterations / dt, res.iterations, dt


def cpu_threads():
    try:
        from threadpoolctl import threadpool_info
        n = [i.get("num_threads", 1) for i in threadpool_info() if i.get("user_api") == "blas"]
        if n:
            return int(max(n))
    except Exception:
        pass
    return os.cpu_count() or 1


# ------------------------------------------------------------------ GPU arm
def launches_per_iteration(has_rows, has_contact, acv):
    """Kernel launches of one captured iteration (every launch runs; after convergence they
    return at once)."""
    n = 1                      # residual
    n += 1 if has_rows else 0  # proj_P
    n += 1 if has_contact else 0
    n += 1                     # ctrl residual
    n += 2 if has_contact else 0
    n += 2 if acv else 0       # ctrl (Gram row, alpha), Green input
    n += 5                     # x, y forward; z forward + Green + z inverse; y, x inverse + increment
    n += 1 if has_rows else 0  # proj_U
    n += 1 if has_contact else 0
    n += 0 if (has_rows and not has_contact) else 1   # ctrl end (else done by proj_U's last CTA)
    return n


def max_over_ranks(value, world, device):
    """The largest value over the ranks (the slowest rank's time), every rank gets it."""
    if world <= 1:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, seconds_max, world):
    """Throughput of the whole job: every rank processes the same units (weak scaling),
    divided by the slowest rank's time."""
    return world * units_per_rank / seconds_max


def run_ours(args, rank, world, local):
    import torch
    from paper_2607_26082_b300 import dtt, rows

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    spec = workload(args.workload)
    if args.workload != "ct":
        raise SystemExit("bench.py times the ct workload; run the indentation block with "
                         "python -m paper_2607_26082_b300.run --workload indent")
    nv = nvox_of(spec)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def make(prec):
        g = rows.setup_grid(spec, prec, stream=stream.cuda_stream)
        g.tuning = g.dtt_autotune(iters=5, acv_mod=spec["acv_mod"])   # kernel tiling, outside the timed region
        return g

    def solve(g, tol, max_iter):
        return g.dtt_solve_step(tol, max_iter, acv_mod=spec["acv_mod"], acv_on=dtt.ACV_P, init=dtt.INIT_ZERO,
                                graph_iters=16)

    def launches_per_solve(iters):
        return ((iters + graph_iters) // graph_iters) * graph_iters * per_it + 1

    graph_iters = 16
    per_it = launches_per_iteration(True, False, True)

    def timed(g, steps, warmup):
        for _ in range(warmup):
            solve(g, spec["tol"], 20000)
        times, iters, launches = [], [], 0
        for _ in range(steps):
            with torch.cuda.stream(stream):
                flush.zero_()            # L2 flush between timed solves (outside the events)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            rep = solve(g, spec["tol"], 20000)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1) / 1e3)
            iters.append(rep.iterations)
            launches += launches_per_solve(rep.iterations)
            if rep.status != dtt.OK:
                raise RuntimeError("solve did not converge: %s" % rep.as_dict())
        return times, iters, rep, launches

    # ---- mixed path (headline)
    gm = make(dtt.PREC_MIXED)
    sampler = ClockSampler(local, args.clock_log)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    sampler.start()
    t_wall0 = time.perf_counter()
    times, iters, rep_m, launches = timed(gm, args.steps, args.warmup)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t_wall0
    clocks = sampler.stop()
    tot_vi = nv * sum(iters)
    tot_t = max_over_ranks(sum(times), world, dev)
    value = whole_job_rate(tot_vi, tot_t, world)

    # ---- kernel-group profile of the mixed iteration (roofline of the dominant group)
    prof = gm.dtt_profile_iteration(20, acv_mod=spec["acv_mod"])
    nn = gm.n_nodes
    # algorithmic bytes of one launch group per iteration (mixed path: T = 4 B fields, u~ as
    # an 8-byte float-float pair, phase ids 1 B per voxel)
    # residual: u~ hi/lo 24, step 12, g_(i-1) 12, three older R slots for the Gram row 36 in;
    # p 12, R 12 out.  Anderson input: p copy (24) or the accelerated combination (132),
    # one in acv_mod.  FFT route: x, y forward passes 24 each; z forward + Green + z
    # inverse 24; y inverse 24, x inverse + increment (u~ hi/lo in and out, step out) 72.
    mod = spec["acv_mod"]
    alg_bytes = {"residual": nn * 108 + nv, "projections": 0,
                 "anderson": nn * (24 * (mod - 1) + 132) / mod,
                 "forward_dt": nn * 48, "green": nn * 24, "inverse_dt": nn * 96, "increment": 0}
    launches_in_group = {"residual": 1, "forward_dt": 2, "inverse_dt": 2, "green": 1, "increment": 1,
                         "anderson": 2, "projections": 4}
    dom = max(prof, key=lambda k: prof[k])
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm = peaks.get("hbm_gbs", 6400.0)
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
    t_launch = prof[dom] / 1e3 / launches_in_group.get(dom, 1)
    b_launch = alg_bytes.get(dom, 0) / launches_in_group.get(dom, 1)
    achieved = b_launch / t_launch / 1e9 if t_launch > 0 else 0.0

    # ---- e2e through the public API with host buffers
    ptr, node, comp, a, b, val = rows.csr_from_intents(spec["nvox"], spec["bc"], spec["intents"])
    h2d = (nv + 16 * len(spec["lam"]) + ptr.nbytes + node.nbytes + comp.nbytes + a.nbytes + b.nbytes +
           val.nbytes)
    d2h = 3 * nn * 8
    e2e_t, e2e_vi = 0.0, 0

    def pinned(x):
        return torch.from_numpy(np.ascontiguousarray(x)).pin_memory().numpy()

    # the step's inputs and its result live in pinned host memory
    phase_h = pinned(spec["phase"].astype(np.uint8))
    ptr, node, comp, a, b, val = (pinned(x) for x in (ptr, node, comp, a, b, val))
    u_host = torch.empty((3,) + tuple(gm.node_shape), dtype=torch.float64).pin_memory().numpy()
    n_e2e = max(1, min(args.steps, 3))
    for k in range(1 + n_e2e):          # one untimed step first: lazy host/device buffers
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        gm.dtt_set_material(phase_h, spec["lam"], spec["mu"])
        gm.dtt_set_constraints(ptr, node, comp, a, b, val)
        rep = solve(gm, spec["tol"], 20000)
        gm.dtt_get_fields(u_out=u_host)
        if k > 0:
            e2e_t += time.perf_counter() - t0
            e2e_vi += nv * rep.iterations
    e2e_value = whole_job_rate(e2e_vi, max_over_ranks(e2e_t, world, dev), world)

    # ---- plain FP64 GPU solver on the same input
    g64 = make(dtt.PREC_FP64)
    t64, it64, rep64, _ = timed(g64, args.fp64_steps, 1)
    fp64 = {"value": nv * sum(it64) / sum(t64), "ms_per_step": 1e3 * sum(t64) / len(t64),
            "iterations": int(statistics.median(it64)), "residual": rep64.residual,
            "tuning": g64.tuning.as_dict()}
    g64.close()

    cpu = None
    if rank == 0 and world == 1:
        v, k, dt = oracle_sample(spec, args.cpu_seconds)
        cpu = {"value": v, "unit": "voxel-iter/s", "cores": cpu_threads(), "kind": "oracle",
               "sample": "%d iterations of Algorithm 1 (float64 numpy oracle) on the full %s, %.1f s" %
                         (k, spec["name"], dt)}

    out = {
        "metric": "voxel-iters/s (time to residual 1e-6: mixed vs plain FP64 GPU)",
        "value": value, "unit": "voxel-iter/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / len(times), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64 (mixed: FP32 transforms/stress, "
        "float-float u~, FP64 norms/Gram/multipliers)", "data": "synthetic",
        "config": {"workload": spec["name"] + ", E=210, nu=0.3, TETRA2, R0=(lambda,mu), tol 1e-6, "
                                "ACV_P mod 2, zero start",
                   "voxels": nv, "nodes": nn, "iterations_per_solve": int(statistics.median(iters)),
                   "time_to_residual_1e-6_ms": 1e3 * tot_t / len(times),
                   "l2": "flushed (512 MB write) before every timed solve", "parallelism": "replicas"},
        "fp64": fp64, "speedup_time_to_residual_vs_fp64": fp64["ms_per_step"] / (1e3 * tot_t / len(times)),
        "speedup_per_iteration_vs_fp64": (tot_vi / tot_t) / fp64["value"],
        "tuning": gm.tuning.as_dict(),
        "roofline": {"bound": "hbm", "kernel_group": dom, "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "peak_source": peak_src, "traffic": profiled_traffic(dom),
                     "group_ms_per_iteration": prof},
        "cpu_baseline": cpu,
        "clocks": clocks,
        "e2e": {"value": e2e_value, "unit": "voxel-iter/s", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": int(launches),
        "wall_s": wall,
    }
    gm.close()
    return out


def run_reference(args, rank, world):
    if rank != 0:
        return None
    spec = workload(args.workload)
    per_step = max(2.0, 150.0 / max(1, args.steps + args.warmup))
    for _ in range(args.warmup):
        oracle_sample(spec, per_step, iters_cap=3)
    vals, ts, ks = [], [], []
    for _ in range(args.steps):
        v, k, dt = oracle_sample(spec, per_step, iters_cap=10)
        vals.append(v)
        ts.append(dt)
        ks.append(k)
    value = nvox_of(spec) * sum(ks) / sum(ts)
    cores = cpu_threads()
    return {
        "impl": "reference", "metric": "voxel-iters/s (time to residual 1e-6: mixed vs plain FP64 GPU)",
        "value": value, "unit": "voxel-iter/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * sum(ts) / len(ts), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": spec["name"] + ", TETRA2, Algorithm 1", "voxels": nvox_of(spec)},
        "cpu_baseline": {"value": value, "unit": "voxel-iter/s", "cores": cores, "kind": "oracle",
                         "sample": "each step: %d-%d iterations of the float64 numpy oracle on the full workload"
                                   % (min(ks), max(ks))},
        "e2e": {"value": value, "unit": "voxel-iter/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    args = parse()
    rank, world, local = dist_env()
    if world > 1 and args.impl == "ours":
        import torch
        torch.distributed.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    if args.impl == "reference":
        out = run_reference(args, rank, world)
    else:
        out = run_ours(args, rank, world, local)
    if rank == 0 and out is not None:
        print(json.dumps(out))
    if world > 1 and args.impl == "ours":
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
