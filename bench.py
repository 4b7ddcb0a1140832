#!/usr/bin/env python3
"""Benchmark: voxel-iterations/s and time to residual 1e-6 of the constrained DTT solver
on one B300 -- learned start + mixed precision against the plain FP64 GPU solver.

Workload: sphere indentation of a 384 x 384 x 192-voxel block (385 x 385 x 193 =
28,607,425 nodes) with seeded stiff spherical inclusions (contrast 5), bottom clamped,
lateral faces traction-free, top face the contact surface (Algorithm 2, Section 5.1), a
rigid sphere of radius 96 pushed in 20 geometric increments to a depth ratio d/R drawn
from U[0.005, 0.05] (seed 3000), reference medium 5 (lambda, mu) of the matrix, Anderson
on p~ every 3 iterations, tolerance 1e-6 (Eq. 5).

One step = one load increment solved to r < 1e-6 (contact set settled) from the start
rule of the arm, all of the iteration's kernels included.  Steps cycle through the 20
increments (the first increment of a cycle starts from u~ = 0); warm-up steps are the
first ones of the cycle.  The working set (~7 GB) is far larger than L2.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Arms on the same increments, same seeds, same process:
  * learned + mixed (the value): the warm-start network's guess (dtt_net_predict) where its
    weights file exists, with the fallback rule (the solve keeps the guess only if its
    Eq. 5 residual is below the previous-step start's); else the previous-step start;
  * plain FP64: previous-step start, on a bounded subset of the timed increments, each
    started from the same field as the mixed arm's start of that increment.
Prints one JSON line.  N > 1 (under torchrun): every rank solves its own replica (the solve
does not shard); value = all ranks' voxel-iterations / the slowest rank's time.
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

METRIC = "voxel-iters/s and time to residual 1e-6: learned+mixed vs plain FP64 GPU"
SEED = 3000
NVOX = (384, 384, 192)
GRAPH_ITERS = 16
L2_FLUSH_BYTES = 512 << 20
# algorithmic bytes per node and iteration (mixed: 4-byte fields): the Green step (forward
# DTT, Green multiply, inverse DTT) reads and writes the three components in three sweeps;
# the residual group (stress, divergence, reference term, Anderson store and Gram row)
# reads u~ and writes p~ (25 B) and stores R and reads three older R slots (60 B)
# kernel launches of one warm-start prediction: the features (5), the network's forward
# pass (11 convolutions, 2 poolings, 2 upsamplings), the guess and its contact zone (2),
# writing the guess (2) and the fallback rule's two start evaluations (2 x 5)
LAUNCHES_PER_PREDICT = 34
B_GREEN = 72
B_RESIDUAL = 85
# ncu DRAM bytes (read + write) of the Green step's five kernels per node and iteration,
# from one capture of the 256x256x128 indentation (8,520,321 nodes; the traffic grows with
# the node count), with the source hash of the kernel file they came from: reported as null
# once that source has changed
PROFILED_TRAFFIC = {"green": {"bytes_per_node": 1062.14e6 / 8520321, "source": "paper_2607_26082_b300/csrc/k_wfft.cu",
                              "sha256_16": "1174ab76d9319731"}}


def profiled_traffic(key, nodes):
    """DRAM bytes per iteration of a profiled kernel group on a grid of the given node count, or
    None when its source has changed since the capture."""
    import hashlib
    rec = PROFILED_TRAFFIC.get(key)
    if not rec:
        return None
    with open(os.path.join(ROOT, rec["source"]), "rb") as f:
        if hashlib.sha256(f.read()).hexdigest()[:16] != rec["sha256_16"]:
            return None
    return rec["bytes_per_node"] * nodes


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--seed", type=int, default=SEED)
    ap.add_argument("--fp64-steps", type=int, default=3,
                    help="timed increments the plain FP64 arm solves (evenly spread over the timed ones)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-ct", action="store_true", help="skip the secondary CT-specimen line")
    ap.add_argument("--weights", default=None, help="warm-start network weights (.npz); default: the package's")
    ap.add_argument("--clock-log", default=None,
                    help="keep the raw nvidia-smi samples of the timed region in this CSV file")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload(seed=SEED, nvox=NVOX):
    return wl.indentation_inclusions(seed, *nvox, steps=20)


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
        with open(self.path) as f:
            out = parse_clock_log(f)
        if not self.keep:
            try:
                os.remove(self.path)
            except OSError:
                pass
        return out


def parse_clock_log(lines):
    """Summary of ClockSampler's nvidia-smi lines (its FIELDS, no header, no units): median
    and largest SM clock, and the throttle reasons that were active in any sample."""
    sm, smax, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in lines:
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
    return {"sm_mhz": statistics.median(sm) if sm else None,
            "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
            "samples": len(sm)}


# ------------------------------------------------------------------ CPU oracle
ORACLE_NVOX = (128, 128, 64)


def oracle_sample(seconds, iters_cap=20, seed=SEED):
    """The oracle as it stands (Algorithm 2, float64 numpy, naive trigonometric sums) on
    a bounded sample: the same generator and seed at 128 x 128 x 64 voxels (R = 32, the
    same R / L), the first increment from u~ = 0, for about `seconds` of CPU work.  The
    full 384 x 384 x 192 block needs tens of GB of host memory and minutes per oracle
    iteration; per voxel the smaller block is cheaper for the oracle (shorter dense
    transforms), so its rate flatters the oracle."""
    from oracle import constraints as ocs, discrete as odz, solver as osv
    spec = workload(seed, ORACLE_NVOX)
    pb = odz.problem_from(spec)
    I = spec["indenter"]
    ind = ocs.Indenter(pb, I["axis"], I["face"], I["centers"][0], I["radius"])
    u0 = np.zeros((3,) + pb.node_shape)
    t0 = time.perf_counter()
    osv.solve_alg2_increment(pb, ind, [], spec["lam0"], spec["mu0"], 0.0, 1, u0, acv_mod=spec["acv_mod"])
    per_it = max(time.perf_counter() - t0, 1e-6)   # one iteration + set-up, an estimate
    k = int(max(1, min(iters_cap, seconds / per_it)))
    t0 = time.perf_counter()
    res = osv.solve_alg2_increment(pb, ind, [], spec["lam0"], spec["mu0"], 0.0, k, u0, acv_mod=spec["acv_mod"])
    dt = time.perf_counter() - t0
    return nvox_of(spec) * res.iterations / dt, res.iterations, dt, spec


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
def launches_per_iteration(has_rows, has_contact, acv, exact=True, split=True):
    """Kernel launches of one captured iteration (every launch runs; after convergence they
    return at once); exact: the exact residual mode's Green-input fix-up over the tiles of
    constrained DOFs; split: its residual as two passes (without the reference flux, then
    the marked tiles' node planes), as short marked z ranges (a contact face) give."""
    n = 2 if (exact and split) else 1   # residual
    n += 1 if has_rows else 0  # proj_P
    n += 1 if has_contact else 0
    n += 1                     # ctrl residual
    n += 2 if has_contact else 0
    n += 2 if acv else 0       # ctrl (Gram row, alpha), Green input
    n += 1 if (acv and exact) else 0
    n += 5                     # x, y forward; z forward + Green + z inverse; y, x inverse + increment
    n += 1 if has_rows else 0  # proj_U
    n += 1 if has_contact else 0
    n += 0 if (has_rows and not has_contact) else 1   # ctrl end (else done by proj_U's last CTA)
    return n


def launches_per_solve(iters, per_it, graph_iters=GRAPH_ITERS, prep=3):
    """The solve's graph runs whole rounds of graph_iters iterations (the round after the
    last Green step detects the finish), each round followed by the loop's condition kernel;
    prep = the start's projections."""
    rounds = (iters + graph_iters) // graph_iters
    return rounds * (graph_iters * per_it + 1) + prep


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


def spread(n, k):
    """k indices spread evenly over range(n) (the last one included)."""
    if k <= 0 or n <= 0:
        return []
    if k >= n:
        return list(range(n))
    return sorted({int(round(i * (n - 1) / (k - 1))) for i in range(k)}) if k > 1 else [n - 1]


def default_weights():
    return os.path.join(ROOT, "paper_2607_26082_b300", "weights", "warmstart_indent.npz")


def run_ct_secondary(torch, dtt, rows, stream, flush, solves=3):
    """The former headline, kept as a secondary figure: the half CT-like specimen
    (128 x 128 x 32, Section 4.1.2) solved from u~ = 0 to r < 1e-6 in mixed precision."""
    spec = wl.ct_plate(128, 128, 32)
    g = rows.setup_grid(spec, dtt.PREC_MIXED, stream=stream.cuda_stream)
    g.dtt_autotune(iters=5, acv_mod=spec["acv_mod"])
    ts, its = [], []
    for k in range(1 + solves):
        with torch.cuda.stream(stream):
            flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rep = g.dtt_solve_step(spec["tol"], 20000, acv_mod=spec["acv_mod"], init=dtt.INIT_ZERO,
                               graph_iters=GRAPH_ITERS)
        e1.record(stream)
        e1.synchronize()
        if k:
            ts.append(e0.elapsed_time(e1) / 1e3)
            its.append(rep.iterations)
    g.close()
    nv = nvox_of(spec)
    return {"workload": spec["name"] + ", mixed, zero start, tol 1e-6", "ms_per_solve": 1e3 * sum(ts) / len(ts),
            "iterations": int(statistics.median(its)), "voxel_iter_per_s": nv * sum(its) / sum(ts)}


def run_ours(args, rank, world, local):
    import torch
    from paper_2607_26082_b300 import dtt, rows

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    spec = workload(args.seed)
    I = spec["indenter"]
    ncyc = len(I["centers"])
    nv, mod, tol = nvox_of(spec), spec["acv_mod"], spec["tol"]
    per_it = launches_per_iteration(False, True, True)

    gm = rows.setup_grid(spec, dtt.PREC_MIXED, stream=stream.cuda_stream)
    nn = gm.n_nodes
    tuning = gm.dtt_autotune(iters=4, acv_mod=mod)            # kernel tiling, outside the timed region
    gm.dtt_set_indenter(I["axis"], I["face"], I["centers"][0], I["radius"])

    # learned start (row a11): the warm-start network, if its trained weights are present
    wpath = args.weights or default_weights()
    net, learned = None, None
    if os.path.exists(wpath):
        from paper_2607_26082_b300 import warmstart
        net = warmstart.load_net(wpath, stream=stream.cuda_stream)
        learned = {"weights": os.path.relpath(wpath, ROOT), "kept": 0, "steps": 0}
    dk = [float(r) * float(I["radius"]) for r in I["ratios"]]

    u_dev = torch.empty((3,) + tuple(gm.node_shape), dtype=torch.float64, device=dev)
    fp64_idx = set(spread(args.steps, args.fp64_steps))
    starts = {}                  # timed step -> (increment, start field on the device)
    hist = {"u2": None, "u1": torch.empty_like(u_dev) if net is not None else None}

    def step(s, record_start=False, centers=None):
        """One increment: the learned arm keeps u~ of the increment before the previous
        one for the network's features; the previous reactions are the grid's own (its last
        solve), read on the device."""
        k = s % ncyc
        if record_start:
            if k == 0:
                starts[s] = (k, None)
            else:
                gm.dtt_get_fields(u_out=u_dev)
                starts[s] = (k, u_dev.clone())
                torch.cuda.current_stream().synchronize()
        if k == 0:
            hist["u2"] = None
        gm.dtt_move_indenter((centers if centers is not None else I["centers"])[k])
        init = dtt.INIT_ZERO if k == 0 else dtt.INIT_PREVIOUS
        if net is not None and k > 0:
            gm.dtt_get_fields(u_out=hist["u1"])          # u~ of increment k-1, before it is replaced
            depth = (dk[k - 2] if k >= 2 else 0.0, dk[k - 1], dk[k])
            net.predict_increment(gm, hist["u2"], None, depth)
            init = dtt.INIT_GUESS
        rep = gm.dtt_solve_step(tol, 20000, acv_mod=mod, init=init, graph_iters=GRAPH_ITERS)
        if rep.status != dtt.OK:
            raise RuntimeError("increment %d did not converge: %s" % (k, rep.as_dict()))
        if net is not None and k > 0:
            if hist["u2"] is None:
                hist["u2"] = torch.empty_like(u_dev)
            hist["u2"], hist["u1"] = hist["u1"], hist["u2"]
        return k, rep

    for s in range(args.warmup):
        step(s)

    sampler = ClockSampler(local, args.clock_log)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    sampler.start()
    t_wall0 = time.perf_counter()
    times, iters, incs, launches, kept = [], [], [], 0, 0
    for t in range(args.steps):
        s = args.warmup + t
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        k, rep = step(s, record_start=(t in fp64_idx))
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
        iters.append(rep.iterations)
        incs.append(k)
        launches += launches_per_solve(rep.iterations, per_it)
        if net is not None and k > 0:
            kept += rep.start_from_guess
            launches += LAUNCHES_PER_PREDICT
    torch.cuda.synchronize()
    wall = time.perf_counter() - t_wall0
    clocks = sampler.stop()
    tot_vi = nv * sum(iters)
    tot_t = max_over_ranks(sum(times), world, dev)
    value = whole_job_rate(tot_vi, tot_t, world)
    if learned is not None:
        learned.update({"kept": kept, "steps": sum(1 for k in incs if k > 0)})

    # ---- kernel-group profile of the mixed iteration (roofline of the Green step)
    prof = gm.dtt_profile_iteration(20, acv_mod=mod)
    t_green = (prof["forward_dt"] + prof["green"] + prof["inverse_dt"] + prof["increment"]) / 1e3
    t_res = prof["residual"] / 1e3
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm = peaks.get("hbm_gbs", 6400.0)
    peak_src = "measured (MEASURED_PEAKS.json hbm_gbs)" if "hbm_gbs" in peaks else "fallback"
    green_ach = B_GREEN * nn / t_green / 1e9
    res_ach = B_RESIDUAL * nn / t_res / 1e9

    # ---- e2e through the public API with host buffers: move the sphere (centre from pinned
    # host memory), solve, read u~ and the contact state back into pinned host memory
    u_host = torch.empty((3,) + tuple(gm.node_shape), dtype=torch.float64).pin_memory()
    centers_h = torch.from_numpy(np.array(I["centers"], dtype=np.float64)).pin_memory().numpy()
    n_e2e = max(1, min(args.steps, 3))
    e2e_t, e2e_vi = 0.0, 0
    s0 = args.warmup + args.steps
    nface = None
    for j in range(n_e2e):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        k, rep = step(s0 + j, centers=centers_h)
        gm.dtt_get_fields(u_out=u_host)
        act, gap, fn, force = gm.dtt_get_contact()
        e2e_t += time.perf_counter() - t0
        e2e_vi += nv * rep.iterations
        nface = len(act)
    e2e_value = whole_job_rate(e2e_vi, max_over_ranks(e2e_t, world, dev), world)
    d2h = 3 * nn * 8 + nface * (1 + 8 + 8) + 24

    # ---- plain FP64 GPU solver on the same increments, from the same starting fields
    gm_tuning = tuning.as_dict()
    g64 = rows.setup_grid(spec, dtt.PREC_FP64, stream=stream.cuda_stream)
    g64.dtt_autotune(iters=2, acv_mod=mod)
    g64.dtt_set_indenter(I["axis"], I["face"], I["centers"][0], I["radius"])
    t64, it64, tmx, itmx = [], [], [], []
    for t in sorted(fp64_idx):
        k, u0 = starts[args.warmup + t]
        if u0 is not None:
            g64.dtt_set_initial(u0)
        g64.dtt_move_indenter(I["centers"][k])
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rep = g64.dtt_solve_step(tol, 20000, acv_mod=mod, init=dtt.INIT_ZERO if u0 is None else dtt.INIT_PREVIOUS,
                                 graph_iters=GRAPH_ITERS)
        e1.record(stream)
        e1.synchronize()
        if rep.status != dtt.OK:
            raise RuntimeError("FP64 increment %d did not converge: %s" % (k, rep.as_dict()))
        t64.append(e0.elapsed_time(e1) / 1e3)
        it64.append(rep.iterations)
        tmx.append(times[t])
        itmx.append(iters[t])
    g64.close()
    starts.clear()
    fp64 = {"increments": [int(incs[t]) for t in sorted(fp64_idx)],
            "seconds": t64, "iterations": it64, "mixed_seconds": tmx, "mixed_iterations": itmx,
            "value": nv * sum(it64) / sum(t64) if t64 else None,
            "start": "the same field as the mixed arm's start of each increment (previous increment's "
                     "solution), plain previous-step start, no network"}

    ct = None
    if not args.no_ct and rank == 0:
        flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
        ct = run_ct_secondary(torch, dtt, rows, stream, flush)
        del flush

    cpu = None
    if rank == 0 and world == 1:
        v, k, dt, ospec = oracle_sample(args.cpu_seconds, seed=args.seed)
        cpu = {"value": v, "unit": "voxel-iter/s", "cores": cpu_threads(), "kind": "oracle",
               "sample": "%d iterations of Algorithm 2 (float64 numpy oracle, first increment) on the same "
                         "generator and seed at %dx%dx%d voxels, %.1f s" % ((k,) + ORACLE_NVOX + (dt,))}

    ms_step = 1e3 * tot_t / len(times)
    out = {
        "metric": METRIC, "value": value, "unit": "voxel-iter/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64 (mixed: FP32 transforms/stress, float-float u~, FP64 norms/Gram/multipliers/gap)",
        "data": "synthetic",
        "config": {"workload": spec["name"] + ", 20 geometric increments, Algorithm 2, TETRA2, R0 = 5 (lambda, mu), "
                               "ACV_P mod 3, tol 1e-6, one step = one increment",
                   "voxels": nv, "nodes": nn, "seed": args.seed,
                   "increments_timed": incs, "iterations_per_step": iters,
                   "start": ("learned (network guess, fallback to the previous-step start)" if net is not None
                             else "previous-step start (no trained network weights found)"),
                   "time_to_residual_1e-6_s": tot_t, "time_to_residual_1e-6_ms_per_increment": ms_step,
                   "l2": "inputs larger than L2 (about 7 GB resident), no flush", "parallelism": "replicas"},
        "learned": learned,
        "fp64_same_increments": fp64,
        "speedup_time_to_residual_vs_fp64": (sum(t64) / sum(tmx)) if t64 else None,
        "speedup_per_iteration_vs_fp64": ((sum(t64) / sum(it64)) / (sum(tmx) / sum(itmx))) if t64 else None,
        "tuning": gm_tuning,
        "roofline": {"bound": "hbm", "kernel_group": "Green step (forward DTT x/y, fused z pass with the Green "
                                                      "multiply, inverse DTT y/x with the increment)",
                     "achieved": green_ach, "peak": hbm, "unit": "GB/s", "frac": green_ach / hbm,
                     "peak_source": peak_src, "traffic": profiled_traffic("green", nn),
                     "alg_bytes_per_node": B_GREEN, "ms_per_iteration": 1e3 * t_green,
                     "residual_group": {"achieved": res_ach, "frac": res_ach / hbm, "alg_bytes_per_node": B_RESIDUAL,
                                        "ms_per_iteration": 1e3 * t_res},
                     "group_ms_per_iteration": prof},
        "cpu_baseline": cpu,
        "clocks": clocks,
        "e2e": {"value": e2e_value, "unit": "voxel-iter/s", "h2d_bytes_per_step": 24, "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": int(launches),
        "ct_secondary": ct,
        "wall_s": wall,
    }
    if net is not None:
        net.close()
    gm.close()
    return out


def run_reference(args, rank, world):
    if rank != 0:
        return None
    per_step = max(2.0, 150.0 / max(1, args.steps + args.warmup))
    for _ in range(args.warmup):
        oracle_sample(per_step, iters_cap=2, seed=args.seed)
    vals, ts, ks = [], [], []
    spec = None
    for _ in range(args.steps):
        v, k, dt, spec = oracle_sample(per_step, iters_cap=4, seed=args.seed)
        vals.append(v)
        ts.append(dt)
        ks.append(k)
    value = nvox_of(spec) * sum(ks) / sum(ts)
    cores = cpu_threads()
    return {
        "impl": "reference", "metric": METRIC,
        "value": value, "unit": "voxel-iter/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * sum(ts) / len(ts), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": spec["name"] + " (the benchmark's generator and seed at %dx%dx%d), Algorithm 2"
                               % ORACLE_NVOX, "voxels": nvox_of(spec)},
        "cpu_baseline": {"value": value, "unit": "voxel-iter/s", "cores": cores, "kind": "oracle",
                         "sample": "each step: %d-%d iterations of the float64 numpy oracle (first increment) at "
                                   "%dx%dx%d voxels" % ((min(ks), max(ks)) + ORACLE_NVOX)},
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
