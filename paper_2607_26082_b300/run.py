"""Command-line runner: solve one of the synthetic workloads with the CUDA path.

  python -m paper_2607_26082_b300.run --workload ct|ct_paper|cube16|indent|indent_cube|indent_inclusions|iso_cell
         [--precision mixed|fp64]
         [--iters K | --tol T] [--steps S] [--graph-iters G] [--nvox nx,ny,nz]
         [--kinematics ss|fs] [--r0-scale K] [--load-steps N] [--max-iter M] [--stop-on-fail] [--learned]
         [--ct-load strong_line|weak_line|strong_node|weak_node|smooth_node] [--acv-on u|p] [--acv-mod M]
         [--medium paux|iso] [--scheme tetra2|hex1] [--contrast K]
  python -m paper_2607_26082_b300.run --workload batch [--cells N] [--seed0 S] [--no-tune]
         [--sequential]

The batch workload draws N uneven two-phase cells (edges 32, 48, 64, 96), tunes the kernel
tiling once per cell size (dtt_autotune on one cell, dtt_set_tuning on the others) and
solves all cells with one dtt_batch_solve; --sequential also solves them one after the
other with dtt_solve_step for comparison.  Under torchrun (one rank per GPU) each rank
takes its share of the cells by voxel count and rank 0 prints the merged report.

--kinematics fs solves with the finite-strain stress step (Section 5.2, Algorithm 3 for
the indentation); --r0-scale multiplies the workload's reference medium (the paper takes a
stiffer one in finite strain); --load-steps N splits the indentation into N geometric
increments (default 20 for indent, whose 10-increment schedule leaves the physical branch
at its last step, and the paper's 80 for indent_cube); --max-iter caps the iterations of each step (default 20000) and
--stop-on-fail ends the run at the first step that does not converge; --radius, --dmin and
--dmax set the indent workload's sphere radius and its first and last depth ratios;
--learned starts every increment of an indentation after the first from the warm-start
network's guess (the package's trained weights; the solve keeps the fallback rule and
reports start_from_guess).  ct_paper is the
paper's 10 x 100 x (50 + 1) CT-like specimen with the loading --ct-load; it reports the
reactions of the load rows and of the ligament rows and their balance.  --acv-on and
--acv-mod override the workload's Anderson settings.  iso_cell is a two-phase cell with
normal mixed conditions on every face (--nvox, --seed0, --contrast: stiffness ratio of
the phases); --medium picks the reference medium
(Section 3.2.3) and --scheme the discretisation for any workload.  --iters K runs
exactly K iterations (tolerance 0) of the first load step, which is the
short, fixed launch sequence a profiler wants; --tol runs to convergence.  For the
indentation block every load step moves the sphere (Algorithm 2, one increment each),
starting from the previous step's solution.  --tune runs dtt_autotune on the grid first
(outside the reported step times).  Prints one JSON report per step.
"""
import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as wl  # noqa: E402

from . import dtt, rows  # noqa: E402


def make_workload(name, nvox=None, load_steps=None, contrast=4.0, radius=None, dmin=None, dmax=None):
    """ct: half compact-tension-like specimen 128x128x32; cube16: 16^3 cube with pinned
    nodes; indent: sphere indentation of a 256x256x128 block, R = 64.  nvox rescales ct and
    indent (the indenter radius scales with the block); indent_inclusions: the 384x384x192
    block with 2-8 stiff spherical inclusions and a sphere of radius 96 (--seed0 picks the
    sample, nvox rescales it); indent_cube: Section 5.4's 65^3 cube
    with a sphere of the cube's diameter, `load_steps` equal steps to d/R = 0.2."""
    if name == "ct":
        return wl.ct_plate(*(nvox or (128, 128, 32)))
    if name == "cube16":
        return wl.cube16()
    if name.startswith("ct_paper:"):
        return wl.ct_specimen(name.split(":", 1)[1])
    if name.startswith("iso_cell:"):
        return wl.iso_cell(int(name.split(":", 1)[1]), nvox=nvox or (128, 128, 128), n_strong=0, contrast=contrast)
    if name.startswith("indent_inclusions:"):
        n = nvox or (384, 384, 192)
        return wl.indentation_inclusions(int(name.split(":", 1)[1]), *n, steps=load_steps or 20)
    if name == "indent_cube":
        return wl.indentation_cube(nvox[0] if nvox else 65, steps=load_steps or 80, dmax=0.2)
    if name == "indent":
        n = nvox or (256, 256, 128)
        return wl.indentation(*n, R=radius or 64.0 * n[0] / 256.0, steps=load_steps or 20,
                              dmin=dmin or 0.001, dmax=dmax or 0.05)
    raise SystemExit("unknown workload %r" % name)


def run_batch(a, prec):
    import time
    from . import shard
    rank, world, local = shard.rank_world()
    all_cells = wl.batch_cells(a.cells, seed0=a.seed0)
    if world > 1:
        # one GPU per rank; the cells are split by voxel count, the reports gathered at the end
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    mine = shard.lpt_partition([int(np.prod(c["nvox"])) for c in all_cells], world)[rank]
    cells = [all_cells[i] for i in mine]
    grids = [rows.setup_grid(c, prec) for c in cells]
    nvox = sum(int(np.prod(c["nvox"])) for c in cells)
    tuned = {}
    t0 = time.perf_counter()
    if not a.no_tune:
        for c, g in zip(cells, grids):
            n = c["nvox"][0]
            if n not in tuned:
                tuned[n] = g.dtt_autotune(iters=4, acv_mod=2)
            else:
                g.dtt_set_tuning(tuned[n])
    t_tune = time.perf_counter() - t0
    out = {"workload": "batch of %d two-phase cells" % len(cells), "precision": a.precision,
           "voxels": nvox, "tuning_s": t_tune,
           "tuning": {str(k): v.as_dict() for k, v in tuned.items()}}
    st, reps, dt = dtt.OK, [], 0.0   # a rank can be left without cells when ranks outnumber them
    for rep_i in range(2 if grids else 0):   # the first call captures the batch graph
        t0 = time.perf_counter()
        st, reps = dtt.dtt_batch_solve(grids, 1e-6, 20000, acv_mod=2, graph_iters=16)
        dt = time.perf_counter() - t0
    vi = sum(int(np.prod(c["nvox"])) * r.iterations for c, r in zip(cells, reps))
    its = [r.iterations for r in reps]
    out.update({"status": st, "batch_s": dt, "voxel_iters": vi, "voxel_iters_per_s": vi / dt if dt > 0 else 0.0,
                "iterations": {"min": min(its), "max": max(its), "mean": float(np.mean(its))} if its else None,
                "failed": [i for i, r in enumerate(reps) if r.status != dtt.OK]})
    if a.sequential:
        t0 = time.perf_counter()
        for g in grids:
            g.dtt_solve_step(1e-6, 20000, acv_mod=2, graph_iters=16)
        out["sequential_s"] = time.perf_counter() - t0
    for g in grids:
        g.close()
    if world == 1:
        print(json.dumps(out), flush=True)
        return 0
    part = {"cells": mine, "voxels": nvox, "voxel_iters": vi, "batch_s": dt,
            "cell_iterations": [r.iterations for r in reps], "failed": [mine[i] for i in out["failed"]]}
    per_rank = shard.gather_to_root(part, rank, world)
    if rank == 0:
        merged = shard.merge_reports(per_rank)
        merged.update({"workload": "batch of %d two-phase cells" % len(all_cells), "precision": a.precision,
                       "split": "cells across ranks by voxel count, longest first"})
        print(json.dumps(merged), flush=True)
    import torch.distributed as dist
    dist.destroy_process_group()
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="ct",
                    choices=["ct", "ct_paper", "cube16", "indent", "indent_cube", "indent_inclusions", "iso_cell",
                             "batch"])
    ap.add_argument("--medium", default=None, choices=["paux", "iso"])
    ap.add_argument("--scheme", default=None, choices=["tetra2", "hex1"])
    ap.add_argument("--contrast", type=float, default=4.0)
    ap.add_argument("--ct-load", default="strong_line", choices=list(wl.CT_LOADS))
    ap.add_argument("--acv-on", default="p", choices=["u", "p"])
    ap.add_argument("--acv-mod", type=int, default=0, help="0: the workload's")
    ap.add_argument("--cells", type=int, default=256)
    ap.add_argument("--seed0", type=int, default=1000)
    ap.add_argument("--no-tune", action="store_true", help="batch: keep the built-in tiling")
    ap.add_argument("--tune", action="store_true",
                    help="single grid: dtt_autotune before the first step (residual z chunk, FFT route)")
    ap.add_argument("--sequential", action="store_true")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--iters", type=int, default=0, help="fixed iteration count (tolerance 0)")
    ap.add_argument("--repeat", type=int, default=1,
                    help="with --iters: solve the first step this many times in one process and "
                         "report every repetition's time per iteration (the first includes one-time set-up)")
    ap.add_argument("--tol", type=float, default=None)
    ap.add_argument("--steps", type=int, default=1, help="load steps (indentation only)")
    ap.add_argument("--graph-iters", type=int, default=0)
    ap.add_argument("--nvox", default=None, help="voxels nx,ny,nz (ct and indent)")
    ap.add_argument("--kinematics", default="ss", choices=["ss", "fs"])
    ap.add_argument("--r0-scale", type=float, default=1.0)
    ap.add_argument("--load-steps", type=int, default=None)
    ap.add_argument("--max-iter", type=int, default=20000)
    ap.add_argument("--radius", type=float, default=None, help="indent: sphere radius (default: a quarter of nx)")
    ap.add_argument("--dmin", type=float, default=None, help="indent: first depth ratio d/R (default 0.001)")
    ap.add_argument("--dmax", type=float, default=None, help="indent: last depth ratio d/R (default 0.05)")
    ap.add_argument("--stop-on-fail", action="store_true")
    ap.add_argument("--learned", action="store_true",
                    help="indentation: increments after the first start from the warm-start network's guess")
    a = ap.parse_args(argv)
    if a.workload == "batch":
        return run_batch(a, dtt.PREC_MIXED if a.precision == "mixed" else dtt.PREC_FP64)
    wname = "ct_paper:" + a.ct_load if a.workload == "ct_paper" else a.workload
    if a.workload == "iso_cell":
        wname = "iso_cell:%d" % a.seed0
    if a.workload == "indent_inclusions":
        wname = "indent_inclusions:%d" % a.seed0
    spec = make_workload(wname, tuple(int(v) for v in a.nvox.split(",")) if a.nvox else None, a.load_steps,
                         a.contrast, a.radius, a.dmin, a.dmax)
    prec = dtt.PREC_MIXED if a.precision == "mixed" else dtt.PREC_FP64
    spec["kinematics"] = a.kinematics.upper()
    if a.medium:
        spec["medium"] = a.medium
    if a.scheme:
        spec["scheme"] = wl.TETRA2 if a.scheme == "tetra2" else wl.HEX1
    spec["lam0"] = a.r0_scale * spec["lam0"]
    spec["mu0"] = a.r0_scale * spec["mu0"]
    g = rows.setup_grid(spec, prec)
    tol = 0.0 if a.iters > 0 else (spec["tol"] if a.tol is None else a.tol)
    max_iter = a.iters if a.iters > 0 else a.max_iter
    ind = spec.get("indenter")
    nsteps = min(a.steps, len(ind["centers"])) if ind else 1
    if ind:
        g.dtt_set_indenter(ind["axis"], ind["face"], ind["centers"][0], ind["radius"])
    tuning = None
    if a.tune:
        t = g.dtt_autotune(iters=4, acv_mod=a.acv_mod or spec["acv_mod"])
        tuning = {"residual_zchunk": t.residual_zchunk, "fft_generic": t.fft_generic, "z_route": t.z_route,
                  "fft_warp": t.fft_warp, "ms_per_iteration": t.ms_per_iteration}
    net, hist = None, {}
    if a.learned and ind:
        import torch
        from paper_2607_26082_b300 import warmstart
        net = warmstart.load_net(os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights",
                                              "warmstart_indent.npz"))
        dk = [float(r) * float(ind["radius"]) for r in ind["ratios"]]
        hist = {"u1": torch.empty((3,) + tuple(g.node_shape), dtype=torch.float64, device="cuda"), "u2": None}
    for s in range(nsteps):
        if ind:
            g.dtt_move_indenter(ind["centers"][s])
        init = dtt.INIT_PREVIOUS if s else dtt.INIT_ZERO
        if net is not None and s > 0:
            # the guess from u~ of the last two increments and the grid's own reactions
            g.dtt_get_fields(u_out=hist["u1"])
            net.predict_increment(g, hist["u2"], None, (dk[s - 2] if s >= 2 else 0.0, dk[s - 1], dk[s]))
            init = dtt.INIT_GUESS
        reps_ms = []
        for _ in range(max(1, a.repeat) if (a.iters > 0 and s == 0) else 1):
            rep = g.dtt_solve_step(tol, max_iter, acv_mod=a.acv_mod or spec["acv_mod"],
                                   acv_on=dtt.ACV_P if a.acv_on == "p" else dtt.ACV_U,
                                   init=init, graph_iters=a.graph_iters)
            reps_ms.append(1e3 * rep.seconds / max(rep.iterations, 1))
        if net is not None and s > 0:
            if hist["u2"] is None:
                hist["u2"] = torch.empty_like(hist["u1"])
            hist["u2"], hist["u1"] = hist["u1"], hist["u2"]
        out = {"workload": spec["name"], "precision": a.precision, "kinematics": a.kinematics, "step": s,
               "medium": spec.get("medium", "paux"), "scheme": "tetra2" if spec["scheme"] == wl.TETRA2 else "hex1",
               "acv_on": a.acv_on, "acv_mod": a.acv_mod or spec["acv_mod"]}
        if tuning:
            out["tuning"] = tuning
        if len(reps_ms) > 1:
            out["repeat_ms_per_iteration"] = reps_ms
        out.update(rep.as_dict())
        if "ligament_rows" in spec and g.n_rows:
            per, _ = g.dtt_get_reactions(g.n_rows)
            nl = spec["ligament_rows"]
            r_l, r_s = float(per[:nl].sum()), float(per[nl:].sum())
            out.update({"reaction_ligament": r_l, "reaction_load": r_s,
                        "balance": abs(r_l + r_s) / max(abs(r_l), 1e-300)})
        if ind:
            # contact force on the sphere and the Hertz value (Eq. 30) at this depth
            act, gap, fn, force = g.dtt_get_contact()
            d = float(ind["ratios"][s]) * ind["radius"]
            Es = ind["E"] / (1.0 - ind["nu"] ** 2)
            out.update({"depth": d, "d_over_R": float(ind["ratios"][s]), "contact_nodes": int(np.sum(act)),
                        "force": float(np.linalg.norm(force)),
                        "hertz": 4.0 / 3.0 * Es * np.sqrt(ind["radius"]) * d ** 1.5,
                        "min_det_F": g.dtt_get_min_jacobian()})
        print(json.dumps(out), flush=True)
        if a.stop_on_fail and rep.status != dtt.OK:
            break
    g.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
