"""Learned warm start: training data from batched solves, training, evaluation.

The training set is produced by the solver itself: many cells are solved together with
dtt_batch_solve and their converged u~ are the targets.  Training calls dtt_net_train_step
(one Adam step per cell, the forward and backward passes in the library's BF16 tensor-core
kernels).  Evaluation solves each held-out cell twice, from u~ = 0 and from the network's
guess with init = INIT_GUESS (which keeps the guess only if its first Eq. 5 residual is
below the plain start's), and reports iterations, starting residuals and times.
"""
import json
import time

import numpy as np

from . import dtt, rows, shard
from .net import Net


def solve_targets(specs, precision=dtt.PREC_MIXED, tol=1e-6, graph_iters=16):
    """Configured grids and their converged u~ (one dtt_batch_solve over all specs)."""
    grids = [rows.setup_grid(s, precision) for s in specs]
    st, reps = dtt.dtt_batch_solve(grids, tol, 20000, acv_mod=2, graph_iters=graph_iters)
    ok = [r.status == dtt.OK for r in reps]
    targets = [g.dtt_get_fields() if k else None for g, k in zip(grids, ok)]
    return grids, targets, reps


def train(net, grids, targets, epochs=30, lr=2e-3, seed=0, log=None):
    """Adam over the cells in a fresh random order each epoch; returns the mean loss per epoch."""
    rng = np.random.default_rng(seed)
    idx = [i for i, t in enumerate(targets) if t is not None]
    hist = []
    for ep in range(epochs):
        rng.shuffle(idx)
        losses = [net.train_step(grids[i], targets[i], lr) for i in idx]
        hist.append(float(np.mean(losses)))
        if log:
            log(ep, hist[-1])
    return hist


def train_data_parallel(net, grids, targets, epochs=30, lr=2e-3, seed=0, group=None, log=None):
    """train across ranks (one GPU each): grids and targets are this rank's own cells (from
    solve_targets), and every step sums the ranks' gradients of one cell each with one
    all-reduce before the same Adam step on every rank (shard.train_data_parallel).  Returns
    the mean loss over all ranks' cells per epoch."""
    import torch
    idx = [i for i, t in enumerate(targets) if t is not None]
    grad = torch.zeros(net.num_params, dtype=torch.float32, device=torch.device("cuda", torch.cuda.current_device()))
    return shard.train_data_parallel(len(idx), lambda j, gbuf: net.grad_step(grids[idx[j]], targets[idx[j]], gbuf),
                                     net.apply_grad, grad, epochs, lambda ep: lr, seed=seed, group=group, log=log)


def evaluate(net, specs, precision=dtt.PREC_MIXED, tol=1e-6, graph_iters=16):
    """Per cell: plain start vs network guess (INIT_GUESS)."""
    out = []
    for s in specs:
        g = rows.setup_grid(s, precision)
        t0 = time.perf_counter()
        r0 = g.dtt_solve_step(tol, 20000, acv_mod=s["acv_mod"], init=dtt.INIT_ZERO, graph_iters=graph_iters)
        t_zero = time.perf_counter() - t0
        h0 = g.dtt_get_history()
        t0 = time.perf_counter()
        net.predict(g)
        r1 = g.dtt_solve_step(tol, 20000, acv_mod=s["acv_mod"], init=dtt.INIT_GUESS, graph_iters=graph_iters)
        t_guess = time.perf_counter() - t0
        out.append({"name": s["name"], "zero_iters": r0.iterations, "zero_r0": float(h0[0]) if len(h0) else None,
                    "zero_status": r0.status, "zero_s": t_zero, "guess_iters": r1.iterations,
                    "guess_r0": r1.start_residual, "guess_used": r1.start_from_guess, "guess_status": r1.status,
                    "guess_s": t_guess})
        g.close()
    return out


def make_net(seed=0, channels=(16, 32, 64)):
    return Net(*channels, seed=seed)


# ---------------------------------------------------------------------------------------
# Increment mode: the warm start of the load increments of a sphere indentation
# (include/dtt_net.h).  Training data are the solver's own converged increments of
# training seeds; the network learns the correction to the secant prediction of each
# increment and the increment's contact pressure, whose sign sets the initial contact zone.
# ---------------------------------------------------------------------------------------
def depths(spec):
    """Indentation depth d_k of every increment (voxels)."""
    I = spec["indenter"]
    return [float(r) * float(I["radius"]) for r in I["ratios"]]


def depth_triple(dk, k):
    """(d_(k-2), d_(k-1), d_k), with d_(-1) = 0 (the unloaded state)."""
    return (dk[k - 2] if k >= 2 else 0.0, dk[k - 1], dk[k])


def contact_reactions(g):
    """Normal reactions of the last solve on its contact set, zero elsewhere (the library
    reports f_n = -W h^3 (p . n) at every surface node; off the set that is the residual of
    a free node, of either sign)."""
    act, _, fn, _ = g.dtt_get_contact()
    return np.where(act.astype(bool), fn, 0.0)


def solve_increments(spec, precision=dtt.PREC_MIXED, tol=1e-6, graph_iters=16, keep=True, store_dtype=None):
    """Solves every increment of an indentation from the previous one; returns the grid,
    the converged fields (CUDA tensors, float32 unless store_dtype says otherwise) and the
    normal reactions of each increment (CUDA float64), and the reports."""
    import torch
    I = spec["indenter"]
    g = rows.setup_grid(spec, precision)
    g.dtt_set_indenter(I["axis"], I["face"], I["centers"][0], I["radius"])
    dev = torch.device("cuda", torch.cuda.current_device())
    U, FN, reps = [], [], []
    u = torch.empty((3,) + tuple(g.node_shape), dtype=torch.float64, device=dev)
    for k, O in enumerate(I["centers"]):
        g.dtt_move_indenter(O)
        r = g.dtt_solve_step(tol, 20000, acv_mod=spec["acv_mod"], init=dtt.INIT_ZERO if k == 0 else dtt.INIT_PREVIOUS,
                             graph_iters=graph_iters)
        reps.append(r)
        if keep:
            g.dtt_get_fields(u_out=u)
            U.append(u.to(store_dtype or torch.float32).clone())
            FN.append(torch.from_numpy(contact_reactions(g)).to(dev))
    torch.cuda.current_stream().synchronize()
    return g, U, FN, reps


def train_increments(net, data, epochs=8, lr=1e-3, seed=0, log=None, k_first=2, last=None):
    """Adam over the increments k >= k_first of the training seeds, in a fresh random order
    each epoch, the step size halved every quarter of the epochs.  data: list of (grid,
    spec, U, FN) from solve_increments.  The second increment (k = 1) extrapolates from the
    unloaded state and its correction targets are an order of magnitude larger than the
    others'; by default it is left out.  Returns the median loss per epoch (a few
    increments whose contact zone jumps carry losses far above the rest); `last`, a dict,
    receives the last epoch's loss per (seed index, k)."""
    import torch
    rng = np.random.default_rng(seed)
    items = [(i, k) for i, (_, spec, U, _) in enumerate(data) for k in range(k_first, len(U))]
    hist = []
    for ep in range(epochs):
        rng.shuffle(items)
        lr_ep = lr * 0.5 ** (4 * ep // max(epochs, 1))
        losses = []
        for i, k in items:
            g, spec, U, FN = data[i]
            dk = depths(spec)
            g.dtt_move_indenter(spec["indenter"]["centers"][k])
            u1 = U[k - 1].double().contiguous()
            u2 = U[k - 2].double().contiguous() if k >= 2 else None
            ut = U[k].double().contiguous()
            # the library works on its own streams: the conversions above (torch's stream)
            # must be complete before it reads them
            torch.cuda.current_stream().synchronize()
            g.dtt_set_initial(u1)
            losses.append(net.train_increment(g, u2, FN[k - 1], depth_triple(dk, k), ut, FN[k], lr_ep))
            if last is not None and ep == epochs - 1:
                last[(i, k)] = losses[-1]
            del u1, u2, ut
        hist.append(float(np.median(losses)))
        if log:
            log(ep, hist[-1])
        torch.cuda.empty_cache()
    return hist


def lr_schedule(lr, epochs):
    """Step size of an epoch: lr, halved every quarter of the epochs (train_increments')."""
    return lambda ep: lr * 0.5 ** (4 * ep // max(epochs, 1))


def train_increments_data_parallel(net, data, epochs=8, lr=1e-3, seed=0, k_first=2, group=None, log=None):
    """train_increments across ranks (one GPU each): data holds this rank's own seeds (from
    solve_increments), and every step sums the ranks' gradients of one increment each with
    one all-reduce of the network's num_params float32 gradient (NCCL between GPUs) before
    the same Adam step on every rank (shard.train_data_parallel).  On one rank it visits the
    increments in shard.local_order and is train_increment called in that order.  Returns the mean loss over all ranks' increments per epoch."""
    import torch
    items = [(i, k) for i, (_, spec, U, _) in enumerate(data) for k in range(k_first, len(U))]
    dev = torch.device("cuda", torch.cuda.current_device())
    grad = torch.zeros(net.num_params, dtype=torch.float32, device=dev)

    def grad_fn(j, gbuf):
        i, k = items[j]
        g, spec, U, FN = data[i]
        g.dtt_move_indenter(spec["indenter"]["centers"][k])
        u1 = U[k - 1].double().contiguous()
        u2 = U[k - 2].double().contiguous() if k >= 2 else None
        ut = U[k].double().contiguous()
        torch.cuda.current_stream().synchronize()
        g.dtt_set_initial(u1)
        return net.grad_increment(g, u2, FN[k - 1], depth_triple(depths(spec), k), ut, FN[k], gbuf)

    hist = shard.train_data_parallel(len(items), grad_fn, net.apply_grad, grad, epochs, lr_schedule(lr, epochs),
                                     seed=seed, group=group, log=log)
    return hist, items


def secant_start(U, FN, dk, k):
    """The start without the network: the secant prediction of increment k (the step of
    the previous increment scaled like the Hertz force, d^(3/2)) and the previous
    increment's contact zone {f_n < 0}."""
    import torch
    d2, d1, d0 = depth_triple(dk, k)
    s = (d0 ** 1.5 - d1 ** 1.5) / (d1 ** 1.5 - d2 ** 1.5)
    u2 = U[k - 2] if k >= 2 else torch.zeros_like(U[k - 1])
    return U[k - 1] + s * (U[k - 1] - u2), (FN[k - 1] < 0).to(torch.uint8)


def evaluate_increments(net, spec, tol=1e-6, graph_iters=16, ks=None):
    """Per increment k >= 1 of a held-out seed, three starts from the same field of
    increment k-1 (the plain run's): the plain previous-step start of Algorithm 2, the
    secant start without the network (secant_start), and the network's guess (INIT_GUESS,
    falling back to the previous-step field).  Returns one dict per increment."""
    import torch
    g, U, FN, reps = solve_increments(spec, tol=tol, graph_iters=graph_iters, store_dtype=torch.float64)
    I = spec["indenter"]
    dk = depths(spec)
    out = []
    for k in (ks or range(1, len(U))):
        g.dtt_move_indenter(I["centers"][k])
        g.dtt_set_initial(U[k - 1])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        net.predict_increment(g, U[k - 2] if k >= 2 else None, FN[k - 1], depth_triple(dk, k))
        r = g.dtt_solve_step(tol, 20000, acv_mod=spec["acv_mod"], init=dtt.INIT_GUESS, graph_iters=graph_iters)
        t_guess = time.perf_counter() - t0
        us, act = secant_start(U, FN, dk, k)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g.dtt_set_initial(us)
        g.dtt_set_initial_contact(act)
        rs = g.dtt_solve_step(tol, 20000, acv_mod=spec["acv_mod"], init=dtt.INIT_PREVIOUS, graph_iters=graph_iters)
        t_sec = time.perf_counter() - t0
        del us, act
        out.append({"k": k, "plain_iters": reps[k].iterations, "plain_s": reps[k].seconds,
                    "plain_updates": reps[k].active_set_updates, "guess_iters": r.iterations, "guess_s": t_guess,
                    "guess_updates": r.active_set_updates, "guess_used": r.start_from_guess,
                    "guess_r0": r.start_residual, "status": r.status, "secant_iters": rs.iterations,
                    "secant_s": t_sec, "secant_status": rs.status})
    g.close()
    return out


def save_net(net, path, meta=None):
    import os
    os.makedirs(os.path.dirname(path), exist_ok=True)
    np.savez_compressed(path, params=net.get_params(), channels=np.array(net.channels),
                        meta=np.array(json.dumps(meta or {})))


def load_net(path, stream=None):
    z = np.load(path)
    c = [int(v) for v in z["channels"]]
    net = Net(*c, seed=0, stream=stream)
    net.set_params(z["params"])
    meta = json.loads(str(z["meta"])) if "meta" in z else {}
    net.set_increment(float(meta.get("pressure_weight", 1.0)), float(meta.get("active_threshold", 0.05)),
                      int(meta.get("window_lateral", 0)), int(meta.get("window_depth", 0)))
    net.meta = meta
    return net


def main(argv=None):
    """python -m paper_2607_26082_b300.warmstart train-indent --seeds 2000:2006 [--nvox 384,384,192]
    [--epochs 60] [--lr 1e-3] [--out paper_2607_26082_b300/weights/warmstart_indent.npz]
    [--eval-seed 3000]

    Under torchrun (WORLD_SIZE > 1, one GPU per rank) the seeds are dealt round-robin to the
    ranks, each rank solves its own, and training is data-parallel (one NCCL all-reduce of
    the gradient per step, train_increments_data_parallel); rank 0 saves and evaluates."""
    import argparse
    import os
    import sys
    import torch
    import workloads as wl
    ap = argparse.ArgumentParser()
    ap.add_argument("cmd", choices=["train-indent"])
    ap.add_argument("--seeds", default="2000:2006")
    ap.add_argument("--nvox", default="384,384,192")
    ap.add_argument("--epochs", type=int, default=60)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--pressure-weight", type=float, default=1.0)
    ap.add_argument("--threshold", type=float, default=0.05)
    ap.add_argument("--window", default="128,48", help="lateral,depth node extents of the network's window "
                                                       "(0,0: the whole grid)")
    ap.add_argument("--out", default=os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights",
                                                  "warmstart_indent.npz"))
    ap.add_argument("--eval-seed", type=int, default=3000)
    ap.add_argument("--seed", type=int, default=1, help="initial weights")
    a = ap.parse_args(argv)
    nv = tuple(int(v) for v in a.nvox.split(","))
    s0, s1 = (int(v) for v in a.seeds.split(":"))
    rank, world, local = shard.rank_world()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    t0 = time.perf_counter()
    data, mine = [], list(range(s0, s1))[rank::world]
    for sd in mine:
        spec = wl.indentation_inclusions(sd, *nv, steps=20)
        g, U, FN, reps = solve_increments(spec)
        data.append((g, spec, U, FN))
        print(json.dumps({"seed": sd, "iterations": sum(r.iterations for r in reps),
                          "s": round(time.perf_counter() - t0, 1)}), flush=True)
    net = make_net(seed=a.seed)
    wl_, wd_ = (int(v) for v in a.window.split(","))
    net.set_increment(a.pressure_weight, a.threshold, wl_, wd_)
    if world > 1:
        hist, _ = train_increments_data_parallel(
            net, data, epochs=a.epochs, lr=a.lr,
            log=lambda ep, l: rank == 0 and print(json.dumps({"epoch": ep, "mean_loss": l, "ranks": world,
                                                              "s": round(time.perf_counter() - t0, 1)}), flush=True))
    else:
        last = {}
        hist = train_increments(net, data, epochs=a.epochs, lr=a.lr, last=last,
                                log=lambda ep, l: print(json.dumps({"epoch": ep, "median_loss": l,
                                                                    "s": round(time.perf_counter() - t0, 1)}),
                                                        flush=True))
        worst = sorted(last.items(), key=lambda kv: -kv[1])[:5]
        print(json.dumps({"largest_last_epoch_losses": [[s0 + i, k, v] for (i, k), v in worst]}), flush=True)
    for g, _, _, _ in data:
        g.close()
    del data
    torch.cuda.empty_cache()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
        if rank != 0:
            return 0
    meta = {"seeds": a.seeds, "nvox": nv, "epochs": a.epochs, "lr": a.lr, "pressure_weight": a.pressure_weight,
            "active_threshold": a.threshold, "window_lateral": wl_, "window_depth": wd_, "loss": hist}
    save_net(net, a.out, meta)
    ev = evaluate_increments(net, wl.indentation_inclusions(a.eval_seed, *nv, steps=20))
    for e in ev:
        print(json.dumps(e), flush=True)
    print(json.dumps({"eval_seed": a.eval_seed, "plain_iters": sum(e["plain_iters"] for e in ev),
                      "secant_iters": sum(e["secant_iters"] for e in ev),
                      "guess_iters": sum(e["guess_iters"] for e in ev), "plain_s": sum(e["plain_s"] for e in ev),
                      "secant_s": sum(e["secant_s"] for e in ev),
                      "guess_s": sum(e["guess_s"] for e in ev), "kept": sum(e["guess_used"] for e in ev)}), flush=True)
    return 0


if __name__ == "__main__":
    import sys
    sys.exit(main())
