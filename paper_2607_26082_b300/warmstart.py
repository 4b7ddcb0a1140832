"""Learned warm start: training data from batched solves, training, evaluation.

The training set is produced by the solver itself: many cells are solved together with
dtt_batch_solve and their converged u~ are the targets.  Training calls dtt_net_train_step
(one Adam step per cell, the forward and backward passes in the library's BF16 tensor-core
kernels).  Evaluation solves each held-out cell twice, from u~ = 0 and from the network's
guess with init = INIT_GUESS (which keeps the guess only if its first Eq. 5 residual is
below the plain start's), and reports iterations, starting residuals and times.
"""
import time

import numpy as np

from . import dtt, rows
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
