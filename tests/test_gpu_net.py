"""Warm-start network on the GPU: BF16 tensor-core forward / backward against the float64
reference (oracle/net.py), input features against the reference, the INIT_GUESS fallback
rule, and what a trained network gains on held-out cells."""
import numpy as np
import pytest

import workloads as wl
from helpers import gpu_grid
from oracle import net as onet

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2607_26082_b300 import dtt, warmstart  # noqa: E402
from paper_2607_26082_b300.net import Net  # noqa: E402


def bf16_round(a):
    """Round float values to bfloat16 (nearest, ties to even), returned as float64."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


@pytest.mark.parametrize("shape,ch,w", [((11, 7, 9), (16, 32, 64), 0.0), ((6, 10, 5), (32, 16, 32), 0.05)])
def test_net_forward_and_gradients_match_reference(shape, ch, w):
    """Tolerances: activations and back-propagated gradients are BF16 tensor-core operands
    (relative rounding 2^-9 per value), through eleven layers in sequence."""
    net = Net(*ch, seed=3)
    net.set_loss(w)
    p = net.get_params()
    rng = np.random.default_rng(4)
    x = rng.standard_normal(shape + (16,)).astype(np.float32)
    t = rng.standard_normal(shape + (3,)).astype(np.float32)
    loss, g = net.loss_grad(x, t)
    y = net.forward(x)
    # the reference takes the same BF16-rounded weights and inputs; what remains is the
    # BF16 rounding of the activations between layers
    layers = onet.unpack(p, *ch)
    layers = [(bf16_round(W), b.astype(np.float64)) for W, b in layers]
    rloss, rgrads, ry = onet.loss_grad(layers, bf16_round(x), t.astype(np.float64), w)
    assert _rel(y, ry[..., :3]) <= 3e-2
    assert abs(loss - rloss) <= 3e-2 * rloss
    gref = onet.pack(rgrads)
    off = 0
    for (ci, co), (gW, gb) in zip(onet.layer_shapes(*ch), rgrads):
        n = 27 * ci * co
        assert _rel(g[off:off + n], gW.ravel()) <= 1e-1, (ci, co)
        off += n
        assert _rel(g[off:off + co], gb) <= 1e-1, (ci, co)
        off += co
    assert off == gref.size
    net.close()


def test_net_features_match_reference():
    net = Net(seed=0)
    for seed in (4400, 4401, 4402):
        c = wl.batch_cell(seed, sizes=(8, 12))
        g = gpu_grid(c, dtt.PREC_MIXED)
        x = net.features(g)
        ref = onet.features(c)
        assert np.abs(x - ref).max() <= 1e-6
        g.close()
    net.close()


def test_guess_fallback_keeps_the_plain_start():
    """An untrained network's guess is rejected when its first residual is worse; the solve
    is then the plain one, iteration for iteration."""
    net = Net(seed=11)
    c = wl.batch_cell(4500, sizes=(16,))
    g0 = gpu_grid(c, dtt.PREC_MIXED)
    r0 = g0.dtt_solve_step(1e-6, 4000, acv_mod=2)
    g = gpu_grid(c, dtt.PREC_MIXED)
    # a deliberately bad guess: the network output scaled far up
    net.predict(g)
    u = g.dtt_get_fields() * 1e3
    g.dtt_set_initial(u)
    r = g.dtt_solve_step(1e-6, 4000, acv_mod=2, init=dtt.INIT_GUESS)
    assert r.start_from_guess == 0
    assert r.iterations == r0.iterations
    assert np.array_equal(g.dtt_get_fields(), g0.dtt_get_fields())
    for q in (g0, g):
        q.close()
    net.close()


def test_trained_warm_start_on_held_out_cells():
    """Train on 32 solver-produced cells, evaluate on 8 held-out cells.  The guess may only
    be kept when its first Eq. 5 residual is below the plain start's (never a worse
    start); the measured effect on iteration counts is printed (it is small on this
    workload: the plain start's residual is set by interface and free-face forces, which a
    network trained on 32 cells does not resolve well enough to beat)."""
    train_specs = [wl.batch_cell(5000 + i, sizes=(12, 16)) for i in range(32)]
    test_specs = [wl.batch_cell(6000 + i, sizes=(12, 16)) for i in range(8)]
    grids, targets, reps = warmstart.solve_targets(train_specs, tol=1e-6)
    assert sum(r.status == dtt.OK for r in reps) >= len(reps) - 1
    net = warmstart.make_net(seed=1)
    hist = warmstart.train(net, grids, targets, epochs=40, lr=3e-3, seed=0)
    assert hist[-1] < hist[0]
    res = warmstart.evaluate(net, test_specs)
    for r in res:
        assert r["zero_status"] == dtt.OK and r["guess_status"] == dtt.OK
        assert r["guess_r0"] <= r["zero_r0"] * (1 + 1e-12)
    zi = np.mean([r["zero_iters"] for r in res])
    gi = np.mean([r["guess_iters"] for r in res])
    used = sum(r["guess_used"] for r in res)
    print("warm start: loss %.4f -> %.4f; guess kept on %d/%d cells; mean iterations %.1f -> %.1f"
          % (hist[0], hist[-1], used, len(res), zi, gi))
    assert gi <= 1.05 * zi
    for q in grids:
        q.close()
    net.close()


def bf16_weights(p, ch):
    return [(bf16_round(W), b) for W, b in onet.unpack(p, *ch)]


@pytest.mark.parametrize("ch", [(16, 32, 64), (32, 16, 32)])
def test_net_layers_match_reference_one_by_one(ch):
    """Every layer on its own: given the layer's input activation and its output gradient
    as the GPU kernels used them (BF16 values), the float64 reference's weight, bias and
    input gradients (with the BF16-rounded weights) agree to 1e-4: the products of BF16
    operands are exact in FP32, so only the order of the FP32 sums remains.  A wrong tap, a
    transposed weight or a shifted index in any layer is an O(1) error here."""
    net = Net(*ch, seed=3)
    rng = np.random.default_rng(5)
    shape = (11, 7, 9)
    x = rng.standard_normal(shape + (16,)).astype(np.float32)
    t = rng.standard_normal(shape + (3,)).astype(np.float32)
    layers = bf16_weights(net.get_params(), ch)
    for l in range(11):
        a, dz, gw, gb, gx = net.layer_trace(x, t, l)
        assert np.abs(dz).max() > 0, l
        rgx, rgW, rgb = onet.conv_backward(a.astype(np.float64), layers[l][0], dz.astype(np.float64))
        assert _rel(gw, rgW) <= 1e-4, l
        assert _rel(gb, rgb) <= 1e-4, l
        if l > 0:
            assert _rel(gx, rgx) <= 1e-4, l
    # the first layer's input is the BF16-rounded features
    a0 = net.layer_trace(x, t, 0)[0]
    assert np.array_equal(a0, bf16_round(x).astype(np.float32))
    net.close()
