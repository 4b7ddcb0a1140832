"""Warm start of the load increments of a sphere indentation (increment mode of
include/dtt_net.h) on the GPU: the increment loss and its gradients against the float64
reference (oracle/net.py), the increment features against the reference recipe on the
same seeded state, the fallback rule (a rejected guess reproduces the plain
previous-increment start bit for bit), and the gain of the trained network on a held-out
seed of the large indentation."""
import os

import numpy as np
import pytest

import workloads as wl
from oracle import net as onet

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2607_26082_b300 import dtt, rows, warmstart  # noqa: E402
from paper_2607_26082_b300.net import Net  # noqa: E402

WEIGHTS = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2607_26082_b300",
                       "weights", "warmstart_indent.npz")


def bf16_round(a):
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def test_increment_loss_gradients_match_reference():
    """BF16 tensor-core operands through eleven layers: the same tolerances as the
    displacement-only loss (3e-2 on the loss, 1e-1 per layer)."""
    net = Net(16, 32, 64, seed=3)
    net.set_increment(0.7, 0.05, 0, 0)
    p = net.get_params()
    rng = np.random.default_rng(6)
    shape = (7, 9, 11)
    x = rng.standard_normal(shape + (16,)).astype(np.float32)
    t = rng.standard_normal(shape + (4,)).astype(np.float32)
    m = np.zeros(shape, np.float32)
    m[-1] = 1.0
    loss, g = net.loss_grad_increment(x, t, m)
    layers = [(bf16_round(W), b) for W, b in onet.unpack(p, 16, 32, 64)]
    rloss, rgrads, _ = onet.increment_loss_grad(layers, bf16_round(x), t.astype(np.float64), m, 0.7)
    assert abs(loss - rloss) <= 3e-2 * rloss
    off = 0
    for (ci, co), (gW, gb) in zip(onet.layer_shapes(16, 32, 64), rgrads):
        n = 27 * ci * co
        assert _rel(g[off:off + n], gW.ravel()) <= 1e-1, (ci, co)
        off += n
        assert _rel(g[off:off + co], gb) <= 1e-1, (ci, co)
        off += co
    net.close()


def _small_indent():
    return wl.indentation_inclusions(11, 48, 40, 24, steps=6)


@pytest.mark.parametrize("window", [(0, 0), (24, 10)])
def test_increment_features_match_reference(window):
    """Seeded state (u~ of increments k-1 and k-2, previous reactions, depths, moved
    sphere) on a 48 x 40 x 24 block with inclusions; every feature channel against the
    reference recipe, on the whole grid and on a window (24 nodes across, 10 layers deep,
    centred under the sphere)."""
    spec = _small_indent()
    I = spec["indenter"]
    g = rows.setup_grid(spec, dtt.PREC_MIXED)
    g.dtt_set_indenter(I["axis"], I["face"], I["centers"][3], I["radius"])
    rng = np.random.default_rng(8)
    shape = (3,) + tuple(g.node_shape)
    u1 = 0.05 * rng.standard_normal(shape)
    u2 = 0.03 * rng.standard_normal(shape)
    for c in range(3):          # Dirichlet nodes (bottom face) hold zero
        u1[c, 0] = 0.0
        u2[c, 0] = 0.0
    nf = g.node_shape[1] * g.node_shape[2]
    fn = -np.abs(rng.standard_normal(nf))
    dev = torch.device("cuda", 0)
    g.dtt_set_initial(u1)
    depth = (0.4, 0.7, 1.1)
    net = Net(16, 32, 64, seed=0)
    net.set_increment(1.0, 0.05, *window)
    u2d, fnd = torch.from_numpy(u2).to(dev), torch.from_numpy(fn).to(dev)
    torch.cuda.synchronize()
    x = net.increment_features(g, u2d, fnd, depth)
    nz, ny, nx = g.node_shape
    surf = [(i, j, nz - 1) for j in range(ny) for i in range(nx)]
    # the mixed grid stores u~ as a float-float pair: read back what it holds
    u1g = g.dtt_get_fields()
    ref = onet.increment_features(onet.features(spec), u1g, u2, fn, depth, surf, I["centers"][3], I["radius"])
    if window[0]:
        lat, dep = window
        ox = min(max(int(round(I["centers"][3][0])) - lat // 2, 0), nx - lat)
        oy = min(max(int(round(I["centers"][3][1])) - lat // 2, 0), ny - lat)
        ref = ref[nz - dep:, oy:oy + lat, ox:ox + lat]
    assert x.shape == ref.shape
    assert np.abs(x[..., :4] - ref[..., :4]).max() <= 1e-6
    assert np.abs(x[..., 4:7] - ref[..., 4:7]).max() <= 1e-5 * np.abs(ref[..., 4:7]).max()
    assert np.array_equal(x[..., 7], ref[..., 7])
    assert np.abs(x[..., 8] - ref[..., 8]).max() <= 1e-5 * max(1.0, np.abs(ref[..., 8]).max())
    assert np.abs(x[..., 9] - ref[..., 9]).max() <= 1e-6
    assert np.abs(x[..., 10:] - ref[..., 10:]).max() <= 1e-6
    net.close()
    g.close()


def test_rejected_guess_reproduces_the_previous_increment_start():
    """An untrained network's guess is worse than the previous increment's field: the
    solve falls back to it (and its contact zone {g < 0}) and reproduces the plain solve
    bit for bit."""
    spec = _small_indent()
    g, U, FN, reps = warmstart.solve_increments(spec, store_dtype=torch.float64)
    I = spec["indenter"]
    dk = warmstart.depths(spec)
    k = 3
    net = Net(16, 32, 64, seed=5)
    g.dtt_move_indenter(I["centers"][k])
    g.dtt_set_initial(U[k - 1])
    net.predict_increment(g, U[k - 2], FN[k - 1], warmstart.depth_triple(dk, k))
    r = g.dtt_solve_step(1e-6, 20000, acv_mod=spec["acv_mod"], init=dtt.INIT_GUESS, graph_iters=16)
    assert r.start_from_guess == 0
    u_guess_path = g.dtt_get_fields()
    g.dtt_set_initial(U[k - 1])
    r2 = g.dtt_solve_step(1e-6, 20000, acv_mod=spec["acv_mod"], init=dtt.INIT_PREVIOUS, graph_iters=16)
    assert r.iterations == r2.iterations
    assert np.array_equal(u_guess_path, g.dtt_get_fields())
    net.close()
    g.close()


def test_prediction_reads_the_grids_own_reactions():
    """fn_prev = NULL: the prediction takes the grid's reactions of its last solve on that
    solve's contact set, on the device; the guess (field and initial zone) equals the one
    from the same reactions passed explicitly."""
    spec = _small_indent()
    g, U, FN, reps = warmstart.solve_increments(spec, store_dtype=torch.float64)
    I = spec["indenter"]
    dk = warmstart.depths(spec)
    k = 3
    net = Net(16, 32, 64, seed=7)
    # the grid's contact state becomes increment k-1's again (same start, same solve)
    g.dtt_move_indenter(I["centers"][k - 1])
    g.dtt_set_initial(U[k - 2])
    r = g.dtt_solve_step(1e-6, 20000, acv_mod=spec["acv_mod"], init=dtt.INIT_PREVIOUS, graph_iters=16)
    assert r.status == dtt.OK
    fn = torch.from_numpy(warmstart.contact_reactions(g)).cuda()
    u_prev = torch.from_numpy(g.dtt_get_fields()).cuda()
    g.dtt_move_indenter(I["centers"][k])
    net.predict_increment(g, U[k - 2], None, warmstart.depth_triple(dk, k))
    u_own, act_own = g.dtt_get_fields(), g.dtt_get_contact()[0].copy()
    g.dtt_set_initial(u_prev)
    net.predict_increment(g, U[k - 2], fn, warmstart.depth_triple(dk, k))
    assert np.array_equal(u_own, g.dtt_get_fields())
    assert np.array_equal(act_own, g.dtt_get_contact()[0])
    net.close()
    g.close()


def test_trained_network_gains_on_a_held_out_seed():
    """The committed network (trained on seeds 2000-2005 of the 384 x 384 x 192 indentation
    with inclusions; its contact-zone threshold chosen on seed 3000) on the held-out seed
    3001, every increment k >= 1 started three ways from the same field of increment k-1:
    the plain previous-increment start of Algorithm 2, the secant start without the
    network (Hertz-scaled secant, previous contact zone), and the network's guess with the
    fallback rule.  The learned start takes at most 80 % of the plain start's iterations and
    fewer than the secant start's."""
    assert os.path.exists(WEIGHTS), "trained warm-start weights missing"
    net = warmstart.load_net(WEIGHTS)
    spec = wl.indentation_inclusions(3001, 384, 384, 192, steps=20)
    ev = warmstart.evaluate_increments(net, spec)
    plain = sum(e["plain_iters"] for e in ev)
    secant = sum(e["secant_iters"] for e in ev)
    guess = sum(e["guess_iters"] for e in ev)
    assert all(e["status"] == dtt.OK and e["secant_status"] == dtt.OK for e in ev)
    assert guess <= 0.8 * plain, (guess, secant, plain)
    assert guess < secant, (guess, secant, plain)
    net.close()
