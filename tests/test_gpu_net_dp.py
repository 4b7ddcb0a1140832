"""Data-parallel training of the warm start on the GPU: the two halves of
dtt_net_train_increment (dtt_net_grad_increment, dtt_net_apply_grad) and of
dtt_net_train_step (dtt_net_grad_step, dtt_net_apply_grad) give their parameters,
the gradient scale of apply_grad is exact for powers of two, the single-rank data-parallel
loop equals train_increment calls in the same order, and the entry points reject host
pointers and bad scales without launching anything.  The all-reduce between ranks is
covered by the two-rank gloo tests of tests/test_shard.py.

The weight-gradient kernels sum their tiles' partial products with float atomics, so two
evaluations of the same gradient agree only up to the order of those sums (about 1e-7
relative): runs are compared through the change of the parameters, where a differing
element is one whose gradient is at that noise level (Adam's first steps move every
parameter by about lr, whatever the gradient's size)."""
import ctypes as C

import numpy as np
import pytest

import workloads as wl

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2607_26082_b300 import dtt, shard, warmstart  # noqa: E402
from paper_2607_26082_b300.net import Net, _lib  # noqa: E402


@pytest.fixture(scope="module")
def increments():
    spec = wl.indentation_inclusions(11, 48, 40, 24, steps=6)
    g, U, FN, reps = warmstart.solve_increments(spec)
    assert all(r.status == dtt.OK for r in reps)
    yield [(g, spec, U, FN)]
    g.close()


def _net():
    net = Net(16, 32, 64, seed=5)
    net.set_increment(1.0, 0.05, 24, 10)
    return net


def _args(data, k):
    g, spec, U, FN = data[0]
    g.dtt_move_indenter(spec["indenter"]["centers"][k])
    u1 = U[k - 1].double().contiguous()
    u2 = U[k - 2].double().contiguous() if k >= 2 else None
    ut = U[k].double().contiguous()
    torch.cuda.synchronize()
    g.dtt_set_initial(u1)
    return g, u2, FN[k - 1], warmstart.depth_triple(warmstart.depths(spec), k), ut, FN[k]


def _same_steps(pa, pb, p0):
    """pa and pb are the same training run up to the atomics' summation order."""
    assert np.linalg.norm(pa - pb) <= 2e-2 * np.linalg.norm(pa - p0)
    assert np.mean(np.abs(pa - pb) > 1e-6) <= 1e-3


def test_grad_then_apply_is_train_increment(increments):
    a, b = _net(), _net()
    p0 = a.get_params()
    grad = torch.full((a.num_params,), float("nan"), dtype=torch.float32, device="cuda")
    again = torch.zeros_like(grad)
    for k, lr in ((2, 1e-3), (3, 5e-4), (4, 1e-3)):
        la = a.train_increment(*_args(increments, k), lr)
        lb = b.grad_increment(*_args(increments, k), grad)
        assert abs(la - lb) <= 1e-5 * abs(la)
        assert bool(torch.isfinite(grad).all())
        if k == 2:
            # the gradient call leaves the parameters as they were, and a second call gives
            # the same gradient up to the atomics' order
            np.testing.assert_array_equal(b.get_params(), p0)
            b.grad_increment(*_args(increments, k), again)
            assert float(torch.linalg.norm(again - grad)) <= 1e-5 * float(torch.linalg.norm(grad))
        b.apply_grad(grad, 1.0, lr)
        _same_steps(a.get_params(), b.get_params(), p0)
    a.close()
    b.close()


def test_apply_grad_scale(increments):
    """A summed gradient 2 g with scale 1/2 is g exactly: the same step."""
    a, b = _net(), _net()
    grad = torch.zeros(a.num_params, dtype=torch.float32, device="cuda")
    a.grad_increment(*_args(increments, 3), grad)
    a.apply_grad(grad, 1.0, 1e-3)
    two = grad * 2.0
    b.apply_grad(two, 0.5, 1e-3)
    np.testing.assert_array_equal(a.get_params(), b.get_params())
    a.close()
    b.close()


def test_single_rank_data_parallel_loop_equals_train_increment(increments):
    epochs, lr, seed = 2, 1e-3, 4
    a, b = _net(), _net()
    p0 = a.get_params()
    hist, items = warmstart.train_increments_data_parallel(a, increments, epochs=epochs, lr=lr, seed=seed)
    lr_at = warmstart.lr_schedule(lr, epochs)
    ref = []
    for ep in range(epochs):
        losses = [b.train_increment(*_args(increments, items[j][1]), lr_at(ep))
                  for j in shard.local_order(seed, ep, 0, len(items))]
        ref.append(float(np.mean(losses)))
    _same_steps(a.get_params(), b.get_params(), p0)
    np.testing.assert_allclose(hist, ref, rtol=1e-3)
    a.close()
    b.close()


def test_grad_entry_points_reject_host_memory_and_bad_scales(increments):
    net = _net()
    host = np.zeros(net.num_params, np.float32)
    hp = C.c_void_p(host.ctypes.data)
    assert _lib().dtt_net_apply_grad(net._h, hp, C.c_float(1.0), C.c_float(1e-3)) == dtt.ERR_ARG
    g, u2, fn1, d, ut, fnt = _args(increments, 2)
    dd = np.ascontiguousarray(d, dtype=np.float64)
    loss = C.c_double()
    st = _lib().dtt_net_grad_increment(net._h, g._h, C.c_void_p(u2.data_ptr()), C.c_void_p(fn1.data_ptr()),
                                       dd.ctypes.data_as(C.c_void_p), C.c_void_p(ut.data_ptr()),
                                       C.c_void_p(fnt.data_ptr()), hp, C.byref(loss))
    assert st == dtt.ERR_ARG
    dev = torch.zeros(net.num_params, dtype=torch.float32, device="cuda")
    p0 = net.get_params()
    for scale in (0.0, -1.0, float("inf"), float("nan")):
        with pytest.raises(dtt.DttError):
            net.apply_grad(dev, scale, 1e-3)
    np.testing.assert_array_equal(net.get_params(), p0)
    net.close()


def test_cell_mode_grad_then_apply_is_train_step():
    """The cell mode's split (dtt_net_grad_step, dtt_net_apply_grad) against
    dtt_net_train_step, and its single-rank data-parallel loop against train_step calls in
    the same order, on solver-produced cells."""
    specs = [wl.batch_cell(5000 + i, sizes=(12, 16)) for i in range(3)]
    grids, targets, reps = warmstart.solve_targets(specs, tol=1e-6)
    assert all(t is not None for t in targets)
    a, b = Net(16, 32, 64, seed=9), Net(16, 32, 64, seed=9)
    p0 = a.get_params()
    grad = torch.zeros(a.num_params, dtype=torch.float32, device="cuda")
    for i, lr in ((0, 2e-3), (1, 1e-3), (2, 2e-3)):
        la = a.train_step(grids[i], targets[i], lr)
        lb = b.grad_step(grids[i], targets[i], grad)
        assert abs(la - lb) <= 1e-5 * abs(la)
        if i == 0:
            np.testing.assert_array_equal(b.get_params(), p0)
        b.apply_grad(grad, 1.0, lr)
        _same_steps(a.get_params(), b.get_params(), p0)
    c, d = Net(16, 32, 64, seed=9), Net(16, 32, 64, seed=9)
    hist = warmstart.train_data_parallel(c, grids, targets, epochs=2, lr=1e-3, seed=2)
    ref = []
    for ep in range(2):
        ref.append(float(np.mean([d.train_step(grids[j], targets[j], 1e-3) for j in shard.local_order(2, ep, 0, 3)])))
    _same_steps(c.get_params(), d.get_params(), p0)
    np.testing.assert_allclose(hist, ref, rtol=1e-3)
    for n in (a, b, c, d):
        n.close()
    for g in grids:
        g.close()
