"""Error behaviour of the C ABI on the host: argument checks that every entry point makes
before it touches the GPU return DTT_ERR_ARG with a message from dtt_last_error(), and on a
machine without a CUDA device a well-formed grid is refused with DTT_ERR_CUDA rather than
solved some other way (the library has no CPU fallback).  Nothing here launches a kernel."""
import ctypes as C

import numpy as np
import pytest

from paper_2607_26082_b300 import dtt

P = C.c_void_p
NULL = P()


def _last_error():
    return dtt.lib().dtt_last_error().decode()


def _create(nvox=(4, 4, 4), h=1.0, bc=None, scheme=dtt.SCHEME_TETRA2, prec=dtt.PREC_FP64, out=True):
    L = dtt.lib()
    h_out = P()
    nv = np.ascontiguousarray(nvox, dtype=np.int32)
    b = np.ascontiguousarray(np.ones(18) if bc is None else np.asarray(bc).reshape(18), dtype=np.int32)
    return L.dtt_grid_create(C.byref(h_out) if out else None, nv.ctypes.data_as(P), float(h), b.ctypes.data_as(P),
                             int(scheme), int(prec), None), h_out


@pytest.mark.parametrize("kw,msg", [
    (dict(out=False), "null"),
    (dict(h=0.0), "h must be > 0"),
    (dict(h=float("nan")), "h must be > 0"),
    (dict(scheme=7), "unknown scheme"),
    (dict(prec=5), "unknown precision"),
    (dict(nvox=(1, 4, 4)), "nvox"),
    (dict(nvox=(4, 4, 5000)), "nvox"),
    (dict(bc=[1] * 17 + [3]), "bc code"),
    (dict(bc=[-1] + [1] * 17), "bc code"),
])
def test_grid_create_rejects_bad_arguments(kw, msg):
    st, h = _create(**kw)
    assert st == dtt.ERR_ARG
    assert msg in _last_error()
    assert not h.value


def test_null_handles_are_rejected():
    L = dtt.lib()
    x = np.zeros(9)
    xp = x.ctypes.data_as(P)
    opts = dtt.SolveOpts(1e-6, 10, 3, dtt.ACV_P, dtt.INIT_ZERO, 1e-2, 0, 0.0)
    rep = dtt.Report()
    n = C.c_int32(1)
    calls = [
        L.dtt_set_material(NULL, xp, 1, xp, xp, 0),
        L.dtt_set_reference(NULL, 1.0, 1.0),
        L.dtt_set_load(NULL, xp),
        L.dtt_set_indenter(NULL, 2, 1, xp, 1.0),
        L.dtt_move_indenter(NULL, xp),
        L.dtt_set_initial(NULL, xp, 0),
        L.dtt_solve_step(NULL, C.byref(opts), C.byref(rep)),
        L.dtt_get_history(NULL, xp, C.byref(n)),
        L.dtt_get_fields(NULL, xp, None, 0),
        L.dtt_get_reactions(NULL, None, xp),
        L.dtt_apply_green(NULL, xp, xp, 0),
        L.dtt_apply_green_noalloc(NULL, xp, xp),
        L.dtt_transform(NULL, 0, 0, xp, xp, 0),
        L.dtt_batch_solve(0, None, C.byref(opts), C.byref(rep)),
    ]
    for k, st in enumerate(calls):
        assert st == dtt.ERR_ARG, (k, st, _last_error())
        assert _last_error()


def test_net_entry_points_reject_bad_arguments():
    from paper_2607_26082_b300.net import _lib
    L = _lib()
    out = P()
    assert L.dtt_net_create(C.byref(out), 16, 24, 64, 0, None) == dtt.ERR_ARG
    assert "channel" in _last_error() and not out.value
    assert L.dtt_net_apply_grad(NULL, NULL, C.c_float(1.0), C.c_float(1e-3)) == dtt.ERR_ARG
    loss = C.c_double()
    assert L.dtt_net_grad_step(NULL, NULL, NULL, NULL, C.byref(loss)) == dtt.ERR_ARG
    d = np.zeros(3)
    assert L.dtt_net_grad_increment(NULL, NULL, NULL, NULL, d.ctypes.data_as(P), NULL, NULL, NULL,
                                    C.byref(loss)) == dtt.ERR_ARG


def test_no_device_means_no_solve():
    """Without a CUDA device a valid grid is refused (DTT_ERR_CUDA), and the Python binding
    raises: the solver never falls back to the host."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    st, h = _create()
    assert st == dtt.ERR_CUDA and not h.value
    with pytest.raises(dtt.DttError) as e:
        dtt.Grid((4, 4, 4), 1.0, np.ones((3, 2, 3)))
    assert e.value.status == dtt.ERR_CUDA
