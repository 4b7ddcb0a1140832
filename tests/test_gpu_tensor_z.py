"""The fused z pass as two split-TF32 tensor-core contractions (tcgen05, accumulators in
tensor memory) against the float64 oracle and against the FFT z pass.

The z transform of each component is the dense product with its DTT matrix (Section
3.2.2, Table 3); the Green multiply sits between the forward and inverse products.  With
both operands split into a TF32 high part and a remainder the products keep FP32-class
accuracy up to the accumulation: a Green step within 8e-6 of the field scale (the FFT
route: 2e-6), converged solves within 1e-6 relative L2 as on the FFT route.
"""
import numpy as np
import pytest

import workloads as wl
from oracle import constraints as ocs, discrete as odz, solver as osv
from tests.helpers import gpu_grid, oracle_problem, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2607_26082_b300 import dtt  # noqa: E402

MIXED = dtt.PREC_MIXED
TENSOR = {"residual_zchunk": 0, "fft_generic": 0, "z_route": 1}
FFT = {"residual_zchunk": 0, "fft_generic": 0, "z_route": 0}
# One Green step on the tensor route: 0.8-5.9e-6 of the field's maximum (relative L2
# 0.6-4.3e-6), growing with the z length (16 ... 200 nodes), against 2-10e-7 for the FP32
# FFT pass: the products are split to about 21 bits, but the tensor core's FP32
# accumulation of up to 3 x 224 terms per output rounds less carefully than the FFT's
# O(log n) stages.  The solver's converged fields are unaffected (tests below, 1e-6).
TOL_GREEN = 8e-6


def _spec(seed, nvox, periodic_prob=0.3, scheme=wl.TETRA2):
    return wl.random_problem(seed, nvox=nvox, scheme=scheme, periodic_prob=periodic_prob, n_strong=0, n_weak=0,
                             n_smooth=0, n_tie=0, anchored=False)


@pytest.mark.parametrize("nvox", [(12, 9, 16), (10, 7, 33), (9, 8, 14), (8, 6, 64), (6, 5, 128), (5, 4, 200)])
@pytest.mark.parametrize("scheme", [wl.TETRA2, wl.HEX1])
@pytest.mark.parametrize("seed", range(3))
def test_tensor_green_step_matches_oracle(nvox, scheme, seed):
    spec = _spec(seed, nvox, scheme=scheme)
    pb, _ = oracle_problem(spec)
    g = gpu_grid(spec, MIXED)
    g.dtt_set_tuning(TENSOR)
    rng = np.random.default_rng(20 + seed)
    pt = rng.standard_normal((3,) + pb.node_shape)
    for c in range(3):
        pt[c][~pb.dof_mask(c)] = 0.0
    ref = odz.green_apply(pb, pt, spec["lam0"], spec["mu0"])
    got = g.dtt_apply_green(pt)
    assert np.abs(got - ref).max() <= TOL_GREEN * np.abs(ref).max()
    assert rel_l2(got, ref) <= TOL_GREEN
    g.close()


def test_tensor_route_refused_where_it_cannot_run():
    spec = _spec(0, (6, 5, 300))
    g = gpu_grid(spec, MIXED)
    with pytest.raises(dtt.DttError) as e:
        g.dtt_set_tuning(TENSOR)
    assert e.value.status == dtt.ERR_ARG
    g.close()
    g = gpu_grid(_spec(0, (6, 5, 16)), dtt.PREC_FP64)
    with pytest.raises(dtt.DttError):
        g.dtt_set_tuning(TENSOR)
    g.close()


def test_tensor_route_converged_cube16():
    spec = wl.cube16()
    pb, rows = oracle_problem(spec)
    ref = osv.solve_alg1(pb, rows, spec["lam0"], spec["mu0"], 1e-13, 3000, acv_mod=3)
    g = gpu_grid(spec, MIXED)
    g.dtt_set_tuning(TENSOR)
    rep = g.dtt_solve_step(1e-7, 3000, acv_mod=3)
    assert rep.status == dtt.OK, rep.as_dict()
    assert rel_l2(g.dtt_get_fields(), ref.u) <= 1e-6
    per, _ = g.dtt_get_reactions(len(rows))
    assert rel_l2(per, ref.reactions) <= 1e-6
    g.close()


def test_tensor_route_contact_increments():
    """Two increments of Algorithm 2 on the tensor route: same active set as the oracle
    away from ties, displacement and force within 1e-6."""
    w = wl.indentation(16, 16, 8, R=6.0, steps=2, dmin=0.01, dmax=0.05)
    pb, _ = oracle_problem(w)
    I = w.indenter
    g = gpu_grid(w, MIXED)
    g.dtt_set_tuning(TENSOR)
    g.dtt_set_indenter(I["axis"], I["face"], I["centers"][0], I["radius"])
    u_ref = np.zeros((3,) + pb.node_shape)
    for step, O in enumerate(I["centers"]):
        ind = ocs.Indenter(pb, I["axis"], I["face"], O, I["radius"])
        ref = osv.solve_alg2_increment(pb, ind, [], w.lam0, w.mu0, 1e-13, 4000, u_ref)
        u_ref = ref.u
        g.dtt_move_indenter(O)
        rep = g.dtt_solve_step(1e-7, 4000, acv_mod=3, init=dtt.INIT_PREVIOUS if step else dtt.INIT_ZERO)
        assert rep.status == dtt.OK, rep.as_dict()
        act, gap, fn, force = g.dtt_get_contact()
        tie = np.abs(ref.gap) < 1e-8 * I["radius"]
        assert np.array_equal(act[~tie], ref.active[~tie])
        assert rel_l2(g.dtt_get_fields(), ref.u) <= 1e-6
        assert np.abs(force - ref.force).max() <= 1e-6 * np.abs(ref.force).max()
    g.close()


def test_tensor_and_fft_routes_agree_on_an_indentation_block():
    """96 x 96 x 48 block with inclusions, first increment to r < 1e-6 on both routes: the
    same converged field within 1e-5 (two solves stopped at the tolerance)."""
    spec = wl.indentation_inclusions(3000, 96, 96, 48, steps=20)
    I = spec["indenter"]
    out = {}
    for name, tun in (("fft", FFT), ("tensor", TENSOR)):
        g = gpu_grid(spec, MIXED)
        g.dtt_set_tuning(tun)
        g.dtt_set_indenter(I["axis"], I["face"], I["centers"][0], I["radius"])
        rep = g.dtt_solve_step(1e-6, 20000, acv_mod=3, graph_iters=16)
        assert rep.status == dtt.OK, (name, rep.as_dict())
        out[name] = (g.dtt_get_fields(), rep.iterations, g.dtt_get_contact()[3])
        g.close()
    assert rel_l2(out["tensor"][0], out["fft"][0]) <= 1e-5
    assert abs(out["tensor"][1] - out["fft"][1]) <= 0.2 * out["fft"][1]
    assert np.abs(out["tensor"][2] - out["fft"][2]).max() <= 1e-5 * np.abs(out["fft"][2]).max()
