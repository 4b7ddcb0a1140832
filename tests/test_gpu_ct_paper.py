"""The paper's CT-like specimen (Sections 4.1.2, 4.1.3, 4.2.3) on the GPU: 10 x 100 x (50 + 1)
voxels with the void buffer, ligament rows and the five loadings of workloads.ct_specimen.

  * FP64 iterate-for-iterate parity with the oracle (Anderson on p~, mod 2);
  * the reaction balance of Section 4.1.3 at convergence: the load rows' reaction and the
    ligament's cancel (the void buffer carries no force);
  * Section 4.2.3: a strong load on a single node moves only its TETRA2 sub-grid (its six
    neighbours stay put), while the weak (element-centre) and smooth loads do not, and
    agree with each other up to the half-voxel shift of the load point;
  * Table 1: period 2 is the better Anderson period, for u~ and for p~.
"""
import numpy as np
import pytest

import workloads as wl
from oracle import solver as osv
from tests.helpers import gpu_grid, oracle_problem, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2607_26082_b300 import dtt  # noqa: E402

FP64, MIXED = dtt.PREC_FP64, dtt.PREC_MIXED
LOAD_NODE = (2, 24, 25)   # (i, j, k): paper position (2, 24, 24), z shifted by the buffer


def _balance(g, spec):
    per, _ = g.dtt_get_reactions(g.n_rows)
    nl = spec["ligament_rows"]
    r_l, r_s = per[:nl].sum(), per[nl:].sum()
    return abs(r_l + r_s) / abs(r_l), r_l, r_s


def test_ct_paper_fixed_iterations_fp64():
    spec = wl.ct_specimen("strong_line")
    pb, rows = oracle_problem(spec)
    K = 20
    ref = osv.solve_alg1(pb, rows, spec["lam0"], spec["mu0"], 0.0, K, acv_on="P", acv_mod=2)
    g = gpu_grid(spec, FP64)
    rep = g.dtt_solve_step(0.0, K, acv_mod=2)
    assert rep.iterations == K and rep.accelerations == ref.accelerations
    assert rel_l2(g.dtt_get_fields(), ref.u) <= 1e-9
    assert np.allclose(g.dtt_get_history(), ref.history, rtol=1e-7, atol=1e-9 * ref.history[0])
    per, _ = g.dtt_get_reactions(len(rows))
    assert rel_l2(per, ref.reactions) <= 1e-8
    g.close()


@pytest.mark.parametrize("prec,tol,bal", [(FP64, 1e-11, 1e-9), (MIXED, 1e-6, 1e-4)])
def test_ct_paper_reaction_balance(prec, tol, bal):
    """Section 4.1.3: the reactions of the load and of the ligament balance at convergence
    (the paper: relative error 5e-12); they do not early in the iteration."""
    spec = wl.ct_specimen("strong_line")
    g = gpu_grid(spec, prec)
    rep = g.dtt_solve_step(0.0, 5, acv_mod=2)
    b0, _, _ = _balance(g, spec)
    rep = g.dtt_solve_step(tol, 20000, acv_mod=2)
    assert rep.status == dtt.OK, rep.as_dict()
    b, r_l, r_s = _balance(g, spec)
    assert b <= bal and b0 > 100 * b
    assert r_s > 0 > r_l
    g.close()


def _neighbour_ratio(u):
    i, j, k = LOAD_NODE
    uz = u[2]
    nb = [uz[k, j, i + 1], uz[k, j, i - 1], uz[k, j + 1, i], uz[k, j - 1, i], uz[k + 1, j, i], uz[k - 1, j, i]]
    return np.mean(nb) / uz[k, j, i]


def test_ct_paper_single_point_loads():
    """Section 4.2.3, Fig. 5: the strong single-node load leaves the other TETRA2 sub-grid
    behind; the weak (element centre) and smooth loads move the neighbourhood with the
    load point and give nearly the same field."""
    u = {}
    for load in ("strong_node", "weak_node", "smooth_node"):
        spec = wl.ct_specimen(load, tol=1e-6)
        g = gpu_grid(spec, MIXED)
        rep = g.dtt_solve_step(1e-6, 20000, acv_mod=2)
        assert rep.status == dtt.OK, (load, rep.as_dict())
        u[load] = g.dtt_get_fields()
        g.close()
    assert abs(_neighbour_ratio(u["strong_node"])) <= 1e-3
    assert _neighbour_ratio(u["weak_node"]) >= 0.5
    assert _neighbour_ratio(u["smooth_node"]) >= 0.5
    assert rel_l2(u["weak_node"], u["smooth_node"]) <= 0.1
    assert rel_l2(u["strong_node"], u["smooth_node"]) >= 2 * rel_l2(u["weak_node"], u["smooth_node"])


def test_ct_paper_weak_line_load():
    """The line load applied weakly over the 44 nodes of the loaded elements: their mean
    displacement is the prescribed 10, and the load and ligament reactions balance."""
    spec = wl.ct_specimen("weak_line", tol=1e-6)
    g = gpu_grid(spec, MIXED)
    rep = g.dtt_solve_step(1e-6, 20000, acv_mod=2)
    assert rep.status == dtt.OK, rep.as_dict()
    u = g.dtt_get_fields()
    nodes = spec["intents"][-1]["nodes"]
    assert abs(np.mean([u[2][k, j, i] for i, j, k in nodes]) - 10.0) <= 1e-5
    b, _, _ = _balance(g, spec)
    assert b <= 1e-4
    g.close()


def test_ct_paper_acceleration_periods():
    """Table 1 at tolerance 1e-4, FP64: period 2 beats period 3 for Anderson on u~ and on
    p~, the paper's best choice being mod_ACV = 2.  The paper also finds p~ ahead of u~;
    with this library's combination rule (the paper prints none; the oracle's is pinned by
    a closed form) the two
    are close at period 2 and that ordering is not asserted.  All four runs reach the same
    reactions to the tolerance's accuracy."""
    spec = wl.ct_specimen("strong_line")
    its, reac = {}, {}
    for on in (dtt.ACV_U, dtt.ACV_P):
        for mod in (2, 3):
            g = gpu_grid(spec, FP64)
            rep = g.dtt_solve_step(1e-4, 20000, acv_mod=mod, acv_on=on)
            assert rep.status == dtt.OK
            its[on, mod] = rep.iterations
            reac[on, mod] = _balance(g, spec)[1]
            g.close()
    for on in (dtt.ACV_U, dtt.ACV_P):
        assert its[on, 2] < its[on, 3]
    vals = np.array(list(reac.values()))
    assert np.ptp(vals) <= 2e-3 * np.abs(vals).max()
