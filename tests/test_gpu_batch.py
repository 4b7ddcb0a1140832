"""Batched solves (dtt_batch_solve) and kernel tuning (dtt_autotune / dtt_set_tuning).

A batch runs every cell's iterations as parallel branches of one CUDA graph; each cell's
arithmetic is the same as in its own solve, so the results are compared bit for bit with
individual solves of identical grids, and one cell against the float64 oracle.
"""
import numpy as np
import pytest

import workloads as wl
from helpers import oracle_problem, gpu_grid, rel_l2
import oracle.solver as osv

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2607_26082_b300 import dtt  # noqa: E402

FP64, MIXED = dtt.PREC_FP64, dtt.PREC_MIXED


def _cells(n=6, seed0=4000, sizes=(8, 12, 16)):
    return wl.batch_cells(n, seed0=seed0, sizes=sizes)


def _tol(prec):
    return 1e-10 if prec == FP64 else 2e-7


@pytest.mark.parametrize("prec", [FP64, MIXED])
def test_batch_matches_individual_solves(prec):
    cells = _cells()
    ref = []
    for c in cells:
        g = gpu_grid(c, prec)
        rep = g.dtt_solve_step(_tol(prec), 4000, acv_mod=c["acv_mod"], graph_iters=8)
        assert rep.status == dtt.OK, (c["name"], rep.as_dict())
        ref.append((rep.iterations, g.dtt_get_fields()))
        g.close()
    grids = [gpu_grid(c, prec) for c in cells]
    st, reps = dtt.dtt_batch_solve(grids, _tol(prec), 4000, acv_mod=2, graph_iters=8)
    assert st == dtt.OK
    for g, rep, (it, u) in zip(grids, reps, ref):
        assert rep.status == dtt.OK
        assert rep.iterations == it
        assert np.array_equal(g.dtt_get_fields(), u)
    # the cached graph is reused for a second solve of the same, unchanged grids
    st, reps2 = dtt.dtt_batch_solve(grids, _tol(prec), 4000, acv_mod=2, graph_iters=8)
    assert st == dtt.OK and [r.iterations for r in reps2] == [r.iterations for r in reps]
    for g, (it, u) in zip(grids, ref):
        assert np.array_equal(g.dtt_get_fields(), u)
        g.close()


def test_batch_cell_matches_oracle():
    c = wl.batch_cell(4101, sizes=(8,))
    pb, rows = oracle_problem(c)
    ref = osv.solve_alg1(pb, rows, c["lam0"], c["mu0"], 1e-12, 4000, acv_mod=c["acv_mod"])
    grids = [gpu_grid(c, FP64), gpu_grid(wl.batch_cell(4102, sizes=(12,)), FP64)]
    st, reps = dtt.dtt_batch_solve(grids, 1e-12, 4000, acv_mod=2)
    assert st == dtt.OK, [r.as_dict() for r in reps]
    assert rel_l2(grids[0].dtt_get_fields(), ref.u) <= 1e-9
    for g in grids:
        g.close()


def test_batch_changed_grid_recaptures():
    cells = _cells(3, seed0=4200)
    grids = [gpu_grid(c, MIXED) for c in cells]
    st, _ = dtt.dtt_batch_solve(grids, 2e-7, 4000, acv_mod=2)
    assert st == dtt.OK
    # a new reference medium changes captured launch arguments: the batch graph is rebuilt
    c0 = cells[0]
    grids[0].dtt_set_reference(1.5 * c0["lam0"], 1.5 * c0["mu0"])
    st, reps = dtt.dtt_batch_solve(grids, 2e-7, 4000, acv_mod=2)
    g = gpu_grid(c0, MIXED)
    g.dtt_set_reference(1.5 * c0["lam0"], 1.5 * c0["mu0"])
    rep = g.dtt_solve_step(2e-7, 4000, acv_mod=2)
    assert st == dtt.OK and reps[0].iterations == rep.iterations
    assert np.array_equal(g.dtt_get_fields(), grids[0].dtt_get_fields())
    for q in grids + [g]:
        q.close()


def test_batch_rejects_duplicates_and_empty():
    c = _cells(1)[0]
    g = gpu_grid(c, MIXED)
    with pytest.raises(dtt.DttError) as e:
        dtt.dtt_batch_solve([g, g], 1e-6, 100)
    assert e.value.status == dtt.ERR_ARG
    with pytest.raises(dtt.DttError):
        dtt.dtt_batch_solve([], 1e-6, 100)
    g.close()


@pytest.mark.parametrize("prec", [FP64, MIXED])
def test_autotune_keeps_results(prec):
    c = wl.batch_cell(4300, sizes=(32,))
    g0 = gpu_grid(c, prec)
    r0 = g0.dtt_solve_step(_tol(prec), 4000, acv_mod=2)
    g = gpu_grid(c, prec)
    t = g.dtt_autotune(iters=3, acv_mod=2)
    assert t.residual_zchunk in (0, 2, 4, 8, 16, 32, 64) and t.fft_generic in (0, 1)
    assert t.ms_per_iteration > 0.0
    r = g.dtt_solve_step(_tol(prec), 4000, acv_mod=2)
    assert r.status == dtt.OK and r0.status == dtt.OK
    # another tiling regroups the partial sums only
    assert rel_l2(g.dtt_get_fields(), g0.dtt_get_fields()) <= (1e-9 if prec == FP64 else 2e-5)
    # the tuned tiling transfers to a grid of the same size; bad values are rejected
    g2 = gpu_grid(c, prec)
    g2.dtt_set_tuning(t)
    r2 = g2.dtt_solve_step(_tol(prec), 4000, acv_mod=2)
    assert r2.iterations == r.iterations
    assert np.array_equal(g2.dtt_get_fields(), g.dtt_get_fields())
    for bad in ({"residual_zchunk": 1, "fft_generic": 0}, {"residual_zchunk": 0, "fft_generic": 2},
                {"residual_zchunk": 65, "fft_generic": 0}):
        with pytest.raises(dtt.DttError) as e:
            g2.dtt_set_tuning(bad)
        assert e.value.status == dtt.ERR_ARG
    for q in (g0, g, g2):
        q.close()


@pytest.mark.parametrize("kind", ["finite_strain", "isotropic"])
def test_batch_with_finite_strain_and_isotropic_cells(kind):
    """Cells with the finite-strain stress step or the isotropic reference medium batch like
    the others: each cell's result equals its own solve bit for bit."""
    if kind == "finite_strain":
        cells = [dict(c, kinematics="FS") for c in _cells(3, seed0=4600)]
    else:
        cells = [wl.iso_cell(4700 + k, nvox=n) for k, n in enumerate([(8, 6, 7), (12, 8, 6), (6, 6, 6)])]
    ref = []
    for c in cells:
        g = gpu_grid(c, MIXED)
        rep = g.dtt_solve_step(2e-7, 4000, acv_mod=2, graph_iters=8)
        assert rep.status == dtt.OK, (kind, rep.as_dict())
        ref.append((rep.iterations, g.dtt_get_fields()))
        g.close()
    grids = [gpu_grid(c, MIXED) for c in cells]
    st, reps = dtt.dtt_batch_solve(grids, 2e-7, 4000, acv_mod=2, graph_iters=8)
    assert st == dtt.OK
    for g, rep, (it, u) in zip(grids, reps, ref):
        assert rep.status == dtt.OK and rep.iterations == it
        assert np.array_equal(g.dtt_get_fields(), u)
        g.close()


@pytest.mark.parametrize("prec", [dtt.PREC_FP64, dtt.PREC_MIXED])
def test_new_values_in_same_layout_keep_graph_and_match_fresh_grid(prec):
    """New Lame values for the same number of phases, and new constraint values for the same
    rows, are taken in place: the captured iteration stays, and the next solve equals a
    fresh grid's bit for bit (and differs from the solve with the old values)."""
    from paper_2607_26082_b300 import rows as prow
    spec = wl.random_problem(21, nvox=(12, 10, 9))
    ptr, node, comp, a, b, val = prow.csr_from_intents(spec["nvox"], spec["bc"], spec["intents"])
    g = gpu_grid(spec, prec)
    g.dtt_solve_step(1e-6, 3000, acv_mod=2, init=dtt.INIT_ZERO)
    u_old = g.dtt_get_fields()
    lam2, mu2, val2 = 1.7 * spec["lam"], 0.6 * spec["mu"], 1.5 * val + 1e-3
    g.dtt_set_material(spec["phase"], lam2, mu2)
    g.dtt_set_constraints(ptr, node, comp, a, b, val2)
    r1 = g.dtt_solve_step(1e-6, 3000, acv_mod=2, init=dtt.INIT_ZERO)
    spec2 = dict(spec, lam=lam2, mu=mu2)
    g2 = gpu_grid(spec2, prec)
    g2.dtt_set_constraints(ptr, node, comp, a, b, val2)
    r2 = g2.dtt_solve_step(1e-6, 3000, acv_mod=2, init=dtt.INIT_ZERO)
    assert r1.status == r2.status == dtt.OK
    assert r1.iterations == r2.iterations
    u1, u2 = g.dtt_get_fields(), g2.dtt_get_fields()
    assert np.array_equal(u1, u2)
    assert rel_l2(u1, u_old) > 1e-3
    per1, _ = g.dtt_get_reactions(len(val))
    per2, _ = g2.dtt_get_reactions(len(val))
    assert np.array_equal(per1, per2)
    g.close()
    g2.close()


@pytest.mark.parametrize("prec", [FP64, MIXED])
def test_device_loop_matches_host_loop(prec, monkeypatch):
    """A solve (and a batch) runs as one graph launch: a conditional WHILE node repeats a
    round of graph_iters iterations while a grid is running.  With DTT_GRAPH_LOOP=0 the
    host launches one round at a time and polls the done flags instead.  Both loops stop at
    the same iterate: fields bit-identical, same iteration counts, the max_iter cap
    honoured mid-round."""
    cells = _cells(4, seed0=4200)

    def run(loop):
        if loop:
            monkeypatch.delenv("DTT_GRAPH_LOOP", raising=False)
        else:
            monkeypatch.setenv("DTT_GRAPH_LOOP", "0")
        one = []
        for c in cells:
            g = gpu_grid(c, prec)
            rep = g.dtt_solve_step(_tol(prec), 4000, acv_mod=c["acv_mod"], graph_iters=8)
            capped = gpu_grid(c, prec)
            rc = capped.dtt_solve_step(_tol(prec), 5, acv_mod=c["acv_mod"], graph_iters=8)
            one.append((rep.status, rep.iterations, g.dtt_get_fields(), rc.status, rc.iterations,
                        capped.dtt_get_fields()))
            g.close()
            capped.close()
        grids = [gpu_grid(c, prec) for c in cells]
        st, reps = dtt.dtt_batch_solve(grids, _tol(prec), 4000, acv_mod=2, graph_iters=8)
        assert st == dtt.OK
        batch = [(r.status, r.iterations, g.dtt_get_fields()) for g, r in zip(grids, reps)]
        for g in grids:
            g.close()
        return one, batch

    dev, host = run(True), run(False)
    for a, b in zip(dev[0], host[0]):
        assert a[0] == b[0] == dtt.OK and a[1] == b[1]
        assert np.array_equal(a[2], b[2])
        assert a[3] == b[3] == dtt.ERR_NOT_CONVERGED and a[4] == b[4] == 5
        assert np.array_equal(a[5], b[5])
    for a, b in zip(dev[1], host[1]):
        assert a[0] == b[0] == dtt.OK and a[1] == b[1]
        assert np.array_equal(a[2], b[2])
