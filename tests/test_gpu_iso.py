"""GPU parity of the isotropic reference medium (Section 3.2.3, Eq. 4) against the oracle:
the coupled Green step against the dense definition (oracle.discrete.make_dense_green), the
residual operator's reference term, iterate-for-iterate solves, a laminate closed form, and
the argument checks.

Tolerances as in test_gpu_parity.py: FP64 1e-11 relative (operators), 1e-9 (accelerated
fixed-iteration runs); mixed 2e-6 of the field scale.
"""
import numpy as np
import pytest

import workloads as wl
from oracle import discrete as odz, solver as osv
from tests.helpers import gpu_grid, oracle_problem, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2607_26082_b300 import dtt  # noqa: E402

FP64, MIXED = dtt.PREC_FP64, dtt.PREC_MIXED
D, N = wl.D, wl.N


def _p(pb, seed):
    p = np.random.default_rng(seed).standard_normal((3,) + pb.node_shape)
    for c in range(3):
        p[c][~pb.dof_mask(c)] = 0.0
    return p


# sizes: dense-route axes (2n not a product of 2s and 3s) and register-radix FFT axes
@pytest.mark.parametrize("scheme", [wl.TETRA2, wl.HEX1])
@pytest.mark.parametrize("nvox,seed", [((3, 4, 5), 0), ((5, 3, 4), 1), ((8, 4, 8), 2), ((8, 8, 4), 3)])
@pytest.mark.parametrize("prec,tol", [(FP64, 1e-11), (MIXED, 2e-6)])
def test_iso_green_step(scheme, nvox, seed, prec, tol):
    spec = wl.iso_cell(seed, nvox=nvox, scheme=scheme, n_strong=0)
    pb, _ = oracle_problem(spec)
    g = gpu_grid(spec, prec)
    p = _p(pb, seed)
    green = odz.make_dense_green(pb, lambda u: odz.apply_A0_iso(pb, u, spec["lam0"], spec["mu0"]))
    ref = green(p)
    got = g.dtt_apply_green(p)
    assert np.abs(got - ref).max() <= tol * np.abs(ref).max()
    # the coupled step differs from the Paux medium's by far more than the tolerance
    paux = odz.green_apply(pb, p, spec["lam0"], spec["mu0"])
    assert np.abs(paux - ref).max() >= 1e-3 * np.abs(ref).max()
    g.close()


@pytest.mark.parametrize("scheme", [wl.TETRA2, wl.HEX1])
@pytest.mark.parametrize("prec,tol", [(FP64, 1e-11), (MIXED, 2e-6)])
def test_iso_reference_term(scheme, prec, tol):
    spec = wl.iso_cell(7, nvox=(13, 7, 10), scheme=scheme, n_strong=0)
    pb, _ = oracle_problem(spec)
    g = gpu_grid(spec, prec)
    u = 1e-2 * _p(pb, 7)
    p_ref, sig = odz.residual(pb, u)
    a0 = odz.apply_A0_iso(pb, u, spec["lam0"], spec["mu0"])
    p, pt, _ = g.dtt_apply_residual(u)
    scale = max(np.abs(p_ref).max(), np.abs(a0).max())
    assert np.abs(pt - (p_ref + a0)).max() <= tol * scale
    g.close()


@pytest.mark.parametrize("seed", range(3))
def test_iso_fixed_iterations_fp64(seed):
    """Algorithm 1 with the isotropic medium and Anderson on p~, same number of Green
    steps: iterate-for-iterate parity with the oracle (dense Green step)."""
    spec = wl.iso_cell(seed, nvox=(6, 5, 7), scheme=wl.TETRA2 if seed % 2 == 0 else wl.HEX1)
    pb, rows = oracle_problem(spec)
    K = 15
    ref = osv.solve_alg1(pb, rows, spec["lam0"], spec["mu0"], 0.0, K, acv_on="P", acv_mod=2, medium="iso")
    g = gpu_grid(spec, FP64)
    rep = g.dtt_solve_step(0.0, K, acv_mod=2)
    assert rep.iterations == K and rep.accelerations == ref.accelerations
    assert rel_l2(g.dtt_get_fields(), ref.u) <= 1e-9
    assert np.allclose(g.dtt_get_history(), ref.history, rtol=1e-7, atol=1e-9 * ref.history[0])
    g.close()


@pytest.mark.parametrize("prec,tol", [(FP64, 1e-9), (MIXED, 5e-6)])
def test_iso_converged_against_oracle(prec, tol):
    spec = wl.iso_cell(11, nvox=(7, 6, 5))
    pb, rows = oracle_problem(spec)
    ref = osv.solve_alg1(pb, rows, spec["lam0"], spec["mu0"], 1e-12, 3000, acv_mod=2, medium="iso")
    assert ref.converged
    g = gpu_grid(spec, prec)
    rep = g.dtt_solve_step(1e-12 if prec == FP64 else 2e-7, 3000, acv_mod=2)
    assert rep.status == dtt.OK, rep.as_dict()
    assert rel_l2(g.dtt_get_fields(), ref.u) <= tol
    g.close()


@pytest.mark.parametrize("scheme", [wl.TETRA2, wl.HEX1])
@pytest.mark.parametrize("prec,tol", [(FP64, 1e-10), (MIXED, 2e-5)])
def test_iso_laminate_closed_form(scheme, prec, tol):
    """Layers stacked along z between sliding walls, stretched by eps*_zz: one-dimensional
    solution, each layer strained by sigma_zz / (lambda_i + 2 mu_i).  Max-norm errors; the
    mixed path stops at residual 2e-7."""
    nv = (16, 12, 32)
    phase = np.zeros(nv[::-1], np.uint8)
    phase[8:20] = 1
    lam, mu = wl.lame(np.array([1.0, 5.0]), 0.3)
    ez = 0.01
    spec = dict(nvox=nv, h=1.0, bc=wl.normal_mixed_bc([[D, D], [D, D], [D, D]]), scheme=scheme, phase=phase,
                lam=lam, mu=mu, eps_star=np.diag([0.0, 0.0, ez]), lam0=float(lam.mean()), mu0=float(mu.mean()),
                intents=[], medium="iso")
    g = gpu_grid(spec, prec)
    rep = g.dtt_solve_step(1e-12 if prec == FP64 else 2e-7, 3000, acv_mod=2)
    assert rep.status == dtt.OK, rep.as_dict()
    M = lam + 2 * mu
    t = np.array([8 + 12, 12])                   # layer thicknesses: phase 0 (z < 8 and z >= 20), phase 1
    sig = ez * nv[2] / (t[0] / M[0] + t[1] / M[1])
    e = sig / M - ez
    z = np.arange(nv[2] + 1.0)
    uz = e[0] * np.minimum(z, 8) + e[1] * np.clip(z - 8, 0, 12) + e[0] * np.clip(z - 20, 0, None)
    u = g.dtt_get_fields()
    scale = np.abs(uz).max()
    assert np.abs(u[2] - uz[:, None, None]).max() <= tol * scale
    assert np.abs(u[0]).max() <= tol * scale and np.abs(u[1]).max() <= tol * scale
    g.close()


def test_iso_argument_checks():
    spec = wl.random_problem(3, nvox=(6, 5, 4))            # general boundary conditions
    g = gpu_grid(spec, FP64)
    with pytest.raises(dtt.DttError) as e:
        g.dtt_set_reference_medium(dtt.MEDIUM_ISOTROPIC)
    assert e.value.status == dtt.ERR_BC
    with pytest.raises(dtt.DttError) as e:
        g.dtt_set_reference_medium(7)
    assert e.value.status == dtt.ERR_ARG
    g.close()
    spec = wl.iso_cell(5, nvox=(6, 5, 4))
    g = gpu_grid(spec, MIXED)
    r1 = g.dtt_solve_step(2e-7, 3000, acv_mod=2)
    u1 = g.dtt_get_fields()
    g.dtt_set_reference_medium(dtt.MEDIUM_PAUX)   # switching back recaptures the iteration
    r2 = g.dtt_solve_step(2e-7, 3000, acv_mod=2)
    assert r1.status == r2.status == dtt.OK
    # two reference media, one discrete problem: the same solution
    assert rel_l2(g.dtt_get_fields(), u1) <= 1e-5
    g.close()


# Periodic axes (Section 3.2.3: the isotropic medium with periodic and normal mixed
# conditions): the Hartley basis of a periodic axis couples u_x at q, u_y and u_z at
# partner positions; every periodic pattern, odd and even periods, both schemes.
PERIODIC = [(1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 0), (1, 0, 1), (0, 1, 1), (1, 1, 1)]


@pytest.mark.parametrize("scheme", [wl.TETRA2, wl.HEX1])
@pytest.mark.parametrize("periodic", PERIODIC)
@pytest.mark.parametrize("nvox", [(6, 5, 4), (4, 8, 6)])
@pytest.mark.parametrize("prec,tol", [(FP64, 1e-11), (MIXED, 2e-6)])
def test_iso_green_step_periodic(scheme, periodic, nvox, prec, tol):
    seed = 20 + 4 * sum(periodic) + nvox[0]
    spec = wl.iso_cell(seed, nvox=nvox, scheme=scheme, n_strong=0, periodic=periodic)
    pb, _ = oracle_problem(spec)
    g = gpu_grid(spec, prec)
    g.dtt_set_reference_medium(dtt.MEDIUM_ISOTROPIC)
    p = _p(pb, seed)
    green = odz.make_dense_green(pb, lambda u: odz.apply_A0_iso(pb, u, spec["lam0"], spec["mu0"]))
    ref = green(p)
    got = g.dtt_apply_green(p)
    assert np.abs(got - ref).max() <= tol * np.abs(ref).max()
    g.close()


@pytest.mark.parametrize("periodic", [(1, 0, 0), (0, 1, 1), (1, 1, 1)])
def test_iso_fixed_iterations_periodic_fp64(periodic):
    """Algorithm 1 with the isotropic medium on a cell with periodic axes: iterate for
    iterate against the oracle (dense Green step)."""
    spec = wl.iso_cell(31 + sum(periodic), nvox=(6, 5, 7), scheme=wl.TETRA2, n_strong=2, periodic=periodic)
    pb, rows = oracle_problem(spec)
    K = 15
    ref = osv.solve_alg1(pb, rows, spec["lam0"], spec["mu0"], 0.0, K, acv_on="P", acv_mod=2, medium="iso")
    g = gpu_grid(spec, FP64)
    g.dtt_set_reference_medium(dtt.MEDIUM_ISOTROPIC)
    rep = g.dtt_solve_step(0.0, K, acv_mod=2)
    assert rep.iterations == K and rep.accelerations == ref.accelerations
    assert rel_l2(g.dtt_get_fields(), ref.u) <= 1e-9
    g.close()
