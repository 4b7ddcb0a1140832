"""GPU parity of the finite-strain path (Section 5.2, Eq. 29, Algorithm 3) against the
float64 oracle: the residual operator with the first Piola-Kirchhoff stress, the stress
outputs, fixed-iteration and converged solves, the homogeneous stretch, a finite rigid
rotation, and contact increments.

Tolerances as in test_gpu_parity.py: FP64 operators 1e-11 relative to the field scale,
plain fixed-iteration solves 1e-10 (a nonlinear stress step between Green steps), mixed
operators 2e-6 of the field scale (float32 rounding of the gradient, of E and of F.S).
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

FP64, MIXED = dtt.PREC_FP64, dtt.PREC_MIXED
P, D, N = wl.P, wl.D, wl.N


def _fs_grid(spec, prec):
    g = gpu_grid(spec, prec)
    g.dtt_set_kinematics(dtt.FINITE_STRAIN)
    return g


def _u(pb, seed, scale):
    u = scale * np.random.default_rng(seed).standard_normal((3,) + pb.node_shape)
    for c in range(3):
        u[c][~pb.dof_mask(c)] = 0.0
    return u


@pytest.mark.parametrize("scheme", [wl.TETRA2, wl.HEX1])
@pytest.mark.parametrize("seed", range(3))
@pytest.mark.parametrize("nvox", [(2, 2, 2), (31, 5, 17), (40, 9, 12)])
def test_fs_residual_operator_fp64(scheme, seed, nvox):
    spec = wl.random_problem(seed, nvox=nvox, scheme=scheme, periodic_prob=0.3, eps_scale=0.03,
                             n_strong=0, n_weak=0, n_smooth=0, n_tie=0, anchored=False)
    pb, _ = oracle_problem(spec)
    g = _fs_grid(spec, FP64)
    u = _u(pb, seed, 5e-2)
    p_ref, Pi = odz.residual(pb, u, "FS")
    a0 = odz.apply_A0(pb, u, spec["lam0"], spec["mu0"])
    p, pt, norms = g.dtt_apply_residual(u)
    scale = max(np.abs(p_ref).max(), np.abs(a0).max())
    assert np.abs(p - p_ref).max() <= 1e-11 * scale
    assert np.abs(pt - (p_ref + a0)).max() <= 1e-11 * scale
    w = np.array([ip[0] for ip in pb.ip_sets()])
    s2 = np.sum(w[:, None, None, None, None, None] * Pi * Pi)
    assert abs(norms[0] - s2) <= 1e-11 * s2
    # the finite-strain terms are far above the tolerance: the test tells the two apart
    p_ss, _ = odz.residual(pb, u, "SS")
    assert np.abs(p_ss - p_ref).max() >= 1e-4 * scale


@pytest.mark.parametrize("scheme", [wl.TETRA2, wl.HEX1])
@pytest.mark.parametrize("seed", range(3))
def test_fs_residual_operator_mixed(scheme, seed):
    spec = wl.random_problem(seed, nvox=(40, 6, 21), scheme=scheme, eps_scale=0.03)
    pb, _ = oracle_problem(spec)
    g = _fs_grid(spec, MIXED)
    u = _u(pb, seed, 5e-2)
    p_ref, Pi = odz.residual(pb, u, "FS")
    p, _, norms = g.dtt_apply_residual(u)
    scale = np.abs(Pi).max() / pb.h
    assert np.abs(p - p_ref).max() <= 2e-6 * scale
    w = np.array([ip[0] for ip in pb.ip_sets()])
    s2 = np.sum(w[:, None, None, None, None, None] * Pi * Pi)
    assert abs(norms[0] - s2) <= 1e-5 * s2


@pytest.mark.parametrize("prec", [FP64, MIXED])
def test_stress_outputs(prec):
    """dtt_get_stress_tensor returns sigma (small strain) or Pi (finite strain), all nine
    values; dtt_get_fields returns sigma or the second Piola-Kirchhoff S."""
    spec = wl.random_problem(11, nvox=(7, 5, 6), eps_scale=0.03)
    pb, _ = oracle_problem(spec)
    g = gpu_grid(spec, prec)
    u = _u(pb, 11, 5e-2)
    g.dtt_set_initial(u)
    tol = 1e-12 if prec == FP64 else 1e-6
    sig = odz.stress(pb, u)
    t9 = g.dtt_get_stress_tensor()
    ref9 = np.moveaxis(sig, (0, 1, 2), (3, 4, 5))   # (vox..., ip, 3, 3)
    assert rel_l2(t9, ref9) <= tol
    g.dtt_set_kinematics(dtt.FINITE_STRAIN)
    Pi = odz.piola(pb, u)
    t9 = g.dtt_get_stress_tensor()
    assert rel_l2(t9, np.moveaxis(Pi, (0, 1, 2), (3, 4, 5))) <= tol
    _, s6 = g.dtt_get_fields(sigma=True)
    # S from Pi = F.S: S = F^-1 Pi
    gr = odz.gradients(pb, u) + pb.eps_star[None, :, :, None, None, None]
    F = np.moveaxis(gr, (0, 1, 2), (3, 4, 5)) + np.eye(3)
    S = np.linalg.solve(F, np.moveaxis(Pi, (0, 1, 2), (3, 4, 5)))
    S6 = np.stack([S[..., 0, 0], S[..., 1, 1], S[..., 2, 2], S[..., 1, 2], S[..., 0, 2], S[..., 0, 1]], axis=-1)
    assert rel_l2(s6, S6) <= 10 * tol


@pytest.mark.parametrize("seed", range(4))
def test_fs_fixed_iterations_plain_fp64(seed):
    """Plain fixed point with the finite-strain stress step, same number of Green steps:
    iterate-for-iterate parity.  The reference medium is four times the default: without
    acceleration the finite-strain HEX1 iteration is unstable with the softer one (the
    paper too takes a stiffer reference medium for finite strain, Section 5.4)."""
    spec = wl.random_problem(seed, nvox=(9, 6, 7), scheme=wl.TETRA2 if seed % 2 == 0 else wl.HEX1,
                             eps_scale=0.03, n_smooth=1 if seed % 2 == 0 else 0)
    spec["lam0"] *= 4.0
    spec["mu0"] *= 4.0
    pb, rows = oracle_problem(spec)
    K = 25
    ref = osv.solve_alg1(pb, rows, spec["lam0"], spec["mu0"], 0.0, K, acv=False, kinematics="FS")
    g = _fs_grid(spec, FP64)
    rep = g.dtt_solve_step(0.0, K, acv_mod=0)
    assert rep.iterations == K
    assert rel_l2(g.dtt_get_fields(), ref.u) <= 1e-10
    hist = g.dtt_get_history()
    assert np.allclose(hist, ref.history, rtol=1e-10, atol=1e-12 * ref.history[0])
    per, _ = g.dtt_get_reactions(len(rows))
    assert np.abs(per - ref.reactions).max() <= 1e-10 * max(np.abs(ref.reactions).max(), 1e-30)


@pytest.mark.parametrize("prec,tol_u", [(FP64, 1e-10), (MIXED, 2e-6)])
def test_fs_converged_with_constraints(prec, tol_u):
    for seed in range(3):
        spec = wl.random_problem(seed, nvox=(11, 8, 9), eps_scale=0.03)
        pb, rows = oracle_problem(spec)
        ref = osv.solve_alg1(pb, rows, spec["lam0"], spec["mu0"], 1e-12, 3000, kinematics="FS")
        assert ref.converged
        g = _fs_grid(spec, prec)
        rep = g.dtt_solve_step(1e-12 if prec == FP64 else 2e-7, 3000)
        assert rep.status == dtt.OK, (seed, rep.as_dict())
        assert rel_l2(g.dtt_get_fields(), ref.u) <= tol_u
        per, _ = g.dtt_get_reactions(len(rows))
        assert rel_l2(per, ref.reactions) <= 10 * tol_u


@pytest.mark.parametrize("scheme", [wl.TETRA2, wl.HEX1])
@pytest.mark.parametrize("prec,tol", [(FP64, 1e-9), (MIXED, 5e-6)])
def test_fs_uniaxial_stretch(scheme, prec, tol):
    """The homogeneous St Venant-Kirchhoff stretch (E_xx = E_yy = -nu E_zz), reached by the
    GPU solver on a 24 x 20 x 16 bar; Section 5.4's force from the mean of Pi.  Max-norm
    errors: the mixed path stops at residual 2e-7, whose float32 floor is a few 1e-6 of
    the displacement scale at the worst node."""
    lam, mu = 1.2, 0.8
    nu = lam / (2 * (lam + mu))
    young = mu * (3 * lam + 2 * mu) / (lam + mu)
    ez = 0.06
    nv = (24, 20, 16)
    bc = np.full((3, 2, 3), N)
    bc[0, 0, 0] = D
    bc[1, 0, 1] = D
    bc[2, :, 2] = D
    eps = np.zeros((3, 3))
    eps[2, 2] = ez
    spec = dict(nvox=nv, h=1.0, bc=bc, scheme=scheme, phase=np.zeros(nv[::-1], np.uint8),
                lam=np.array([lam]), mu=np.array([mu]), eps_star=eps, lam0=2 * lam, mu0=2 * mu, intents=[])
    pb, _ = oracle_problem(spec)
    g = _fs_grid(spec, prec)
    rep = g.dtt_solve_step(1e-12 if prec == FP64 else 2e-7, 3000, acv_mod=2)
    assert rep.status == dtt.OK, rep.as_dict()
    Ezz = ((1 + ez) ** 2 - 1) / 2
    b = np.sqrt(1 - 2 * nu * Ezz) - 1
    X = pb.node_positions()
    u = g.dtt_get_fields()
    scale = abs(b) * nv[0]
    assert np.abs(u[0] - b * X[0]).max() <= tol * scale
    assert np.abs(u[1] - b * X[1]).max() <= tol * scale
    assert np.abs(u[2]).max() <= tol * scale
    t9 = g.dtt_get_stress_tensor()
    mean = t9.mean(axis=(0, 1, 2, 3))
    Pzz = (1 + ez) * young * Ezz
    assert abs(mean[2, 2] - Pzz) <= 10 * tol * Pzz


@pytest.mark.parametrize("prec,tol", [(FP64, 1e-12), (MIXED, 2e-6)])
def test_fs_rigid_rotation_has_no_residual(prec, tol):
    """A finite rotation of the whole cell carries no stress in finite strain; the
    small-strain residual of the same field is large."""
    bc = np.full((3, 2, 3), N)
    nv = (20, 12, 9)
    spec = dict(nvox=nv, h=1.0, bc=bc, scheme=wl.TETRA2, phase=np.zeros(nv[::-1], np.uint8),
                lam=np.array([1.0]), mu=np.array([0.7]), eps_star=np.zeros((3, 3)), lam0=2.0, mu0=1.4,
                intents=[])
    pb, _ = oracle_problem(spec)
    th = 0.4
    a = np.array([2.0, -1.0, 2.0]) / 3.0
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    Q = np.eye(3) + np.sin(th) * K + (1 - np.cos(th)) * K @ K
    X = pb.node_positions()
    u = np.einsum("ab,bzyx->azyx", Q - np.eye(3), X)
    g = gpu_grid(spec, prec)
    p_ss, _, _ = g.dtt_apply_residual(u)
    g.dtt_set_kinematics(dtt.FINITE_STRAIN)
    p_fs, _, _ = g.dtt_apply_residual(u)
    big = np.abs(p_ss).max()
    assert big >= 0.01
    assert np.abs(p_fs).max() <= tol * max(1.0, np.abs(u).max())


@pytest.mark.parametrize("prec", [FP64, MIXED])
def test_fs_contact_increments(prec):
    """Algorithm 3 on a 16 x 16 x 8 block, two increments, against the oracle."""
    w = wl.indentation(16, 16, 8, R=6.0, steps=2, dmin=0.01, dmax=0.05)
    pb, _ = oracle_problem(w)
    I = w.indenter
    g = _fs_grid(w, prec)
    u_ref = np.zeros((3,) + pb.node_shape)
    g.dtt_set_indenter(I["axis"], I["face"], I["centers"][0], I["radius"])
    for step, O in enumerate(I["centers"]):
        ind = ocs.Indenter(pb, I["axis"], I["face"], O, I["radius"])
        ref = osv.solve_alg2_increment(pb, ind, [], w.lam0, w.mu0, 1e-10, 2000, u_ref, kinematics="FS")
        u_ref = ref.u
        g.dtt_move_indenter(O)
        rep = g.dtt_solve_step(1e-10 if prec == FP64 else 1e-7, 2000, acv_mod=3,
                               init=dtt.INIT_PREVIOUS if step else dtt.INIT_ZERO)
        assert rep.status == dtt.OK, rep.as_dict()
        act, gap, fn, force = g.dtt_get_contact()
        if prec == FP64:
            assert np.array_equal(act, ref.active)
            assert rel_l2(g.dtt_get_fields(), ref.u) <= 1e-9
            assert np.abs(force - ref.force).max() <= 1e-8 * np.abs(ref.force).max()
        else:
            tie = np.abs(ref.gap) < 1e-8 * I["radius"]
            assert np.array_equal(act[~tie], ref.active[~tie])
            assert rel_l2(g.dtt_get_fields(), ref.u) <= 1e-5
            assert np.abs(force - ref.force).max() <= 1e-5 * np.abs(ref.force).max()
        # Section 5.4: the contact force from the mean of Pi over the block
        t9 = g.dtt_get_stress_tensor()
        fz = t9.mean(axis=(0, 1, 2, 3))[2, 2] * w.nvox[0] * w.nvox[1]
        assert abs(fz - force[2]) <= (1e-8 if prec == FP64 else 1e-4) * abs(force[2])


def test_kinematics_switch_recaptures_and_rejects_bad_values():
    spec = wl.random_problem(21, nvox=(10, 8, 6), eps_scale=0.03)
    g = gpu_grid(spec, MIXED)
    r_ss = g.dtt_solve_step(1e-6, 2000)
    g.dtt_set_kinematics(dtt.FINITE_STRAIN)
    r_fs = g.dtt_solve_step(1e-6, 2000)
    g2 = _fs_grid(spec, MIXED)
    r2 = g2.dtt_solve_step(1e-6, 2000)
    assert r_ss.status == r_fs.status == r2.status == dtt.OK
    assert r_fs.iterations == r2.iterations
    assert np.array_equal(g.dtt_get_fields(), g2.dtt_get_fields())
    for bad in (2, -1):
        with pytest.raises(dtt.DttError) as e:
            g.dtt_set_kinematics(bad)
        assert e.value.status == dtt.ERR_ARG
    for q in (g, g2):
        q.close()


@pytest.mark.parametrize("prec,tol", [(FP64, 1e-12), (MIXED, 1e-6)])
def test_min_jacobian(prec, tol):
    """dtt_get_min_jacobian against det(1 + eps* + grad u) from the oracle's gradients: a
    random field, a field that inverts part of the cell, and a finite rotation (det F = 1
    everywhere).  Traction-free faces, so that every nodal value is an unknown."""
    spec = wl.random_problem(31, nvox=(9, 7, 8), eps_scale=0.03, scheme=wl.HEX1,
                             n_strong=0, n_weak=0, n_smooth=0, n_tie=0, anchored=False)
    spec["bc"] = np.full((3, 2, 3), N)
    pb, _ = oracle_problem(spec)
    g = gpu_grid(spec, prec)

    def ref_min(u, eps):
        gr = odz.gradients(pb, u) + eps[None, :, :, None, None, None]
        F = np.moveaxis(gr, (1, 2), (-2, -1)) + np.eye(3)
        return np.linalg.det(F).min()

    u = 0.2 * np.random.default_rng(31).standard_normal((3,) + pb.node_shape)
    g.dtt_set_initial(u)
    assert abs(g.dtt_get_min_jacobian() - ref_min(u, pb.eps_star)) <= tol
    X = pb.node_positions()
    u_inv = np.zeros_like(u)
    u_inv[0] = np.where(X[0] < 4, -2.5 * X[0], -10.0)   # F_xx about -1.5 left of x = 4
    g.dtt_set_initial(u_inv)
    m = g.dtt_get_min_jacobian()
    assert m < 0 and abs(m - ref_min(u_inv, pb.eps_star)) <= 10 * tol
    g.dtt_set_load(np.zeros((3, 3)))
    th = 0.7
    Q = np.array([[np.cos(th), -np.sin(th), 0], [np.sin(th), np.cos(th), 0], [0, 0, 1.0]])
    g.dtt_set_initial(np.einsum("ab,bzyx->azyx", Q - np.eye(3), X))
    assert abs(g.dtt_get_min_jacobian() - 1.0) <= tol
    g.close()
