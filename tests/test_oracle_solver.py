"""Pins of the oracle solvers: Algorithm 1 against closed forms and the dense
multiplier system (Section 4.3), the smooth-condition weights (Section 4.2.2), the
TETRA2 sub-grid decoupling (Section 4.2.3), and Algorithm 2 against contact
complementarity (Eq. 33), force balance (Section 5.4) and the Hertz law (Eq. 30)."""
import os

import numpy as np
import pytest

import workloads as wl
from oracle import constraints as cs, discrete as dz, hertz, kkt, solver as sv

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
P, D, N = wl.P, wl.D, wl.N


@pytest.mark.parametrize("scheme", [dz.TETRA2, dz.HEX1])
@pytest.mark.parametrize("acv_on", ["P", "U"])
def test_affine_closed_form(scheme, acv_on):
    """P3: uniaxial stress; both schemes are exact for affine fields, so the discrete
    solution is u_x = -nu eps x, u_y = -nu eps y, u_z = eps z, reached from u~ = 0."""
    E, nu, eps = 1.0, 0.3, 1e-2
    lam, mu = wl.lame(E, nu)
    bc = np.full((3, 2, 3), N)
    bc[2, :, 2] = D
    bc[0, 0, 0] = D
    bc[1, 0, 1] = D
    es = np.zeros((3, 3))
    es[2, 2] = eps
    pb = dz.Problem((6, 5, 7), 1.0, bc, scheme, np.zeros((7, 5, 6)), [lam], [mu], es)
    res = sv.solve_alg1(pb, [], 5 * lam, 5 * mu, 1e-12, 500, acv_on=acv_on)
    X = pb.node_positions()
    exact = np.stack([-nu * eps * X[0], -nu * eps * X[1], 0 * X[2]])
    assert res.converged
    assert np.abs(res.u - exact).max() < 1e-13
    sig = dz.stress(pb, res.u)
    assert np.allclose(sig[:, 2, 2], E * eps, atol=1e-13)
    assert np.abs(sig[:, 0, 0]).max() < 1e-13


@pytest.mark.parametrize("seed", range(5))
def test_kkt_tetra2_random(seed):
    """P4: Algorithm 1 (ACV_P) converged to 1e-12 equals the dense solve of the
    multiplier system, random BCs / phases / eps* / strong, weak, smooth, tie rows."""
    w = wl.random_problem(seed)
    pb = dz.problem_from(w)
    rows = cs.rows_from_intents(pb, w.intents)
    uk, fk = kkt.solve_kkt(pb, rows, cs.targets(pb, rows))
    res = sv.solve_alg1(pb, rows, w.lam0, w.mu0, 1e-12, 2000)
    assert res.converged
    assert np.abs(res.u - uk).max() <= 1e-10 * np.abs(uk).max()
    assert np.abs(res.f - fk).max() <= 1e-10 * np.abs(fk).max()


@pytest.mark.parametrize("acv_on", ["P", "U"])
def test_kkt_hex1_weak_rows(acv_on):
    """P4 for HEX1 with weakly applied conditions (Section 4.2.3: HEX1 converges with
    weak conditions); two Dirichlet axes per component remove hourglass modes."""
    rng = np.random.default_rng(0)
    bc = np.full((3, 2, 3), N)
    bc[0, 0, :] = D
    bc[1, 0, :] = D
    ph = rng.integers(0, 2, size=(4, 5, 4))
    es = np.array([[1e-3, 2e-3, 0], [2e-3, 0, 0], [0, 0, -1e-3]])
    pb = dz.Problem((4, 5, 4), 1.0, bc, dz.HEX1, ph, [0.6, 1.5], [0.4, 1.0], es)
    rows = [cs.weak_voxel_row(pb, (1, 1, 2), 1, 0.01), cs.weak_voxel_row(pb, (2, 3, 1), 2, -0.01),
            cs.weak_face_row(pb, 2, 4, (1, 1), 2, -0.02),
            cs.tie_row(pb, [(3, 4, 4), (4, 4, 4), (3, 5, 4)], 0, -0.01)]
    uk, fk = kkt.solve_kkt(pb, rows, cs.targets(pb, rows))
    res = sv.solve_alg1(pb, rows, 1.5, 1.0, 1e-13, 3000, acv_on=acv_on, acv_mod=2)
    assert res.converged
    assert np.abs(res.u - uk).max() <= 1e-10 * np.abs(uk).max()
    assert np.abs(res.f - fk).max() <= 1e-10 * np.abs(fk).max()


def _golden_weights():
    out = {}
    with open(os.path.join(GOLDEN, "smooth_weights.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            name, wme, wmf, wco, nme, nmf, nco, tot = line.split()
            out[name] = (float(wme), None if wmf == "-" else float(wmf), float(wco),
                         int(nme), int(nmf), int(nco), float(tot))
    return out


def test_smooth_weights_match_paper_table():
    """P8: weights and total reaction factor of smooth rows (Section 4.2.2 table)."""
    g = _golden_weights()
    bc = np.full((3, 2, 3), N)
    pb = dz.Problem((4, 4, 4), 1.0, bc, dz.TETRA2, np.zeros((4, 4, 4)), [1.0], [1.0])
    vol = cs.smooth_row(pb, (2, 2, 2), 0, 0.0)
    surf = cs.smooth_row(pb, (2, 2, 4), 0, 0.0)
    for row, key in ((vol, "volume"), (surf, "surface")):
        wme, wmf, wco, nme, nmf, nco, tot = g[key]
        b = np.sort(row.b[1:])
        expect = [wco] * nco + [wme] * nme + ([wmf] * nmf if wmf else [])
        assert np.allclose(b, np.sort(expect))
        assert abs(np.sum(row.b) - tot) < 1e-15
        assert row.a[0] == 1.0 and np.all(row.a[1:] == 0.0)


def test_tetra2_subgrids_decouple():
    """P9 (Section 4.2.3, Fig. 6): a strong load on a single node moves only the nodes of
    its parity sub-grid; the other sub-grid stays at rest."""
    lam, mu = wl.lame(1.0, 0.3)
    bc = np.full((3, 2, 3), D)
    pb = dz.Problem((6, 6, 6), 1.0, bc, dz.TETRA2, np.zeros((6, 6, 6)), [lam], [mu])
    rows = [cs.strong_row(pb, (3, 3, 2), 2, 0.1)]
    res = sv.solve_alg1(pb, rows, lam, mu, 1e-12, 2000)
    k, j, i = np.meshgrid(*[np.arange(7)] * 3, indexing="ij")
    par = (i + j + k) % 2
    assert res.converged
    assert np.abs(res.u[:, par == 1]).max() < 1e-13
    assert np.abs(res.u[:, par == 0]).max() > 1e-3


def test_reaction_balance_and_acv_order():
    """P7 on a miniature of the paper's half CT-like set-up (Section 4.1.2, Fig. 2): a
    zero-stiffness buffer layer below the ligament carries the Dirichlet face of the
    opening component; the ligament nodes are held at u_y = 0 and a line of nodes is
    pulled.  The two reactions balance (R_S + R_L = 0, Section 4.1.3; the paper reports
    a relative imbalance of 5e-12 at convergence) with either accelerated quantity.
    (The paper's iteration counts -- ACV_P faster than ACV_U on its CT specimen -- are
    not a property of every problem and are not asserted.)"""
    lam, mu = wl.lame(1.0, 0.3)
    nx, ny, nz = 6, 9, 3
    bc = np.full((3, 2, 3), N)
    bc[1, 0, 1] = D
    ph = np.zeros((nz, ny, nx), np.uint8)
    ph[:, 0, :] = 1                                   # buffer layer y in [0, 1)
    pb = dz.Problem((nx, ny, nz), 1.0, bc, dz.TETRA2, ph, [lam, 0.0], [mu, 0.0])
    rows, lig, line = [], [], []
    for k in range(nz + 1):
        for i in range(nx + 1):
            if i >= 3:
                lig.append(len(rows))
                rows.append(cs.strong_row(pb, (i, 1, k), 1, 0.0))
            line.append(len(rows))
            rows.append(cs.strong_row(pb, (i, 6, k), 1, 0.1))
    for acv_on in ("P", "U"):
        res = sv.solve_alg1(pb, rows, lam / 2, mu / 2, 1e-10, 3000, acv_on=acv_on, acv_mod=2)
        assert res.converged
        RS = res.reactions[lig].sum()
        RL = res.reactions[line].sum()
        assert abs(RS + RL) < 1e-9 * abs(RL)
        assert abs(res.total_reaction[1]) < 1e-9 * abs(RL)


def test_null_mode_components_reject_constraints():
    """All-Neumann component + a constraint row: rejected (no fixed point exists)."""
    bc = np.full((3, 2, 3), N)
    pb = dz.Problem((4, 4, 4), 1.0, bc, dz.TETRA2, np.zeros((4, 4, 4)), [1.0], [1.0])
    with pytest.raises(ValueError):
        cs.check_rows(pb, [cs.strong_row(pb, (1, 1, 1), 0, 0.0)])
    assert dz.has_null_modes(pb, 0)
    bc[0, 0, 0] = D
    pb = dz.Problem((4, 4, 4), 1.0, bc, dz.TETRA2, np.zeros((4, 4, 4)), [1.0], [1.0])
    assert not dz.has_null_modes(pb, 0)
    pbh = dz.Problem((4, 4, 4), 1.0, bc, dz.HEX1, np.zeros((4, 4, 4)), [1.0], [1.0])
    assert dz.has_null_modes(pbh, 0)       # hourglass: q_y = q_z = pi


def _indent(nx, nz, R, ratios):
    w = wl.indentation(nx, nx, nz, R=R, steps=len(ratios), dmin=ratios[0], dmax=ratios[-1])
    pb = dz.problem_from(w)
    return w, pb


def test_contact_complementarity_and_balance():
    """P5 + P7: after each increment of Algorithm 2: gap >= 0 on the surface, normal
    reaction <= 0 on the contact zone, gap * reaction = 0 (Eq. 33), and the total
    contact force equals A0 e3.<sigma>.e3 (Section 5.4)."""
    w, pb = _indent(16, 8, 6.0, [0.01, 0.05])
    I = w.indenter
    u = np.zeros((3,) + pb.node_shape)
    for O in I["centers"]:
        ind = cs.Indenter(pb, I["axis"], I["face"], O, I["radius"])
        res = sv.solve_alg2_increment(pb, ind, [], w.lam0, w.mu0, 1e-9, 2000, u)
        u = res.u
        assert res.converged
        act = res.active
        assert act.any()
        fmax = np.abs(res.fn[act]).max()
        assert res.gap.min() >= -1e-10 * I["radius"]
        assert res.fn[act].max() <= 1e-10 * fmax
        assert np.abs(res.gap[act]).max() < 1e-10
        ms = sv.mean_stress(pb, res.sigma)
        assert abs(ms[2, 2] * pb.nvox[0] * pb.nvox[1] - res.force[2]) < 1e-9 * abs(res.force[2])


def test_hertz_trend_coarse():
    """P6 (weak form on a coarse grid): the force follows the Hertz law (Eq. 30) to
    within 25% and grows like delta^(3/2) between the two increments (within 15%)."""
    w, pb = _indent(24, 12, 8.0, [0.02, 0.05])
    I = w.indenter
    u = np.zeros((3,) + pb.node_shape)
    F = []
    for O, r in zip(I["centers"], I["ratios"]):
        ind = cs.Indenter(pb, I["axis"], I["face"], O, I["radius"])
        res = sv.solve_alg2_increment(pb, ind, [], w.lam0, w.mu0, 1e-8, 2000, u)
        u = res.u
        F.append(-res.force[2])
        Fh = hertz.hertz_force(I["E"], I["nu"], I["radius"], r * I["radius"])
        assert abs(F[-1] / Fh - 1.0) < 0.25
    expo = np.log(F[1] / F[0]) / np.log(I["ratios"][1] / I["ratios"][0])
    assert abs(expo - 1.5) < 0.15 * 1.5


def test_anderson_skips_singular_gram():
    """A Gram matrix with a repeated residual is singular: the step is skipped."""
    a = sv.Anderson(mod=2)
    x = np.ones(5)
    for i in range(5):
        y = a.step(i, x.copy())
    assert a.accelerated == 0
    assert np.array_equal(y, x)


def test_constraint_validation():
    bc = np.full((3, 2, 3), N)
    bc[0, 0, 0] = D
    pb = dz.Problem((3, 3, 3), 1.0, bc, dz.TETRA2, np.zeros((3, 3, 3)), [1.0], [1.0])
    with pytest.raises(ValueError):
        cs.check_rows(pb, [cs.strong_row(pb, (0, 1, 1), 0, 0.0)])
    with pytest.raises(ValueError):
        cs.check_rows(pb, [cs.strong_row(pb, (1, 1, 1), 1, 0.0), cs.weak_voxel_row(pb, (1, 1, 1), 1, 0.0)])


def test_contact_solution_is_a_kkt_point_of_the_assembled_energy():
    """Pin of Algorithm 2 against the plain definition of the contact problem (Section 5.1,
    Eq. 33): the converged increments minimise the discrete energy over the points outside
    the sphere.  With K and the prescribed-strain force assembled element by element in
    kkt.py (independently of the solver's operators), the energy gradient r = K u~ + F* at
    the oracle's solution vanishes at every free DOF off the contact zone, is normal to the
    sphere at every contact node (no tangential part: frictionless), points into the body
    (a non-negative multiplier of the constraint g >= 0, whose gradient is -n_c), and its
    normal part is the reported reaction f_n, whose sum is the reported force."""
    w = wl.indentation(10, 10, 6, R=4.0, steps=2, dmin=0.05, dmax=0.15)
    pb = dz.problem_from(w)
    I = w.indenter
    K, Fs = kkt.assemble(pb)
    nn = int(np.prod(pb.node_shape))
    free = np.concatenate([pb.dof_mask(c).ravel() for c in range(3)])
    u = np.zeros((3,) + pb.node_shape)
    for O in I["centers"]:
        ind = cs.Indenter(pb, I["axis"], I["face"], O, I["radius"])
        res = sv.solve_alg2_increment(pb, ind, [], w.lam0, w.mu0, 1e-11, 5000, u)
        assert res.converged
        u = res.u
        r = K @ u.ravel() + Fs
        act = res.active
        an = ind.nodes[act]
        assert act.sum() >= 5
        cdofs = np.concatenate([an + c * nn for c in range(3)])
        assert free[cdofs].all()
        off = free.copy()
        off[cdofs] = False
        R3 = np.stack([r[an + c * nn] for c in range(3)])
        scale = np.abs(R3).max()
        assert np.abs(r[off]).max() <= 1e-11 * scale
        _, n = cs.contact_geometry(pb, ind, u)
        N3 = n[:, act]
        rn = (R3 * N3).sum(axis=0)
        assert np.abs(R3 - rn * N3).max() <= 1e-11 * scale
        assert (rn < 0).all()
        assert np.allclose(rn, res.fn[act], rtol=1e-10, atol=1e-12 * scale)
        assert abs(R3[2].sum() - res.force[2]) <= 1e-10 * abs(res.force[2])
