"""Pins of the finite-strain oracle (oracle.discrete.piola, the FS solver loops) against
facts outside it:

  * the nodal force from Pi is the gradient of the discrete St Venant-Kirchhoff energy
    sum_vox sum_t w_t h^3 (lambda/2 (tr E)^2 + mu E:E), checked by central differences
    (pins Pi = F.S, its index order and its pairing with grad u);
  * a finite rigid rotation carries no stress (frame indifference of S = C:E), while the
    small-strain stress of the same field is large;
  * small displacements give the small-strain residual to first order;
  * the FS solver reaches the textbook homogeneous uniaxial stretch of a St Venant-Kirchhoff
    bar (lateral Green-Lagrange strain -nu E_zz, S_zz = Young * E_zz) and Section 5.4's
    force A0 e.<Pi>.e equals the sum of the Dirichlet-face reactions.
"""
import numpy as np
import pytest

from oracle import discrete as dz
from oracle import solver as osv

P, D, N = 0, 1, 2


def _problem(nvox, bc, scheme, lam=(1.0, 2.5), mu=(0.8, 1.7), seed=0, eps=None, h=1.0):
    rng = np.random.default_rng(seed)
    phase = rng.integers(0, len(lam), size=tuple(reversed(nvox))).astype(np.uint8)
    return dz.Problem(nvox, h, bc, scheme, phase, np.array(lam), np.array(mu), eps)


def _energy(pb, u):
    """Discrete St Venant-Kirchhoff energy, written from its definition."""
    g = dz.gradients(pb, u)
    Fm = g + pb.eps_star[None, :, :, None, None, None] + np.eye(3)[None, :, :, None, None, None]
    C = np.einsum("tkazyx,tkbzyx->tabzyx", Fm, Fm)
    E = 0.5 * (C - np.eye(3)[None, :, :, None, None, None])
    lam, mu = pb.material()
    trE = E[:, 0, 0] + E[:, 1, 1] + E[:, 2, 2]
    W = 0.5 * lam * trE ** 2 + mu * np.sum(E * E, axis=(1, 2))
    w = np.array([ip[0] for ip in pb.ip_sets()])
    return pb.h ** 3 * float(np.sum(w[:, None, None, None] * W))


@pytest.mark.parametrize("scheme", [dz.TETRA2, dz.HEX1])
@pytest.mark.parametrize("periodic_x", [False, True])
def test_piola_force_is_energy_gradient(scheme, periodic_x):
    bc = np.full((3, 2, 3), N)
    bc[2, 0, :] = D
    if periodic_x:
        bc[0] = P
    pb = _problem((3, 2, 2), bc, scheme, seed=1, h=0.7,
                  eps=np.array([[0.02, 0.01, 0.0], [0.01, -0.03, 0.005], [0.0, 0.005, 0.04]]))
    rng = np.random.default_rng(2)
    u = 0.15 * rng.standard_normal((3,) + pb.node_shape)
    Fn = dz.nodal_force(pb, dz.piola(pb, u))
    hstep = 1e-6
    worst = 0.0
    for c in range(3):
        for idx in np.ndindex(pb.node_shape):
            up, um = u.copy(), u.copy()
            up[(c,) + idx] += hstep
            um[(c,) + idx] -= hstep
            fd = (_energy(pb, up) - _energy(pb, um)) / (2 * hstep)
            worst = max(worst, abs(fd - Fn[(c,) + idx]))
    assert worst <= 1e-7 * max(1.0, np.abs(Fn).max())


@pytest.mark.parametrize("scheme", [dz.TETRA2, dz.HEX1])
def test_rigid_rotation_is_stress_free(scheme):
    bc = np.full((3, 2, 3), N)
    pb = _problem((4, 3, 5), bc, scheme, seed=3)
    th = 0.6   # a finite rotation about the axis (1, 2, 2) / 3
    a = np.array([1.0, 2.0, 2.0]) / 3.0
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    Q = np.eye(3) + np.sin(th) * K + (1 - np.cos(th)) * K @ K
    z, y, x = np.meshgrid(*[np.arange(n) * pb.h for n in pb.node_shape], indexing="ij")
    X = np.stack([x, y, z])
    u = np.einsum("ab,bzyx->azyx", Q - np.eye(3), X)
    Pi = dz.piola(pb, u)
    sig = dz.stress(pb, u)
    assert np.abs(Pi).max() <= 1e-13
    assert np.abs(sig).max() >= 0.1   # the small-strain stress of the same field is not small
    p, _ = dz.residual(pb, u, "FS")
    assert np.abs(p).max() <= 1e-12


def test_small_displacements_give_the_small_strain_residual():
    bc = np.full((3, 2, 3), N)
    bc[2, 0, :] = D
    bc[0] = P
    pb = _problem((4, 4, 3), bc, dz.TETRA2, seed=4)
    u = np.random.default_rng(5).standard_normal((3,) + pb.node_shape)
    for s in (1e-4, 1e-6):
        pf, _ = dz.residual(pb, s * u, "FS")
        ps, _ = dz.residual(pb, s * u, "SS")
        rel = np.linalg.norm(pf - ps) / np.linalg.norm(ps)
        assert rel <= 20 * s   # the difference is quadratic in u, relative O(s)
    assert rel >= 1e-9         # ... and it is there


@pytest.mark.parametrize("scheme", [dz.TETRA2, dz.HEX1])
def test_uniaxial_stretch_closed_form(scheme):
    """u_z prescribed by the lift (E_zz on a bar clamped in z between its end faces, the
    lateral faces free, the x = 0 / y = 0 faces symmetry planes): the discrete solution is
    homogeneous and the St Venant-Kirchhoff bar contracts laterally by E_xx = -nu E_zz."""
    lam, mu = 1.2, 0.8
    nu = lam / (2 * (lam + mu))
    young = mu * (3 * lam + 2 * mu) / (lam + mu)
    ez = 0.06
    nv = (3, 4, 4)
    bc = np.full((3, 2, 3), N)
    bc[0, 0, 0] = D            # u_x = 0 on x = 0
    bc[1, 0, 1] = D            # u_y = 0 on y = 0
    bc[2, :, 2] = D            # u~_z = 0 on both z faces: u_z = ez z from the lift
    eps = np.zeros((3, 3))
    eps[2, 2] = ez
    pb = _problem(nv, bc, scheme, lam=(lam,), mu=(mu,), eps=eps)
    res = osv.solve_alg1(pb, [], 2 * lam, 2 * mu, 1e-13, 3000, acv_mod=2, kinematics="FS")
    assert res.converged, res.residual
    Ezz = ((1 + ez) ** 2 - 1) / 2
    b = np.sqrt(1 - 2 * nu * Ezz) - 1          # lateral stretch - 1
    z, y, x = np.meshgrid(*[np.arange(n) * pb.h for n in pb.node_shape], indexing="ij")
    assert np.abs(res.u[0] - b * x).max() <= 1e-10
    assert np.abs(res.u[1] - b * y).max() <= 1e-10
    assert np.abs(res.u[2]).max() <= 1e-10
    mean = osv.mean_stress(pb, res.sigma)
    Pzz = (1 + ez) * young * Ezz
    assert abs(mean[2, 2] - Pzz) <= 1e-10 * Pzz
    assert np.abs(mean - np.diag([0, 0, Pzz])).max() <= 1e-10 * Pzz
    # Section 5.4's force A0 e.<Pi>.e against the sum of the nodal forces on the z = n face
    F = dz.nodal_force(pb, res.sigma)
    top = F[2][-1].sum()
    area = nv[0] * nv[1] * pb.h ** 2
    assert abs(top - area * mean[2, 2]) <= 1e-10 * area * Pzz


def _indent_fs(nx, nz, R):
    import workloads as wl
    w = wl.indentation(nx, nx, nz, R=R, steps=2, dmin=0.01, dmax=0.05)
    return w, dz.problem_from(w)


def test_fs_contact_complementarity_and_balance():
    """Algorithm 3 increments: gap >= 0 on the surface, normal reaction <= 0 on the contact
    zone, gap * reaction = 0 (Eq. 33, unchanged in finite strain, Section 5.2), and the
    contact force equals A0 e3.<Pi>.e3 (Section 5.4)."""
    from oracle import constraints as cs
    w, pb = _indent_fs(16, 8, 6.0)
    I = w.indenter
    u = np.zeros((3,) + pb.node_shape)
    for O in I["centers"]:
        ind = cs.Indenter(pb, I["axis"], I["face"], O, I["radius"])
        res = osv.solve_alg2_increment(pb, ind, [], w.lam0, w.mu0, 1e-9, 3000, u, kinematics="FS")
        u = res.u
        assert res.converged
        act = res.active
        assert act.any()
        fmax = np.abs(res.fn[act]).max()
        assert res.gap.min() >= -1e-10 * I["radius"]
        assert res.fn[act].max() <= 1e-10 * fmax
        assert np.abs(res.gap[act]).max() < 1e-10
        ms = osv.mean_stress(pb, res.sigma)
        assert abs(ms[2, 2] * pb.nvox[0] * pb.nvox[1] - res.force[2]) < 1e-9 * abs(res.force[2])


def test_fs_contact_tends_to_small_strain():
    """With the same contact zone, the FS force departs from the SS force by an amount
    first order in the depth (Section 5.4: the two agree at small depth ratios and depart
    as the ratio grows); the SS force is linear in the depth."""
    from oracle import constraints as cs
    w, pb = _indent_fs(12, 6, 5.0)
    I = w.indenter
    F = {}
    for r in (0.0005, 0.005):
        O = np.array([6.0, 6.0, 6.0 + 5.0 - r * 5.0])
        for kin in ("SS", "FS"):
            ind = cs.Indenter(pb, I["axis"], I["face"], O, I["radius"])
            res = osv.solve_alg2_increment(pb, ind, [], w.lam0, w.mu0, 1e-11, 3000,
                                           np.zeros((3,) + pb.node_shape), kinematics=kin)
            assert res.converged
            F[kin, r] = (-res.force[2], int(res.active.sum()))
    assert F["SS", 0.0005][1] == F["SS", 0.005][1] == F["FS", 0.0005][1] == F["FS", 0.005][1]
    assert abs(F["SS", 0.005][0] / F["SS", 0.0005][0] - 10.0) < 1e-8
    d1 = F["FS", 0.0005][0] / F["SS", 0.0005][0] - 1.0
    d2 = F["FS", 0.005][0] / F["SS", 0.005][0] - 1.0
    assert abs(d2) > 1e-3 and abs(d2 / d1 - 10.0) < 0.5


def test_fs_contact_solution_is_stationary_for_the_svk_energy():
    """Pin of Algorithm 3's converged increments against the energy they minimise over the
    points outside the sphere (Section 5.2 with Eq. 33): central differences of the discrete
    St Venant-Kirchhoff energy (_energy, written from its definition, not from the solver's
    Pi) vanish along a random direction of the free DOFs off the contact zone and along the
    sphere's tangent at every contact node, and along the normal n_c of a contact node they
    equal the reported reaction f_n (negative: the multiplier of g >= 0 is non-negative)."""
    from oracle import constraints as cs
    w = __import__("workloads").indentation(10, 10, 6, R=4.0, steps=2, dmin=0.05, dmax=0.15)
    pb = dz.problem_from(w)
    I = w.indenter
    free = np.stack([pb.dof_mask(c) for c in range(3)])
    rng = np.random.default_rng(1)
    u = np.zeros((3,) + pb.node_shape)
    step = 1e-6

    def slope(v):
        return (_energy(pb, u + step * v) - _energy(pb, u - step * v)) / (2 * step)

    for O in I["centers"]:
        ind = cs.Indenter(pb, I["axis"], I["face"], O, I["radius"])
        res = osv.solve_alg2_increment(pb, ind, [], w.lam0, w.mu0, 1e-11, 5000, u, kinematics="FS")
        assert res.converged
        u = res.u
        act = res.active
        an = ind.nodes[act]
        assert act.sum() >= 5
        fn = res.fn[act]
        tol = 1e-8 * np.abs(fn).max()
        _, n = cs.contact_geometry(pb, ind, u)
        v = rng.standard_normal(u.shape) * free
        v.reshape(3, -1)[:, an] = 0.0
        assert abs(slope(v / np.linalg.norm(v))) <= tol
        for j, M in enumerate(an):
            nv = n[:, act][:, j]
            t = np.cross(nv, [1.0, 0.3, 0.0])
            t /= np.linalg.norm(t)
            for d, want in ((nv, fn[j]), (t, 0.0)):
                e = np.zeros_like(u)
                e.reshape(3, -1)[:, M] = d
                assert abs(slope(e) - want) <= tol, (M, slope(e), want)
        assert (fn < 0).all()
