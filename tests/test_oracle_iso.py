"""Pins of the isotropic-reference-medium oracle (Section 3.2.3, Eq. 4) against facts
outside it:

  * the dense Green step (discrete.green_apply_dense: A0^-1 with null modes removed in the
    W inner product) reproduces the spectral Green step of the Paux medium on grids with
    every kind of boundary condition, periodic axes and null modes included -- so the
    dense construction is the spectral step;
  * the isotropic A0 is the gradient of the discrete quadratic energy
    sum w h^3 (lambda0 (tr G)^2 + mu0 G : (G + G^T)) / 2 (central differences);
  * on HEX1 grids with normal mixed conditions the dense isotropic Green step maps a single
    DTT mode to the same mode of every component with the coefficients of Eq. 4 (the
    inverse of mu0 |xi|^2 1 + (lambda0 + mu0) xi xi^T, by the Sherman-Morrison formula the
    paper prints), xi the HEX1 modified wave vector, its entries signed by the parity of
    each axis' normal transform;
  * the isotropic Algorithm 1 reaches the closed form of a layered cell between sliding walls.
"""
import itertools

import numpy as np
import pytest

from oracle import discrete as dz, solver as osv, transforms as otr

P, D, N = 0, 1, 2


def _problem(nvox, bc, scheme, seed=0, eps=None, h=1.0, nphase=2):
    rng = np.random.default_rng(seed)
    phase = rng.integers(0, nphase, size=tuple(reversed(nvox))).astype(np.uint8)
    lam, mu = np.array([1.0, 2.5])[:nphase], np.array([0.8, 1.7])[:nphase]
    return dz.Problem(nvox, h, bc, scheme, phase, lam, mu, eps)


def _normal_mixed_bc(normal_types):
    """normal_types[d][f] in (D, N): the normal component's condition on face f of axis d;
    the tangential components take the other one."""
    bc = np.zeros((3, 2, 3), dtype=np.int64)
    for d in range(3):
        for f in range(2):
            nt = normal_types[d][f]
            for c in range(3):
                bc[d, f, c] = nt if c == d else (N if nt == D else D)
    return bc


def _p(pb, seed):
    p = np.random.default_rng(seed).standard_normal((3,) + pb.node_shape)
    for c in range(3):
        p[c][~pb.dof_mask(c)] = 0.0
    return p


@pytest.mark.parametrize("scheme", [dz.TETRA2, dz.HEX1])
@pytest.mark.parametrize("case", range(4))
def test_dense_green_is_the_spectral_green_step(scheme, case):
    rng = np.random.default_rng(100 + case)
    bc = rng.choice([D, N], size=(3, 2, 3))
    if case == 1:
        bc[0] = P
    if case == 2:
        bc[:] = N          # null modes on every component
    if case == 3:
        bc[1] = P
        bc[2] = P
    pb = _problem((3, 4, 3), bc, scheme, seed=case)
    p = _p(pb, case)
    ref = dz.green_apply(pb, p, 1.3, 0.9)
    got = dz.green_apply_dense(pb, p, lambda u: dz.apply_A0(pb, u, 1.3, 0.9))
    assert np.abs(got - ref).max() <= 1e-10 * np.abs(ref).max()


@pytest.mark.parametrize("scheme", [dz.TETRA2, dz.HEX1])
def test_iso_operator_is_energy_gradient(scheme):
    bc = _normal_mixed_bc([[D, N], [N, N], [D, D]])
    pb = _problem((3, 2, 3), bc, scheme, h=0.8)
    lam0, mu0 = 1.1, 0.7
    w = np.array([ip[0] for ip in pb.ip_sets()])

    def energy(u):
        g = dz.gradients(pb, u)
        tr = g[:, 0, 0] + g[:, 1, 1] + g[:, 2, 2]
        dens = lam0 * tr ** 2 + mu0 * np.sum(g * (g + np.swapaxes(g, 1, 2)), axis=(1, 2))
        return 0.5 * pb.h ** 3 * float(np.sum(w[:, None, None, None] * dens))

    u = np.random.default_rng(3).standard_normal((3,) + pb.node_shape)
    Au = dz.apply_A0_iso(pb, u, lam0, mu0)
    hs = 1e-5
    for c in range(3):
        W = pb.weight_W(c)
        for idx in np.ndindex(pb.node_shape):
            if not pb.dof_mask(c)[idx]:
                continue
            up, um = u.copy(), u.copy()
            up[(c,) + idx] += hs
            um[(c,) + idx] -= hs
            fd = (energy(up) - energy(um)) / (2 * hs)
            assert abs(fd - Au[(c,) + idx] * pb.h ** 3 * W[idx]) <= 1e-7 * max(1.0, abs(fd))


@pytest.mark.parametrize("normal", [[[D, D], [N, N], [D, N]], [[N, D], [D, D], [N, N]]])
def test_iso_green_of_a_mode_follows_eq4_hex1(normal):
    """HEX1, normal mixed conditions: u = G(p) for p a single interior DTT mode of one
    component is that mode in every component, with the coefficients of Eq. 4."""
    bc = _normal_mixed_bc(normal)
    nvox = (4, 5, 4)
    pb = dz.Problem(nvox, 1.0, bc, dz.HEX1, np.zeros(tuple(reversed(nvox)), np.uint8),
                    np.array([1.0]), np.array([0.8]))
    lam0, mu0 = 1.4, 0.9
    a0 = lambda u: dz.apply_A0_iso(pb, u, lam0, mu0)     # noqa: E731
    # sin-like normal transform on axis d -> +1, cos-like -> -1
    eps = np.array([1.0 if pb.types[d][d] in (otr.DST1, otr.DST3) else -1.0 for d in range(3)])
    for c0, (kx, ky, kz) in itertools.product(range(3), [(1, 2, 1), (2, 1, 2), (1, 3, 2)]):
        q = []
        Xs = []
        for c in range(3):
            qc = otr.wave_numbers(pb.types[c], nvox)
            Xs.append(np.zeros((len(qc[2]), len(qc[1]), len(qc[0]))))
            q.append(qc)
        # the mode's wave vector, then its index on every component's spectral grid
        qx = q[c0][0][min(kx, len(q[c0][0]) - 1)]
        qy = q[c0][1][min(ky, len(q[c0][1]) - 1)]
        qz = q[c0][2][min(kz, len(q[c0][2]) - 1)]
        idx = []
        ok = True
        for c in range(3):
            ii = [np.flatnonzero(np.isclose(q[c][d], v)) for d, v in enumerate((qx, qy, qz))]
            if any(len(a) == 0 for a in ii):
                ok = False
                break
            idx.append((ii[2][0], ii[1][0], ii[0][0]))
        if not ok or min(np.sin([qx, qy, qz])) < 1e-9:
            continue
        Xs[c0][idx[c0]] = 1.0
        p = np.stack([otr.inverse_3d(Xs[c], pb.types[c], nvox) for c in range(3)])
        u = dz.green_apply_dense(pb, p, a0)
        Y = [otr.forward_3d(u[c], pb.types[c], nvox) for c in range(3)]
        # HEX1 modified wave vector: xi_d = 2 sin(q_d / 2) cos(q_e / 2) cos(q_f / 2)
        qv = np.array([qx, qy, qz])
        xi = np.array([2 * np.sin(qv[d] / 2) * np.prod([np.cos(qv[e] / 2) for e in range(3) if e != d])
                       for d in range(3)]) * eps
        x2 = xi @ xi
        # Eq. 4 (Sherman-Morrison form): u = p / (mu0 |xi|^2) - (lambda0 + mu0) (p.xi) xi / ((lambda0 + 2 mu0) mu0 |xi|^4)
        e0 = np.zeros(3)
        e0[c0] = 1.0
        expect = e0 / (mu0 * x2) - (lam0 + mu0) * (e0 @ xi) * xi / ((lam0 + 2 * mu0) * mu0 * x2 * x2)
        for c in range(3):
            got = Y[c][idx[c]]
            assert abs(got - expect[c]) <= 1e-9 * np.abs(expect).max(), (c0, c, got, expect[c])
            rest = Y[c].copy()
            rest[idx[c]] = 0.0
            assert np.abs(rest).max() <= 1e-9 * np.abs(expect).max()


@pytest.mark.parametrize("scheme", [dz.TETRA2, dz.HEX1])
def test_iso_solver_laminate_closed_form(scheme):
    """A two-layer laminate stacked along z between sliding walls (normal Dirichlet,
    tangential Neumann on every face), stretched by the lift eps*_zz: the solution is one
    dimensional, sigma_zz is the same in both layers and the lateral strains vanish, so
    each layer strains by sigma_zz / (lambda_i + 2 mu_i) (exact for both schemes: the
    field is linear in every voxel)."""
    bc = _normal_mixed_bc([[D, D], [D, D], [D, D]])
    nvox = (2, 3, 4)
    phase = np.zeros((4, 3, 2), np.uint8)
    phase[2:] = 1
    lam, mu = np.array([1.0, 3.0]), np.array([0.7, 2.0])
    ez = 0.01
    pb = dz.Problem(nvox, 1.0, bc, scheme, phase, lam, mu, np.diag([0.0, 0.0, ez]))
    res = osv.solve_alg1(pb, [], 2 * lam.mean(), 2 * mu.mean(), 1e-12, 3000, acv_mod=2, medium="iso")
    assert res.converged
    M = lam + 2 * mu
    sig = ez * 4 / (2 / M[0] + 2 / M[1])     # both layers 2 voxels thick
    e = sig / M - ez                          # d u~_z / dz per layer
    z = np.arange(5.0)
    uz = np.where(z <= 2, e[0] * z, e[0] * 2 + e[1] * (z - 2))
    assert np.abs(res.u[2] - uz[:, None, None]).max() <= 1e-10
    assert np.abs(res.u[0]).max() <= 1e-10 and np.abs(res.u[1]).max() <= 1e-10


def _axis_forward(ttype, n):
    """Forward transform of one axis with the spectral index k of the library (DST1: k = 1
    .. n-1 at index k); a periodic axis takes the Hartley transform sum_j x_j cas(2 pi j k / n)."""
    if ttype == otr.DFT:
        a = 2 * np.pi * np.outer(np.arange(n), np.arange(n)) / n
        return np.cos(a) + np.sin(a)
    F = otr.forward_matrix(ttype, n)
    _, kidx, _ = otr.selection(ttype, n)
    full = np.zeros((n + 1, n + 1))
    for a, k in enumerate(kidx):
        full[k] = F[a]
    return full


def _axis_inverse(ttype, n):
    if ttype == otr.DFT:
        a = 2 * np.pi * np.outer(np.arange(n), np.arange(n)) / n
        return (np.cos(a) + np.sin(a)) / n
    B = otr.inverse_matrix(ttype, n)
    _, kidx, _ = otr.selection(ttype, n)
    full = np.zeros((n + 1, n + 1))
    for a, k in enumerate(kidx):
        full[:, k] = B[:, a]
    return full


@pytest.mark.parametrize("scheme", [dz.TETRA2, dz.HEX1])
@pytest.mark.parametrize("periodic", [(1, 0, 0), (0, 1, 1), (1, 1, 1)])
def test_iso_operator_couples_partner_positions(scheme, periodic):
    """The isotropic A0 (Section 3.2.3) in the per-axis bases: along a periodic axis the
    Hartley cas(q x) is mapped by a first difference onto cas(-q x), so the operator couples
    u_x at q with u_y at q flipped on the periodic axes of {x, y} and u_z at q flipped on
    those of {x, z}, and nothing else; the 3 x 3 blocks are M_cc = 4 ((lambda0 + mu0) S_c +
    mu0 sum S) and M_cd = (lambda0 + mu0) sign_c sign_d tau_cd sin q_c sin q_d (times
    cos^2(q_e / 2) for HEX1), sines signed at the x position on periodic axes, sign_d = +1
    for a sine-type normal transform along d (-1 otherwise, a periodic axis -1), tau = -1 for
    the pairs with x when x is periodic.  Checked entry by entry on the operator's spectral
    matrix (h = 1)."""
    rng = np.random.default_rng(7)
    normal = rng.choice([D, N], size=(3, 2))
    bc = _normal_mixed_bc(normal)
    for d in range(3):
        if periodic[d]:
            bc[d] = P
    nvox = (4, 5, 3)
    pb = dz.Problem(nvox, 1.0, bc, scheme, np.zeros(tuple(reversed(nvox)), np.uint8), np.array([1.0]),
                    np.array([1.0]))
    lam0, mu0 = 0.7, 0.4
    nx, ny, nz = pb.nn
    n_all = nx * ny * nz
    F = np.zeros((3 * n_all, 3 * n_all))
    B = np.zeros_like(F)
    for c in range(3):
        fx, fy, fz = (_axis_forward(pb.types[c][d], nvox[d]) for d in range(3))
        bx, by, bz = (_axis_inverse(pb.types[c][d], nvox[d]) for d in range(3))
        F[c * n_all:(c + 1) * n_all, c * n_all:(c + 1) * n_all] = np.kron(fz, np.kron(fy, fx))
        B[c * n_all:(c + 1) * n_all, c * n_all:(c + 1) * n_all] = np.kron(bz, np.kron(by, bx))
    A = np.zeros_like(F)
    for e in range(3 * n_all):
        u = np.zeros(3 * n_all)
        u[e] = 1.0
        A[:, e] = dz.apply_A0_iso(pb, u.reshape((3, nz, ny, nx)), lam0, mu0).reshape(-1)
    S = F @ A @ B
    qv = [[dict(zip(otr.selection(pb.types[c][d], nvox[d])[1], otr.selection(pb.types[c][d], nvox[d])[2]))
           for d in range(3)] for c in range(3)]
    sgn = [1.0 if pb.types[d][d] in (otr.DST1, otr.DST3) else -1.0 for d in range(3)]
    lm = lam0 + mu0

    def flip(pos, axes):
        return tuple(((-p) % pb.nn[a]) if (a in axes and periodic[a]) else p for a, p in enumerate(pos))

    def idx(c, pos):
        return c * n_all + (pos[2] * ny + pos[1]) * nx + pos[0]

    for k, j, i in itertools.product(range(nz), range(ny), range(nx)):
        q = (i, j, k)
        pos = [q, flip(q, (0, 1)), flip(q, (0, 2))]
        on = [all(pos[c][d] in qv[c][d] for d in range(3)) for c in range(3)]
        rows = [idx(c, pos[c]) for c in range(3)]
        for c in range(3):
            if not on[c]:
                continue
            # nothing outside the triple
            others = np.delete(S[rows[c]], [rows[d] for d in range(3) if on[d]])
            assert np.abs(others).max() <= 1e-12
            qq = [qv[c][d][pos[c][d]] for d in range(3)]
            s = [np.sin(x / 2) ** 2 for x in qq]
            cp = [np.cos(x / 2) ** 2 for x in qq]
            if scheme == dz.TETRA2:
                Sx = s[0] * cp[1] + s[2] * (s[1] - s[0])
                Sy = s[1] * cp[2] + s[0] * (s[2] - s[1])
                Sz = s[2] * cp[0] + s[1] * (s[0] - s[2])
            else:
                Sx, Sy, Sz = s[0] * cp[1] * cp[2], s[1] * cp[0] * cp[2], s[2] * cp[0] * cp[1]
            assert abs(S[rows[c], rows[c]] - 4 * (lm * (Sx, Sy, Sz)[c] + mu0 * (Sx + Sy + Sz))) <= 1e-12
            for d in range(3):
                if d == c or not on[d]:
                    continue
                e = 3 - c - d

                def sine(a):
                    if periodic[a]:
                        return np.sin(2 * np.pi * q[a] / nvox[a])
                    return np.sin(qv[c][a][pos[c][a]] if a == c else qv[d][a][pos[d][a]])

                tau = -1.0 if (periodic[0] and 0 in (c, d)) else 1.0
                want = lm * sgn[c] * sgn[d] * tau * sine(c) * sine(d)
                if scheme == dz.HEX1:
                    want *= np.cos(qv[c][e][pos[c][e]] / 2) ** 2
                assert abs(S[rows[c], rows[d]] - want) <= 1e-12
