"""Pins of the oracle operators: gradients, divergence, the Paux symbol (P2 eigenmodes),
the Green step and the Eq. 5 residual (Sections 3.1-3.2)."""

import numpy as np
import pytest

import workloads as wl
from oracle import discrete as dz, transforms as tr


def _pb(seed, scheme, nvox=(5, 4, 6), periodic_prob=0.25, nphase=2):
    rng = np.random.default_rng(seed)
    bc = wl.random_bc(rng, periodic_prob)
    ph = rng.integers(0, nphase, size=(nvox[2], nvox[1], nvox[0]))
    lam, mu = wl.lame(np.array([1.0, 2.5][:nphase]), 0.3)
    return dz.Problem(nvox, 1.0, bc, scheme, ph, lam, mu)


def _mode(pb, c, ks):
    basis = []
    for d in range(3):
        t = pb.types[c][d]
        j = np.arange(pb.nn[d])
        v = np.cos(ks[d] * j) if t in (tr.DCT1, tr.DCT3, tr.DFT) else np.sin(ks[d] * j)
        if t == tr.DCT3:
            v[pb.nvox[d]] = 0.0
        basis.append(v)
    return basis[2][:, None, None] * basis[1][None, :, None] * basis[0][None, None, :]


@pytest.mark.parametrize("scheme", [dz.TETRA2, dz.HEX1])
@pytest.mark.parametrize("seed", range(8))
def test_eigenmodes_of_reference_operator(scheme, seed):
    """P2: the real-space Paux operator (finite-element scatter divided by W) maps every
    separable DTT mode to a_c(q) times itself -- pins the S_j symbols, the selection
    sets and the W (symmetry-extension) convention together."""
    pb = _pb(seed, scheme)
    rng = np.random.default_rng(100 + seed)
    lam0, mu0 = 0.7, 0.3
    for c in range(3):
        for _ in range(4):
            ks = []
            for d in range(3):
                _, _, q = tr.selection(pb.types[c][d], pb.nvox[d])
                ks.append(q[rng.integers(len(q))])
            u = np.zeros((3,) + pb.node_shape)
            u[c] = _mode(pb, c, ks)
            out = dz.apply_A0(pb, u, lam0, mu0)
            S = dz.S_symbols(pb, np.array([ks[0]]), np.array([ks[1]]), np.array([ks[2]]))
            a_c = (lam0 * S[c] + 2 * mu0 * (S[0] + S[1] + S[2])).item()
            m = pb.dof_mask(c)
            assert np.abs(out[c][m] - a_c * u[c][m]).max() < 1e-12 * max(1.0, a_c)
            others = [x for x in range(3) if x != c]
            assert np.abs(out[others]).max() < 1e-13


@pytest.mark.parametrize("seed", range(6))
def test_green_inverts_reference_operator_tetra2(seed):
    """Away from null modes the Green step is the exact inverse of A0."""
    rng = np.random.default_rng(seed)
    while True:
        pb = _pb(seed, dz.TETRA2, nvox=(6, 5, 7))
        # no q = 0 / checkerboard null modes: every component has a Dirichlet face
        if all(any(tr.BC_D in pb.bc[d, :, c] for d in range(3)) for c in range(3)):
            break
        seed += 1000
    u = rng.standard_normal((3,) + pb.node_shape)
    for c in range(3):
        u[c][~pb.dof_mask(c)] = 0.0
    u2 = dz.green_apply(pb, dz.apply_A0(pb, u, 1.3, 0.6), 1.3, 0.6)
    assert np.abs(u2 - u).max() < 1e-12


def test_symbols_closed_form_values():
    """S_j at q = 0 and at the checkerboard (pi,pi,pi) vanish for both schemes; HEX1
    also vanishes whenever two wave numbers equal pi (hourglass), TETRA2 does not."""
    class P_:
        h = 1.0
    for scheme in (dz.TETRA2, dz.HEX1):
        P_.scheme = scheme
        z = np.array([0.0])
        p = np.array([np.pi])
        S = dz.S_symbols(P_, z, z, z)
        assert all(abs(s.item()) < 1e-15 for s in S)
        S = dz.S_symbols(P_, p, p, p)
        tot = (S[0] + S[1] + S[2]).item()
        assert abs(tot) < 1e-15                     # checkerboard: null for both
        S = dz.S_symbols(P_, np.array([0.3]), p, p)
        tot = (S[0] + S[1] + S[2]).item()
        assert (abs(tot) < 1e-15) == (scheme == dz.HEX1)
    # small-q limit: both schemes -> |q|^2 (continuum Laplacian) per component
    P_.scheme = dz.TETRA2
    q = np.array([1e-3])
    S = dz.S_symbols(P_, q, 2 * q, 3 * q)
    assert np.allclose([s.item() for s in S], [1e-6, 4e-6, 9e-6], rtol=1e-4)
    P_.scheme = dz.HEX1
    S = dz.S_symbols(P_, q, 2 * q, 3 * q)
    assert np.allclose([s.item() for s in S], [1e-6, 4e-6, 9e-6], rtol=1e-4)


@pytest.mark.parametrize("scheme", [dz.TETRA2, dz.HEX1])
def test_gradients_exact_for_affine_fields(scheme):
    """Both schemes reproduce the gradient of an affine displacement exactly, at every
    integration point (Section 3.1.1: HEX1 linear element, TETRA2 linear tetrahedra)."""
    bc = np.full((3, 2, 3), tr.BC_N)
    pb = dz.Problem((4, 3, 5), 0.5, bc, scheme, np.zeros((5, 3, 4)), [1.0], [1.0])
    Gm = np.array([[0.1, -0.2, 0.3], [0.05, 0.4, -0.1], [-0.3, 0.2, 0.15]])
    X = pb.node_positions()
    u = np.einsum("ab,bkji->akji", Gm, X) + 0.7
    g = dz.gradients(pb, u)
    for t in range(g.shape[0]):
        for c in range(3):
            for d in range(3):
                assert np.allclose(g[t, c, d], Gm[c, d], atol=1e-14)


def test_hex1_gradient_is_mean_of_tetra2():
    rng = np.random.default_rng(3)
    bc = np.full((3, 2, 3), tr.BC_N)
    ph = np.zeros((3, 4, 5))
    pt = dz.Problem((5, 4, 3), 1.0, bc, dz.TETRA2, ph, [1.0], [1.0])
    ph_ = dz.Problem((5, 4, 3), 1.0, bc, dz.HEX1, ph, [1.0], [1.0])
    u = rng.standard_normal((3,) + pt.node_shape)
    gt = dz.gradients(pt, u)
    gh = dz.gradients(ph_, u)
    assert np.abs(0.5 * (gt[0] + gt[1]) - gh[0]).max() < 1e-14


@pytest.mark.parametrize("scheme", [dz.TETRA2, dz.HEX1])
def test_divergence_is_energy_gradient(scheme):
    """p = -dE/du~ / (h^3 W): checked against a central finite difference of the energy
    E = sum w h^3 sigma:eps/2 (Eq. 18's quadratic form)."""
    rng = np.random.default_rng(11)
    pb = _pb(4, scheme, nvox=(3, 4, 3))
    pb.eps_star = np.array([[1e-3, 2e-4, 0], [2e-4, -5e-4, 1e-4], [0, 1e-4, 2e-4]])
    u = 1e-3 * rng.standard_normal((3,) + pb.node_shape)
    for c in range(3):
        u[c][~pb.dof_mask(c)] = 0.0
    w = np.array([ip[0] for ip in pb.ip_sets()])

    def energy(v):
        sig = dz.stress(pb, v)
        g = dz.gradients(pb, v)
        eps = 0.5 * (g + np.swapaxes(g, 1, 2)) + pb.eps_star[None, :, :, None, None, None]
        return 0.5 * pb.h ** 3 * np.sum(w[:, None, None, None, None, None] * sig * eps)

    p, _ = dz.residual(pb, u)
    for _ in range(12):
        c = int(rng.integers(3))
        idx = tuple(int(rng.integers(s)) for s in pb.node_shape)
        if not pb.dof_mask(c)[idx]:
            continue
        hstep = 1e-6
        up, um = u.copy(), u.copy()
        up[c][idx] += hstep
        um[c][idx] -= hstep
        dE = (energy(up) - energy(um)) / (2 * hstep)
        assert abs(-dE / (pb.h ** 3 * pb.weight_W(c)[idx]) - p[c][idx]) < 1e-7


def test_residual_norm_definition():
    """Eq. 5 with RMS norms on a hand-made field."""
    bc = np.full((3, 2, 3), tr.BC_N)
    pb = dz.Problem((2, 2, 2), 2.0, bc, dz.HEX1, np.zeros((2, 2, 2)), [1.0], [1.0])
    p = np.zeros((3,) + pb.node_shape)
    p[0, 0, 0, 0] = 3.0
    p[1, 1, 1, 1] = 4.0
    sig = np.zeros((1, 3, 3) + pb.vox_shape)
    sig[0, 0, 0] = 2.0
    r = dz.residual_norm(pb, p, sig)
    assert abs(r - 2.0 * np.sqrt(25.0 / 27.0) / 2.0) < 1e-15
