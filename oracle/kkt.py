"""Oracle: the plain definition of the discrete problem -- element-by-element
assembly of the stiffness matrix and a dense solve of the Lagrange-multiplier system.

Test infrastructure only (see oracle/__init__.py).  Only for tiny grids (<= 6^3 voxels).

Paper passages followed:
  * Section 4.3, Eq. 18-23: the converged iterate of Algorithm 1 is the saddle point of
    the constrained energy, i.e. the solution of
        [ K   -h^3 W B ] [ u~ ]   [ -F* ]
        [ A       0    ] [ f  ] = [  t  ]
    K = sum over voxels and integration points of w h^3 G^T C G (G = the 9x24
    displacement-gradient matrix of Section 3.1.1 / Fig. 1), restricted to the unknowns
    (nodes not on a Dirichlet face of their component); F* = the nodal force of the
    prescribed strain eps* at u~ = 0; A, B, t = the constraint rows (Eq. 21-23) and their
    targets on u~.  The factor h^3 W converts the extension-form multiplier of the
    projections into a finite-element nodal force (face nodes halved, edges quartered,
    Section 4.1.3); for rows whose support avoids Neumann faces W = 1 and this is
    exactly Eq. 20 / Eq. 23 up to the sign convention of f.
This module assembles K from an explicit per-element loop, independently of the
vectorised operators in discrete.py.
"""
import itertools
import numpy as np


def element_G(pb, t):
    """9x24 matrix: rows (c, d) -> d u_c/d x_d at point t; columns (corner, component)."""
    ips = pb.ip_sets()
    _, corners, coef = ips[t]
    allc = list(itertools.product((0, 1), repeat=3))
    G = np.zeros((9, 24))
    for ci, delta in enumerate(allc):
        if delta not in corners:
            continue
        for c in range(3):
            for d in range(3):
                s = 1.0 if delta[d] == 1 else -1.0
                G[3 * c + d, 3 * ci + c] = coef * s
    return G, allc


def iso_C(lam, mu):
    """9x9 isotropic stiffness acting on the full displacement gradient."""
    C = np.zeros((9, 9))
    for a in range(3):
        for b in range(3):
            for c in range(3):
                for d in range(3):
                    v = lam * (a == b) * (c == d) + mu * ((a == c) * (b == d) + (a == d) * (b == c))
                    C[3 * a + b, 3 * c + d] = v
    return C


def assemble(pb):
    """Full K over all (node, component) pairs and the eps* force vector F*."""
    nn = int(np.prod(pb.node_shape))
    K = np.zeros((3 * nn, 3 * nn))
    Fs = np.zeros(3 * nn)
    h3 = pb.h ** 3
    nx, ny, nz = pb.nvox
    eps = pb.eps_star.reshape(9)
    for t, (w, _, _) in enumerate(pb.ip_sets()):
        G, allc = element_G(pb, t)
        for vz in range(nz):
            for vy in range(ny):
                for vx in range(nx):
                    ph = pb.phase[vz, vy, vx]
                    C = iso_C(pb.lam[ph], pb.mu[ph])
                    ke = w * h3 * G.T @ C @ G
                    fe = w * h3 * G.T @ (C @ eps)
                    dofs = []
                    for (dx, dy, dz) in allc:
                        i = (vx + dx) % pb.nn[0]
                        j = (vy + dy) % pb.nn[1]
                        k = (vz + dz) % pb.nn[2]
                        node = i + pb.nn[0] * (j + pb.nn[1] * k)
                        for c in range(3):
                            dofs.append(c * nn + node)
                    dofs = np.array(dofs)
                    K[np.ix_(dofs, dofs)] += ke
                    Fs[dofs] += fe
    return K, Fs


def solve_kkt(pb, rows, tgt):
    """Dense solve of the multiplier system; returns (u~ (3, nodes), f per row)."""
    nn = int(np.prod(pb.node_shape))
    K, Fs = assemble(pb)
    free = np.concatenate([np.flatnonzero(pb.dof_mask(c).ravel()) + c * nn for c in range(3)])
    pos = -np.ones(3 * nn, dtype=np.int64)
    pos[free] = np.arange(len(free))
    Wfull = np.concatenate([pb.weight_W(c).ravel() for c in range(3)])
    n, m = len(free), len(rows)
    M = np.zeros((n + m, n + m))
    rhs = np.zeros(n + m)
    M[:n, :n] = K[np.ix_(free, free)]
    rhs[:n] = -Fs[free]
    h3 = pb.h ** 3
    for r, row in enumerate(rows):
        for node, c, a, b in zip(row.nodes, row.comps, row.a, row.b):
            g = c * nn + node
            M[pos[g], n + r] -= h3 * Wfull[g] * b
            M[n + r, pos[g]] += a
        rhs[n + r] = tgt[r]
    sol = np.linalg.solve(M, rhs)
    u = np.zeros(3 * nn)
    u[free] = sol[:n]
    return u.reshape((3,) + pb.node_shape), sol[n:]
