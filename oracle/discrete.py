"""Oracle: the discrete mechanical problem -- grid, boundary conditions, HEX1/TETRA2
gradients, stress, nodal divergence, the Paux reference operator and its symbol.

Test infrastructure only (see oracle/__init__.py).  Plain float64 numpy.

Paper passages followed:
  * Section 2 (notations): nodes at integer positions, voxel centres at half
    positions; node (i, j, k) sits at h*(i, j, k).
  * Section 3.1.1 and Fig. 1: HEX1 = one integration point per voxel (linear hexahedron,
    reduced integration); TETRA2 = two integration points, one per tetrahedron T1, T2
    inscribed in the voxel.  The strain of a TETRA2 point is the exact gradient of the
    linear interpolant on its tetrahedron.  With corner offsets delta in {0,1}^3 and
    s_d(delta) = +1 if delta_d = 1 else -1:
        TETRA2: T1 = corners with even delta_x+delta_y+delta_z, T2 = odd ones,
                grad_d u = (1/(2h)) sum_{delta in T} s_d u(delta), weight 1/2 each;
        HEX1:   grad_d u = (1/(4h)) sum_{all 8} s_d u(delta), weight 1.
  * Eq. 3: sigma = C : (eps* + sym grad_D u~), p = div_D(sigma - R0 : grad_D u~).
    Finite strain (Section 5.2, Eq. 29): sigma is replaced by the first Piola-Kirchhoff
    stress Pi (function piola); the reference term is unchanged.
    div_D is the discrete divergence at nodes, the negative adjoint of grad_D; it is
    computed here as  p = -F / (h^3 W)  with F = dE/du~ the finite-element nodal force of
    the real cell and W the symmetry weight below.
  * Table 1: the symmetry extensions.  At a node lying on k Neumann faces of
    component c, the divergence of the symmetry-extended stress equals 2^k times the
    one-sided (finite-element) divergence -- the paper's own "divide by 2 on faces, by
    4 at corners" rule of Section 4.1.3.  So W_c(node) = 2^-k.  Dirichlet-face nodes of
    component c carry no unknown (u~_c = 0 there) and p_c = 0.
  * Section 3.2.3: Paux reference medium  R0 : grad u = lambda0 (grad u (.) I)
    + 2 mu0 grad u  (Hadamard product), which decouples the components.  Its discrete
    symbol for component c is  a_c(q) = lambda0 S_c(q) + 2 mu0 sum_j S_j(q), with
    (c_j = cos q_j, {j,k,l} a permutation of the axes)
        TETRA2: S_j = (1 + c_k c_l - c_j c_k - c_j c_l) / h^2
        HEX1:   S_j = (1 - c_j)(1 + c_k)(1 + c_l) / (2 h^2)
    (S_j = sum over integration points of w |symbol of grad_j|^2, derived here because
    the paper gives these operators by reference only).  Points where a_c vanishes
    (q = 0, and q = (pi,pi,pi) for TETRA2 / two components equal to pi for HEX1) are
    null modes; the Green step sets them to zero.
"""
import itertools
import numpy as np

from .transforms import (BC_P, BC_D, BC_N, DFT, transform_type, node_count,
                         forward_3d, inverse_3d, wave_numbers)

TETRA2, HEX1 = 0, 1


class Problem:
    """A voxel cell: sizes, spacing, per-face per-component BCs, scheme, material.

    nvox  = (nx, ny, nz) voxels; h = voxel size
    bc    = int array [axis][face][component], codes 0 P, 1 D, 2 N
    phase = uint8 voxel array of shape (nz, ny, nx) (x fastest)
    lam, mu = per-phase Lame coefficients
    eps_star = 3x3 symmetric prescribed strain (affine lift u* = eps* . x)
    Node arrays have shape (nnz, nny, nnx): nn_d = n_d for a periodic axis else n_d+1.
    """

    def __init__(self, nvox, h, bc, scheme, phase, lam, mu, eps_star=None):
        self.nvox = tuple(int(v) for v in nvox)
        self.h = float(h)
        self.bc = np.asarray(bc, dtype=np.int64).reshape(3, 2, 3)
        self.scheme = int(scheme)
        self.phase = np.asarray(phase, dtype=np.uint8).reshape(self.nvox[2], self.nvox[1], self.nvox[0])
        self.lam = np.asarray(lam, dtype=np.float64)
        self.mu = np.asarray(mu, dtype=np.float64)
        self.eps_star = np.zeros((3, 3)) if eps_star is None else np.asarray(eps_star, dtype=np.float64)
        self.types = [tuple(transform_type(self.bc[d, 0, c], self.bc[d, 1, c]) for d in range(3))
                      for c in range(3)]
        self.periodic = []
        for d in range(3):
            per = [self.types[c][d] == DFT for c in range(3)]
            if any(per) and not all(per):
                raise ValueError("an axis is periodic for all components or for none")
            self.periodic.append(per[0])
        self.nn = tuple(node_count(self.types[0][d], self.nvox[d]) for d in range(3))
        self.node_shape = (self.nn[2], self.nn[1], self.nn[0])
        self.vox_shape = (self.nvox[2], self.nvox[1], self.nvox[0])

    # ---- boundary structure ------------------------------------------------
    def _face_masks(self, d):
        """Boolean node masks of face 0 and face 1 of axis d (empty if periodic)."""
        shape = self.node_shape
        ax = 2 - d
        m0 = np.zeros(shape, dtype=bool)
        m1 = np.zeros(shape, dtype=bool)
        if self.periodic[d]:
            return m0, m1
        sl0 = [slice(None)] * 3
        sl1 = [slice(None)] * 3
        sl0[ax] = 0
        sl1[ax] = self.nn[d] - 1
        m0[tuple(sl0)] = True
        m1[tuple(sl1)] = True
        return m0, m1

    def dof_mask(self, c):
        """True where component c is an unknown (not on a Dirichlet face of c)."""
        m = np.ones(self.node_shape, dtype=bool)
        for d in range(3):
            f0, f1 = self._face_masks(d)
            if self.bc[d, 0, c] == BC_D:
                m &= ~f0
            if self.bc[d, 1, c] == BC_D:
                m &= ~f1
        return m

    def weight_W(self, c):
        """W_c = 2^-k, k = number of Neumann faces (of component c) the node lies on."""
        W = np.ones(self.node_shape)
        for d in range(3):
            f0, f1 = self._face_masks(d)
            if self.bc[d, 0, c] == BC_N:
                W[f0] *= 0.5
            if self.bc[d, 1, c] == BC_N:
                W[f1] *= 0.5
        return W

    def node_positions(self):
        """(3, nnz, nny, nnx) reference positions h*(i, j, k) of the nodes."""
        k, j, i = np.meshgrid(np.arange(self.nn[2]), np.arange(self.nn[1]), np.arange(self.nn[0]),
                              indexing="ij")
        return self.h * np.stack([i, j, k]).astype(np.float64)

    def lift(self):
        """Affine lift u*_a = sum_b eps*_ab x_b at the nodes, shape (3, nodes)."""
        X = self.node_positions()
        return np.einsum("ab,bkji->akji", self.eps_star, X)

    # ---- element geometry ----------------------------------------------------
    def ip_sets(self):
        """List of (weight, corner list, gradient coefficient) per integration point."""
        corners = list(itertools.product((0, 1), repeat=3))   # (dx, dy, dz)
        if self.scheme == TETRA2:
            even = [c for c in corners if sum(c) % 2 == 0]
            odd = [c for c in corners if sum(c) % 2 == 1]
            return [(0.5, even, 1.0 / (2.0 * self.h)), (0.5, odd, 1.0 / (2.0 * self.h))]
        if self.scheme == HEX1:
            return [(1.0, corners, 1.0 / (4.0 * self.h))]
        raise ValueError("scheme")

    def corner_ix(self, delta):
        """np.ix_ index selecting, for every voxel, its corner node at offset delta."""
        idx = []
        for d in range(3):
            n = self.nvox[d]
            idx.append((np.arange(n) + delta[d]) % self.nn[d])
        return np.ix_(idx[2], idx[1], idx[0])

    def material(self):
        return self.lam[self.phase], self.mu[self.phase]


def gradients(pb, u):
    """Displacement gradients at the integration points.

    u: (3, nodes).  Returns g of shape (n_ip, 3 [component c], 3 [direction d], voxels)
    with g[t, c, d] = d u_c / d x_d at point t.
    """
    ips = pb.ip_sets()
    g = np.zeros((len(ips), 3, 3) + pb.vox_shape)
    for t, (_, corners, coef) in enumerate(ips):
        for delta in corners:
            ix = pb.corner_ix(delta)
            for c in range(3):
                uc = u[c][ix]
                for d in range(3):
                    s = 1.0 if delta[d] == 1 else -1.0
                    g[t, c, d] += coef * s * uc
    return g


def stress(pb, u):
    """sigma = lambda tr(eps) I + 2 mu eps,  eps = eps* + sym(grad u): (n_ip, 3, 3, voxels)."""
    g = gradients(pb, u)
    lam, mu = pb.material()
    eps = 0.5 * (g + np.swapaxes(g, 1, 2)) + pb.eps_star[None, :, :, None, None, None]
    tr = eps[:, 0, 0] + eps[:, 1, 1] + eps[:, 2, 2]
    sig = 2.0 * mu * eps
    for a in range(3):
        sig[:, a, a] += lam * tr
    return sig


def piola(pb, u):
    """First Piola-Kirchhoff stress at the integration points (finite strain, Section 5.2).

    Eq. 29 replaces sigma by Pi = F(F~) with F~ = 1 + grad_D u; the behaviour used is the
    example given right after Eq. 29 (and in Section 5.4): S = C : E with the per-phase
    isotropic C, E = (F^T F - 1) / 2 the Green-Lagrange strain, Pi = F . S.  The prescribed
    load eps* enters as an imposed displacement gradient (u* = eps* . x, as in small strain),
    so F = 1 + eps* + grad u~.  Returns Pi[t, c, d] (n_ip, 3, 3, voxels); Pi[t, c, d] is
    the derivative of the strain energy density with respect to grad_d u_c, so it pairs
    with grad u in nodal_force exactly as sigma does.
    """
    g = gradients(pb, u)
    F = g + pb.eps_star[None, :, :, None, None, None]
    for a in range(3):
        F[:, a, a] += 1.0
    E = 0.5 * np.einsum("tkazyx,tkbzyx->tabzyx", F, F)
    for a in range(3):
        E[:, a, a] -= 0.5
    lam, mu = pb.material()
    tr = E[:, 0, 0] + E[:, 1, 1] + E[:, 2, 2]
    S = 2.0 * mu * E
    for a in range(3):
        S[:, a, a] += lam * tr
    return np.einsum("tckzyx,tkdzyx->tcdzyx", F, S)


def nodal_force(pb, tau):
    """F_c(node) = sum_voxels sum_t w_t h^3 sum_d tau[t, c, d] * d(grad_d u_c)/d u_c(node).

    tau: (n_ip, 3, 3, voxels) -- the stress-like tensor paired with grad u.
    """
    F = np.zeros((3,) + pb.node_shape)
    h3 = pb.h ** 3
    for t, (w, corners, coef) in enumerate(pb.ip_sets()):
        for delta in corners:
            ix = pb.corner_ix(delta)
            for c in range(3):
                acc = np.zeros(pb.vox_shape)
                for d in range(3):
                    s = 1.0 if delta[d] == 1 else -1.0
                    acc += tau[t, c, d] * (coef * s)
                F[c][ix] += w * h3 * acc
    return F


def div_from_force(pb, F):
    """Extension-form divergence p_c = -F_c / (h^3 W_c) on unknowns, 0 elsewhere."""
    p = np.zeros_like(F)
    for c in range(3):
        m = pb.dof_mask(c)
        p[c][m] = -F[c][m] / (pb.h ** 3 * pb.weight_W(c)[m])
    return p


def residual(pb, u, kinematics="SS"):
    """Eq. 3 first two lines: (p, sigma) for the current fluctuation u (3, nodes).
    kinematics "FS": Eq. 29, the stress and divergence steps of Algorithm 3: p = div_D(Pi), returned with Pi."""
    sig = piola(pb, u) if kinematics == "FS" else stress(pb, u)
    return div_from_force(pb, nodal_force(pb, sig)), sig


def apply_A0(pb, u, lam0, mu0):
    """A0 u = -div_D(R0 : grad_D u) with the Paux R0 (Section 3.2.3), extension form."""
    g = gradients(pb, u)
    tau = np.zeros_like(g)
    for c in range(3):
        for d in range(3):
            tau[:, c, d] = (2.0 * mu0 + (lam0 if c == d else 0.0)) * g[:, c, d]
    F = nodal_force(pb, tau)
    out = np.zeros_like(F)
    for c in range(3):
        m = pb.dof_mask(c)
        out[c][m] = F[c][m] / (pb.h ** 3 * pb.weight_W(c)[m])
    return out


def is_normal_mixed(pb):
    """True when every axis is periodic for all components or has "normal mixed"
    conditions on both faces: the normal component's condition differs from both tangential
    components' (normal Dirichlet with tangential Neumann, or the reverse).  Section 3.2.3:
    the isotropic reference medium is usable with the per-component transforms for
    periodic and normal mixed conditions."""
    for d in range(3):
        if pb.periodic[d]:
            continue
        for f in range(2):
            normal = pb.bc[d, f, d]
            for c in range(3):
                if c != d and pb.bc[d, f, c] == normal:
                    return False
    return True


def apply_A0_iso(pb, u, lam0, mu0):
    """A0 u = -div_D(R0 : grad_D u) for the isotropic reference medium of Section 3.2.3,
    R0 : grad u = lambda0 tr(grad u) 1 + mu0 (grad u + grad u^T), extension form.  Unlike
    the Paux medium it couples the components (through lambda0 div u and mu0 grad u^T)."""
    g = gradients(pb, u)
    tr = g[:, 0, 0] + g[:, 1, 1] + g[:, 2, 2]
    tau = mu0 * (g + np.swapaxes(g, 1, 2))
    for a in range(3):
        tau[:, a, a] += lam0 * tr
    F = nodal_force(pb, tau)
    out = np.zeros_like(F)
    for c in range(3):
        m = pb.dof_mask(c)
        out[c][m] = F[c][m] / (pb.h ** 3 * pb.weight_W(c)[m])
    return out


def make_dense_green(pb, apply_op, rcond=1e-10):
    """The Green step by its definition, for small grids: returns p~ -> u~ = A0^-1 p~ on
    the unknowns, where A0 = apply_op (a linear map of nodal fields), with the part of p~
    along the null space of A0 discarded and u~ orthogonal to it, both in the W-weighted
    inner product <a, b> = sum a b W.  A0 is symmetric in that inner product, and the DTT
    bases are orthogonal in it, so this is the spectral Green step with null modes set to
    zero (a pin compares the two for the Paux medium).  Dense matrix of the map, symmetric
    eigen-decomposition in float64, built once."""
    masks = [pb.dof_mask(c) for c in range(3)]
    sizes = [int(m.sum()) for m in masks]
    n = sum(sizes)
    off = np.cumsum([0] + sizes)

    def gather(f):
        return np.concatenate([f[c][masks[c]] for c in range(3)])

    def scatter(v):
        f = np.zeros((3,) + pb.node_shape)
        for c in range(3):
            f[c][masks[c]] = v[off[c]:off[c + 1]]
        return f

    A = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        A[:, j] = gather(apply_op(scatter(e)))
    w = gather(np.stack([pb.weight_W(c) for c in range(3)]))
    sw = np.sqrt(w)
    B = sw[:, None] * A / sw[None, :]
    B = 0.5 * (B + B.T)
    lam, V = np.linalg.eigh(B)
    keep = lam > rcond * np.max(np.abs(lam))
    Vk, lk = V[:, keep], lam[keep]

    def green(ptilde):
        y = Vk @ ((Vk.T @ (sw * gather(ptilde))) / lk)
        return scatter(y / sw)
    return green


def green_apply_dense(pb, ptilde, apply_op, rcond=1e-10):
    """One application of make_dense_green(pb, apply_op)."""
    return make_dense_green(pb, apply_op, rcond)(ptilde)


def S_symbols(pb, qx, qy, qz):
    """(S_x, S_y, S_z) on the broadcast grid of wave numbers (z, y, x array order)."""
    cx = np.cos(qx)[None, None, :]
    cy = np.cos(qy)[None, :, None]
    cz = np.cos(qz)[:, None, None]
    h2 = pb.h ** 2
    if pb.scheme == TETRA2:
        Sx = (1.0 + cy * cz - cx * cy - cx * cz) / h2
        Sy = (1.0 + cx * cz - cy * cx - cy * cz) / h2
        Sz = (1.0 + cx * cy - cz * cx - cz * cy) / h2
    else:
        Sx = (1.0 - cx) * (1.0 + cy) * (1.0 + cz) / (2.0 * h2)
        Sy = (1.0 - cy) * (1.0 + cx) * (1.0 + cz) / (2.0 * h2)
        Sz = (1.0 - cz) * (1.0 + cx) * (1.0 + cy) / (2.0 * h2)
    return Sx, Sy, Sz


NULL_REL = 1e-12


def green_symbol(pb, c, lam0, mu0):
    """a_c(q) = lambda0 S_c + 2 mu0 (S_x + S_y + S_z) on component c's spectral grid."""
    qx, qy, qz = wave_numbers(pb.types[c], pb.nvox)
    S = S_symbols(pb, qx, qy, qz)
    return lam0 * S[c] + 2.0 * mu0 * (S[0] + S[1] + S[2])


def green_apply(pb, ptilde, lam0, mu0):
    """Green step of Algorithm 1 (DT, Green operator, iDT): u~ = iDT( DT(p~) / a ), null modes set to 0."""
    out = np.zeros_like(ptilde)
    for c in range(3):
        a = green_symbol(pb, c, lam0, mu0)
        X = forward_3d(ptilde[c], pb.types[c], pb.nvox)
        a = np.broadcast_to(a, X.shape)
        null = a <= NULL_REL * np.max(a)
        Y = np.where(null, 0.0, X / np.where(null, 1.0, a))
        out[c] = inverse_3d(Y, pb.types[c], pb.nvox)
    return out


def residual_norm(pb, p, sig):
    """Eq. 5 with RMS norms: r = h ||p||_rms / ||sigma||_rms (||Pi||_rms in finite strain:
    the stress that p is the divergence of).

    ||p||_rms^2 = sum_nodes sum_c p_c^2 / N_nodes;
    ||sigma||_rms^2 = sum_voxels sum_t w_t sum_ab sigma_ab^2 / N_voxels.
    """
    n_nodes = float(np.prod(pb.node_shape))
    n_vox = float(np.prod(pb.vox_shape))
    pn = np.sqrt(np.sum(p * p) / n_nodes)
    w = np.array([ip[0] for ip in pb.ip_sets()])
    sn = np.sqrt(np.sum(w[:, None, None, None, None, None] * sig * sig) / n_vox)
    if sn == 0.0:
        return 0.0 if pn == 0.0 else np.inf
    return pb.h * pn / sn


def problem_from(spec):
    """Build a Problem from a mapping with keys nvox, h, bc, scheme, phase, lam, mu,
    eps_star (the layout the seeded input generators produce)."""
    return Problem(spec["nvox"], spec["h"], spec["bc"], spec["scheme"], spec["phase"],
                   spec["lam"], spec["mu"], spec.get("eps_star"))


def has_null_modes(pb, c):
    """True if the Green symbol of component c vanishes somewhere on its spectral grid
    (q = 0 on all axes, the TETRA2 checkerboard q = (pi,pi,pi), or a HEX1 hourglass
    with two wave numbers equal to pi).  The Green step sets those coefficients to
    zero, so a component with null modes cannot carry constraint rows: the fixed point
    would require the constrained solution to have zero null-mode content.  The paper
    meets this in Section 4.1.2 and removes it with a void buffer layer carrying a
    Dirichlet face."""
    has0, haspi = [], []
    for d in range(3):
        t = pb.types[c][d]
        n = pb.nvox[d]
        has0.append(t in ("DCT1", "DFT"))
        haspi.append(t == "DCT1" or (t == "DFT" and n % 2 == 0))
    if all(has0):
        return True
    if pb.scheme == TETRA2:
        return all(haspi)
    return sum(haspi) >= 2
