"""Oracle: Anderson convergence acceleration and the fixed-point solvers of
Algorithm 1 (local Dirichlet / linear constraints) and Algorithm 2 (frictionless
sphere contact, small strain); with kinematics="FS" the same loops are Algorithm 3 (and
its Algorithm 1 counterpart): Pi replaces sigma in the divergence, in the Eq. 5 norm and
in the contact reaction, nothing else changes (Section 5.2).

Test infrastructure only (see oracle/__init__.py).  Plain float64 numpy, the steps in
the paper's order.

Readings where the paper is silent (the same readings are implemented by the CUDA path):
  * Anderson (Section 4.1.1: depth 4, cycling indices, after the four first iterations
    and every mod_ACV iterations; the formula itself is only cited).  At local
    iteration i with current value x_i:
        if i > 0:                    R_{i-1} = x_i - S_{i-1}            (storeR)
        if i >= 4 and i % mod == 0:  alpha = argmin || sum_k alpha_k R_k ||_2,
                                     sum_k alpha_k = 1, over the 4 stored pairs,
                                     x_i <- sum_k alpha_k (S_k + R_k)    (accelerate)
        S_i = x_i                                                      (storeS)
    The constrained least squares is solved as G y = 1, alpha = y / sum(y), with
    G_kl = <R_k, R_l> (Euclidean, all nodal values) in float64 by Gaussian
    elimination with partial pivoting; if a pivot is <= 1e-14 * max_k G_kk or
    sum(y) is 0 the acceleration is skipped for that iteration.  The paper prints no
    accelerated iterate; the rule is pinned by a closed form instead: for an affine map
    whose start error lies in a four-dimensional invariant subspace, the first
    accelerated iterate is fixed by a weighted least-norm problem over the cubic
    residual polynomials (Lagrange form on the four eigenvalues, no Gram matrix).
  * Residual: Eq. 5 with RMS norms (discrete.residual_norm), evaluated on p after
    proj_P, as in Algorithm 1.  Algorithm 2 prints the test before
    proj_P; it is read in the same order, and the contact solve exits only when the
    residual is below tol AND both violation sets are empty.
  * Iterations: count of Green-operator steps performed; a run stops after max_iter
    of them whatever the residual.
"""
import numpy as np

from . import discrete as dz
from . import constraints as cs


def solve_small_spd(G, rhs, rel=1e-14):
    """Gaussian elimination with partial pivoting; returns None when a pivot is tiny."""
    n = len(rhs)
    A = np.array(G, dtype=np.float64).copy()
    b = np.array(rhs, dtype=np.float64).copy()
    scale = max(np.max(np.abs(np.diag(A))), 0.0)
    if scale == 0.0:
        return None
    for col in range(n):
        piv = col + int(np.argmax(np.abs(A[col:, col])))
        if abs(A[piv, col]) <= rel * scale:
            return None
        if piv != col:
            A[[col, piv]] = A[[piv, col]]
            b[[col, piv]] = b[[piv, col]]
        for r in range(col + 1, n):
            m = A[r, col] / A[col, col]
            A[r, col:] -= m * A[col, col:]
            b[r] -= m * b[col]
    y = np.zeros(n)
    for r in range(n - 1, -1, -1):
        y[r] = (b[r] - np.dot(A[r, r + 1:], y[r + 1:])) / A[r, r]
    return y


class Anderson:
    DEPTH = 4

    def __init__(self, mod):
        self.mod = int(mod)
        self.S = [None] * self.DEPTH
        self.R = [None] * self.DEPTH
        self.accelerated = 0

    def step(self, i, x):
        m = self.DEPTH
        if i > 0:
            self.R[(i - 1) % m] = x - self.S[(i - 1) % m]
        if i >= m and i % self.mod == 0:
            G = np.array([[np.sum(self.R[k] * self.R[l]) for l in range(m)] for k in range(m)])
            y = solve_small_spd(G, np.ones(m))
            if y is not None and np.sum(y) != 0.0:
                alpha = y / np.sum(y)
                x = sum(alpha[k] * (self.S[k] + self.R[k]) for k in range(m))
                self.accelerated += 1
        self.S[i % m] = x.copy()
        return x


class Result:
    pass


def solve_alg1(pb, rows, lam0, mu0, tol, max_iter, acv_on="P", acv_mod=3, u0=None,
               acv=True, kinematics="SS", medium="paux"):
    """Algorithm 1 (Section 4.1.1).  Returns a Result with u, p, sigma, multipliers,
    iterations, residual history.  medium "iso": the isotropic reference medium of Section
    3.2.3 (A0 by discrete.apply_A0_iso, the Green step by discrete.green_apply_dense; small
    grids with normal mixed conditions)."""
    if medium == "iso":
        a0 = lambda u: dz.apply_A0_iso(pb, u, lam0, mu0)          # noqa: E731
        green = dz.make_dense_green(pb, a0)
    else:
        a0 = lambda u: dz.apply_A0(pb, u, lam0, mu0)              # noqa: E731
        green = lambda p: dz.green_apply(pb, p, lam0, mu0)        # noqa: E731
    cs.check_rows(pb, rows)
    tgt = cs.targets(pb, rows)
    u = np.zeros((3,) + pb.node_shape) if u0 is None else np.array(u0, dtype=np.float64)
    for c in range(3):
        u[c][~pb.dof_mask(c)] = 0.0
    cs.proj_U(pb, u, rows, tgt)
    ander = Anderson(acv_mod)
    hist = []
    i = 0
    it = 0
    while True:
        if acv and acv_on == "U":
            u = ander.step(i, u)
        p, sig = dz.residual(pb, u, kinematics)
        f = cs.proj_P(pb, p, rows)
        r = dz.residual_norm(pb, p, sig)
        hist.append(r)
        if r < tol or it >= max_iter:
            break
        pt = p + a0(u)
        if acv and acv_on == "P":
            pt = ander.step(i, pt)
        u = green(pt)
        cs.proj_U(pb, u, rows, tgt)
        i += 1
        it += 1
    res = Result()
    res.u, res.p, res.sigma, res.f = u, p, sig, f
    res.iterations, res.residual, res.history = it, hist[-1], hist
    res.converged = hist[-1] < tol
    res.accelerations = ander.accelerated
    res.reactions, res.total_reaction = cs.row_reactions(pb, rows, f)
    return res


def solve_alg2_increment(pb, ind, rows, lam0, mu0, tol, max_iter, u_prev, acv_on="P",
                         acv_mod=3, update_tol=1e-2, kinematics="SS"):
    """One load increment of Algorithm 2 (Section 5.1.3); ind.center is the moved
    sphere centre O'_s.  u_prev is u~ at the end of the previous increment."""
    cs.check_rows(pb, rows)
    tgt = cs.targets(pb, rows)
    u = np.array(u_prev, dtype=np.float64)
    g, _ = cs.contact_geometry(pb, ind, u)
    active = g < 0.0
    cs.proj_U(pb, u, rows, tgt)
    cs.contact_proj_U(pb, ind, u, active)
    ander = Anderson(acv_mod)
    hist = []
    prev_sets = None
    updates = 0
    i = 0
    it = 0
    while True:
        if acv_on == "U":
            u = ander.step(i, u)
        p, sig = dz.residual(pb, u, kinematics)
        f_rows = cs.proj_P(pb, p, rows)
        g, _ = cs.contact_geometry(pb, ind, u)
        fn, _ = cs.contact_proj_P(pb, ind, u, p, active)
        v_gap = (~active) & (g < 0.0)
        v_react = active & (fn > 0.0)
        r = dz.residual_norm(pb, p, sig)
        hist.append(r)
        if (r < tol and not v_gap.any() and not v_react.any()) or it >= max_iter:
            break
        sets = (v_gap.tobytes(), v_react.tobytes())
        if prev_sets is not None and sets == prev_sets and r < update_tol:
            old = active.copy()
            active = (active | v_gap) & ~v_react
            if not np.array_equal(active, old):
                i = 0
                updates += 1
        prev_sets = sets
        pt = p + dz.apply_A0(pb, u, lam0, mu0)
        if acv_on == "P":
            pt = ander.step(i, pt)
        u = dz.green_apply(pb, pt, lam0, mu0)
        cs.proj_U(pb, u, rows, tgt)
        cs.contact_proj_U(pb, ind, u, active)
        i += 1
        it += 1
    res = Result()
    res.u, res.p, res.sigma = u, p, sig
    res.active, res.gap, res.fn = active, g, fn
    res.iterations, res.residual, res.history = it, hist[-1], hist
    res.converged = r < tol and not v_gap.any() and not v_react.any()
    res.updates = updates
    _, n = cs.contact_geometry(pb, ind, u)
    res.force = np.sum(np.where(active, fn, 0.0)[None, :] * n, axis=1)
    res.f_rows = f_rows
    return res


def mean_stress(pb, sig):
    """Volume average of sigma (or Pi) over the cell: sum_vox sum_t w_t sigma / N_vox
    (Section 5.4 takes the reaction force from it)."""
    w = np.array([ip[0] for ip in pb.ip_sets()])
    return np.einsum("t,tabzyx->ab", w, sig) / float(np.prod(pb.vox_shape))
