"""Pin of the oracle's Anderson rule (Section 4.1.1: depth 4, stored pairs cycling
through four slots, an acceleration after the first four iterations and then every
mod_ACV iterations) against a closed form that the mathematics fixes.

Take an affine map F(S) = M S + b with fixed point S*, M symmetric, and a start whose
error e_0 lies in the span of four orthonormal eigenvectors v_j of M (eigenvalues
mu_j != 1, e_0 = sum_j c_j v_j).  Before the first acceleration the iterates are plain,
so the stored pairs have errors e_k = M^k e_0 and residuals R_k = F(S_k) - S_k =
(M - I) M^k e_0.  Any combination sum_k alpha_k (S_k + R_k) with sum_k alpha_k = 1 is
S* + M q(M) e_m, where q(t) = sum_k alpha_k t^k and e_m is the error of the oldest stored
pair, and its residual is (M - I) q(M) e_m.  Minimising that residual over cubics with
q(1) = 1 is a weighted least-norm problem in the values z_j = q(mu_j): q(1) =
sum_j l_j(1) z_j with the Lagrange basis l_j on the nodes mu_j, the objective is
sum_j w_j z_j^2 with w_j = (c_j (mu_j - 1))^2, so z_j = (l_j(1) / w_j) / sum_k
(l_k(1)^2 / w_k).  The accelerated iterate is S* + sum_j c_j mu_j z_j v_j.  No Gram matrix
or linear solve enters this closed form.

A mistake in the stored pairs (a residual filed in the wrong slot), in the combination
(S_k without R_k) or in the constraint (no normalisation of alpha) moves the result away
from it; the last tests plant such mistakes in copies of the oracle's class and check
that the pin catches them.
"""
import numpy as np
import pytest

from oracle import solver as sv

MU = np.array([0.9, -0.6, 0.5, 0.2])        # eigenvalues carrying the start error
MU_REST = np.array([0.7, -0.3, 0.1])        # eigenvalues the error never touches
C = np.array([1.0, -0.7, 0.4, 2.0])


def _problem(seed=5):
    rng = np.random.default_rng(seed)
    n = len(MU) + len(MU_REST)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    M = Q @ np.diag(np.concatenate([MU, MU_REST])) @ Q.T
    s_star = rng.standard_normal(n)
    b = s_star - M @ s_star
    V = Q[:, :len(MU)]
    return M, b, s_star, V


def _closed_form(s_star, V, c):
    """S* + sum_j c_j mu_j z_j v_j with the weighted least-norm z (module docstring)."""
    m = len(MU)
    ell1 = np.array([np.prod([(1.0 - MU[k]) / (MU[j] - MU[k]) for k in range(m) if k != j]) for j in range(m)])
    w = (c * (MU - 1.0)) ** 2
    z = (ell1 / w) / np.sum(ell1 ** 2 / w)
    assert abs(np.dot(ell1, z) - 1.0) < 1e-12       # q(1) = 1
    return s_star + V @ (c * MU * z)


def _run(anderson, M, b, x0, i_last):
    """The oracle's calling pattern: x_0 is the start, x_i = F(S_(i-1)) for i >= 1 where
    S_(i-1) is what step(i-1, .) returned."""
    x = x0
    for i in range(i_last + 1):
        y = anderson.step(i, x)
        if i == i_last:
            return y
        x = M @ y + b


@pytest.mark.parametrize("mod", [2, 4])
def test_first_acceleration_matches_closed_form(mod):
    """mod 2 and 4: the first acceleration is at i = 4, over the pairs k = 0..3."""
    M, b, s_star, V = _problem()
    x0 = s_star + V @ C
    a = sv.Anderson(mod)
    y = _run(a, M, b, x0, 4)
    assert a.accelerated == 1
    want = _closed_form(s_star, V, C)
    assert np.abs(y - want).max() <= 1e-12 * np.abs(want).max()


def test_first_acceleration_mod3_uses_pairs_two_to_five():
    """mod 3: no acceleration at i = 4, 5; the first is at i = 6 over the pairs
    k = 2..5, whose oldest error is M^2 e_0, i.e. coefficients c_j mu_j^2."""
    M, b, s_star, V = _problem()
    a = sv.Anderson(3)
    y = _run(a, M, b, s_star + V @ C, 6)
    assert a.accelerated == 1
    want = _closed_form(s_star, V, C * MU ** 2)
    assert np.abs(y - want).max() <= 1e-12 * np.abs(want).max()


def test_no_acceleration_before_the_fourth_iteration():
    M, b, s_star, V = _problem()
    a = sv.Anderson(2)
    x0 = s_star + V @ C
    y = _run(a, M, b, x0, 3)
    assert a.accelerated == 0
    plain = s_star + np.linalg.matrix_power(M, 3) @ (x0 - s_star)
    assert np.abs(y - plain).max() < 1e-13


class _ResidualInWrongSlot(sv.Anderson):
    """Planted mistake: R_(i-1) filed in slot i mod 4 (the slot of S_i) instead of the
    slot of S_(i-1)."""

    def step(self, i, x):
        m = self.DEPTH
        if i > 0:
            self.R[i % m] = x - self.S[(i - 1) % m]
        if i >= m and i % self.mod == 0 and all(r is not None for r in self.R):
            G = np.array([[np.sum(self.R[k] * self.R[l]) for l in range(m)] for k in range(m)])
            y = sv.solve_small_spd(G, np.ones(m))
            if y is not None and np.sum(y) != 0.0:
                alpha = y / np.sum(y)
                x = sum(alpha[k] * (self.S[k] + self.R[k]) for k in range(m))
                self.accelerated += 1
        self.S[i % m] = x.copy()
        return x


class _CombinationWithoutResiduals(sv.Anderson):
    """Planted mistake: x <- sum alpha_k S_k."""

    def step(self, i, x):
        m = self.DEPTH
        if i > 0:
            self.R[(i - 1) % m] = x - self.S[(i - 1) % m]
        if i >= m and i % self.mod == 0:
            G = np.array([[np.sum(self.R[k] * self.R[l]) for l in range(m)] for k in range(m)])
            y = sv.solve_small_spd(G, np.ones(m))
            if y is not None and np.sum(y) != 0.0:
                alpha = y / np.sum(y)
                x = sum(alpha[k] * self.S[k] for k in range(m))
                self.accelerated += 1
        self.S[i % m] = x.copy()
        return x


class _UnnormalisedWeights(sv.Anderson):
    """Planted mistake: alpha = G^-1 1 without dividing by its sum."""

    def step(self, i, x):
        m = self.DEPTH
        if i > 0:
            self.R[(i - 1) % m] = x - self.S[(i - 1) % m]
        if i >= m and i % self.mod == 0:
            G = np.array([[np.sum(self.R[k] * self.R[l]) for l in range(m)] for k in range(m)])
            y = sv.solve_small_spd(G, np.ones(m))
            if y is not None:
                x = sum(y[k] * (self.S[k] + self.R[k]) for k in range(m))
                self.accelerated += 1
        self.S[i % m] = x.copy()
        return x


@pytest.mark.parametrize("cls", [_ResidualInWrongSlot, _CombinationWithoutResiduals, _UnnormalisedWeights])
def test_pin_catches_planted_mistakes(cls):
    M, b, s_star, V = _problem()
    a = cls(2)
    y = _run(a, M, b, s_star + V @ C, 4)
    want = _closed_form(s_star, V, C)
    assert np.abs(y - want).max() > 1e-3 * np.abs(want).max()
