"""Pins of oracle/hertz.py (Eq. 30) against the elastic half-space, not against the formula
itself.

Hertz's solution loads the surface of a half-space with the elliptical pressure
p(r) = p0 sqrt(1 - r^2 / a^2) on a disk of radius a = sqrt(R delta).  The force is the
integral of p, so p0 = 3 F / (2 pi a^2) for the force F that the oracle returns.  Under
any surface pressure, Boussinesq's point-load solution gives the normal surface
displacement u(x) = (1 - nu^2) / (pi E) * integral p(s) / |x - s| dA(s).  Feeding the
oracle's force through these two steps must reproduce the sphere's shape inside the
contact disk, u(r) = delta - r^2 / (2 R): a wrong constant (3/4 for 4/3), modulus
(1 - nu for 1 - nu^2) or exponent of delta moves u(0) away from delta.  The integral is
taken numerically, in polar coordinates centred at x, where the 1 / |x - s| singularity
cancels against the area element.
"""
import math

import pytest
from scipy import integrate

from oracle import hertz


def _surface_displacement(E, nu, a, p0, r):
    """u_z at distance r < a from the centre under p0 sqrt(1 - s^2 / a^2) on the disk."""
    def inner(theta):
        rho_max = -r * math.cos(theta) + math.sqrt(a * a - (r * math.sin(theta)) ** 2)

        def p_at(rho):
            sx, sy = r + rho * math.cos(theta), rho * math.sin(theta)
            return p0 * math.sqrt(max(0.0, 1.0 - (sx * sx + sy * sy) / (a * a)))

        return integrate.quad(p_at, 0.0, rho_max, epsabs=0.0, epsrel=1e-11, limit=200)[0]

    total = integrate.quad(inner, 0.0, 2.0 * math.pi, epsabs=0.0, epsrel=1e-10, limit=200)[0]
    return (1.0 - nu * nu) / (math.pi * E) * total


@pytest.mark.parametrize("E,nu,R,delta", [(1.0, 0.3, 64.0, 0.064), (210.0, 0.25, 96.0, 0.5), (3.0, 0.45, 10.0, 0.02)])
def test_hertz_force_reproduces_the_sphere_shape_through_boussinesq(E, nu, R, delta):
    F = hertz.hertz_force(E, nu, R, delta)
    a = math.sqrt(R * delta)
    p0 = 3.0 * F / (2.0 * math.pi * a * a)
    # the elliptical pressure integrates to F (shape normalisation, checked numerically)
    F_num = integrate.quad(lambda s: 2.0 * math.pi * s * p0 * math.sqrt(1.0 - (s / a) ** 2), 0.0, a,
                           epsabs=0.0, epsrel=1e-12)[0]
    assert abs(F_num - F) <= 1e-9 * F
    for frac in (0.0, 0.3, 0.6, 0.85):
        r = frac * a
        u = _surface_displacement(E, nu, a, p0, r)
        assert abs(u - (delta - r * r / (2.0 * R))) <= 1e-7 * delta, (frac, u, delta - r * r / (2.0 * R))


def test_hertz_force_scaling():
    """F grows like delta^(3/2) and R^(1/2), and is linear in the plane-strain modulus."""
    F = hertz.hertz_force(2.0, 0.3, 50.0, 0.1)
    assert hertz.hertz_force(2.0, 0.3, 50.0, 0.4) == pytest.approx(8.0 * F, rel=1e-14)
    assert hertz.hertz_force(2.0, 0.3, 200.0, 0.1) == pytest.approx(2.0 * F, rel=1e-14)
    assert hertz.hertz_force(6.0, 0.3, 50.0, 0.1) == pytest.approx(3.0 * F, rel=1e-14)


@pytest.mark.parametrize("E,nu", [(1.0, 0.3), (210.0, 0.0), (7.5, 0.49)])
def test_lame_parameters_give_back_young_and_poisson(E, nu):
    lam, mu = hertz.lame_from_E_nu(E, nu)
    # isotropic elasticity: E = mu (3 lam + 2 mu) / (lam + mu), nu = lam / (2 (lam + mu))
    assert mu * (3.0 * lam + 2.0 * mu) / (lam + mu) == pytest.approx(E, rel=1e-13)
    assert lam / (2.0 * (lam + mu)) == pytest.approx(nu, abs=1e-14)
    # uniaxial stress sigma_zz = 1: strain_zz = 1 / E, lateral strains -nu / E
    import numpy as np
    C = np.zeros((3, 3, 3, 3))
    for i in range(3):
        for j in range(3):
            C[i, i, j, j] += lam
            C[i, j, i, j] += mu
            C[i, j, j, i] += mu
    M = C.reshape(9, 9)
    sig = np.zeros((3, 3))
    sig[2, 2] = 1.0
    eps = np.linalg.lstsq(M, sig.ravel(), rcond=None)[0].reshape(3, 3)
    assert eps[2, 2] == pytest.approx(1.0 / E, rel=1e-12)
    assert eps[0, 0] == pytest.approx(-nu / E, abs=1e-12 / E)
