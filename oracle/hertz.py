"""Oracle: Hertz contact law, Eq. 30 (Section 5.4).

Test infrastructure only (see oracle/__init__.py).

  F_Hertz = 4 E / (3 (1 - nu^2)) * sqrt(R delta^3)
for a rigid sphere of radius R pressed a depth delta into an elastic half-space of
Young modulus E and Poisson ratio nu; valid for small delta / R.
"""
import math


def hertz_force(E, nu, R, delta):
    return 4.0 * E / (3.0 * (1.0 - nu * nu)) * math.sqrt(R * delta ** 3)


def lame_from_E_nu(E, nu):
    """(lambda, mu) of an isotropic material."""
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    mu = E / (2.0 * (1.0 + nu))
    return lam, mu
