"""Closed forms the oracle is pinned against (TEST INFRASTRUCTURE ONLY).

Each function states the relation it evaluates and where the paper gives it.
"""
from __future__ import annotations

import math

from scipy.optimize import brentq

#: b^2 = v_S^2 = 1/3 on regular lattices (Sec. 2, after Eq. 12).
B2 = 1.0 / 3.0


def wave_speeds(lam: float, mu: float, rho0: float):
    """Eq. 4: v_P = sqrt((lambda + 2 mu)/rho0), v_S = sqrt(mu/rho0)."""
    return math.sqrt((lam + 2.0 * mu) / rho0), math.sqrt(mu / rho0)


def vp_over_vs(nu: float) -> float:
    """Eq. 5: v_P / v_S = sqrt((2 - 2 nu) / (1 - 2 nu))."""
    return math.sqrt((2.0 - 2.0 * nu) / (1.0 - 2.0 * nu))


def poisson_ratio(lam: float, mu: float) -> float:
    """Eq. 6: nu = lambda / (2 (lambda + mu))."""
    return lam / (2.0 * (lam + mu))


def lame_from_nu(nu: float, rho0: float = 1.0):
    """(lambda, mu) with mu/rho0 = b^2 (Sec. 4, after Eq. 31) and Eq. 6 solved
    for lambda: lambda = 2 mu nu / (1 - 2 nu)."""
    mu = rho0 * B2
    return 2.0 * mu * nu / (1.0 - 2.0 * nu), mu


def Lambda_of_nu(nu: float) -> float:
    """Eq. 32: Lambda = (mu - lambda)/(rho0 b^2) = (1 - 4 nu)/(1 - 2 nu)."""
    return (1.0 - 4.0 * nu) / (1.0 - 2.0 * nu)


def rayleigh_xi(nu: float) -> float:
    """xi = (v_R / v_S)^2: the root in (0, 1) of the Rayleigh equation
    (2 - xi)^2 = 4 sqrt(1 - xi) sqrt(1 - xi v_S^2 / v_P^2)
    (standard plane-strain elastodynamics; Sec. 7 quotes its nu = 0.25 root)."""
    r = 1.0 / vp_over_vs(nu) ** 2

    def g(xi):
        return (2.0 - xi) ** 2 - 4.0 * math.sqrt(1.0 - xi) * math.sqrt(1.0 - xi * r)

    return brentq(g, 1e-6, 1.0 - 1e-12, xtol=1e-15)


def ricker(t: float, f: float, t0: float) -> float:
    """Ricker wavelet (Sec. 5): (1 - 2 a) exp(-a), a = pi^2 f^2 (t - t0)^2."""
    a = (math.pi * f * (t - t0)) ** 2
    return (1.0 - 2.0 * a) * math.exp(-a)


def ricker_dt(t: float, f: float, t0: float) -> float:
    """Time derivative of :func:`ricker`."""
    c = (math.pi * f) ** 2
    s = t - t0
    a = c * s * s
    return (-4.0 * c * s - 2.0 * c * s * (1.0 - 2.0 * a)) * math.exp(-a)


def rayleigh_xi_scheme(nu: float) -> float:
    """xi = (v_R / v_S)^2 of the surface wave that the free-surface rule of
    Sec. 6.2 supports.

    That rule imposes P_air n = 0 at the wall (Eqs. 37-42: only the
    tangential stress of P_air is kept).  P is conserved by the collision
    (Eq. 22) and moves with the equilibrium third moment
    b^2 (j d + d j + j.d), so to leading order P = -2 mu eps(u) + b^2 rho I
    with rho = -rho0 div u and mu = rho0 b^2.  P n = 0 on a wall of normal
    n = e_y therefore reads mu div u + 2 mu d_y u_y = 0 and eps_xy = 0: the
    traction-free condition with lambda replaced by mu (identical for
    lambda = mu, nu = 0.25).  Rayleigh's ansatz (potentials decaying as
    exp(-q y), exp(-s y)) gives the determinant condition
    (2 - xi)(2 - 3 r xi) = 4 sqrt(1 - xi) sqrt(1 - r xi), r = v_S^2 / v_P^2;
    it reduces to :func:`rayleigh_xi`'s equation at r = 1/3."""
    r = 1.0 / vp_over_vs(nu) ** 2

    def g(xi):
        return (2.0 - xi) * (2.0 - 3.0 * r * xi) - 4.0 * math.sqrt(1.0 - xi) * math.sqrt(1.0 - xi * r)

    return brentq(g, 1e-6, 1.0 - 1e-12, xtol=1e-15)
