"""Pins of the oracle's lattice, equilibrium, forcing and source routines
against identities the paper states (no GPU)."""
import itertools
import math

import numpy as np
import pytest

import oracle
from oracle import theory


def _delta(a, b):
    return 1.0 if a == b else 0.0


def test_lattice_isotropy_exact(golden):
    """Eq. 27: the D2Q9 moment identities up to sixth order, and b^2 = 1/3
    (Sec. 2).  A wrong weight or velocity fails one of these."""
    cx, cy, w, b2 = oracle.lattice()
    assert b2 == pytest.approx(golden["lattice"]["b2"], abs=1e-16)
    c = np.stack([cx, cy], 1).astype(float)
    assert np.sum(w) == pytest.approx(1.0, abs=1e-15)
    for a in range(2):
        assert np.sum(w * c[:, a]) == pytest.approx(0.0, abs=1e-16)
        for b in range(2):
            assert np.sum(w * c[:, a] * c[:, b]) == pytest.approx(b2 * _delta(a, b), abs=1e-15)

    def d4(a, b, g, k):
        return _delta(a, b) * _delta(g, k) + _delta(a, g) * _delta(b, k) + _delta(a, k) * _delta(b, g)

    for a, b, g, k in itertools.product(range(2), repeat=4):
        s = np.sum(w * c[:, a] * c[:, b] * c[:, g] * c[:, k])
        assert s == pytest.approx(b2 ** 2 * d4(a, b, g, k), abs=1e-15)
    for idx in itertools.product(range(2), repeat=6):
        a, b, g, k, t, p = idx
        s = np.sum(w * c[:, a] * c[:, b] * c[:, g] * c[:, k] * c[:, t] * c[:, p])
        d6 = (_delta(a, b) * d4(g, k, t, p) + _delta(a, g) * d4(b, k, t, p)
              + _delta(a, k) * d4(b, g, t, p) + _delta(a, t) * d4(b, g, k, p)
              + _delta(a, p) * d4(b, g, k, t))
        all_eq = 1.0 if len(set(idx)) == 1 else 0.0
        assert s == pytest.approx(b2 ** 3 * (d6 - 6 * all_eq), abs=1e-15)
    # odd moments vanish
    for a, b, g in itertools.product(range(2), repeat=3):
        assert np.sum(w * c[:, a] * c[:, b] * c[:, g]) == pytest.approx(0.0, abs=1e-16)


def test_equilibrium_moments():
    """Eq. 12 under the consistent reading: the moments of f^eq (Eqs. 14-15)
    are rho, j, P and Q^eq = b^2 (j_a d_bg + j_b d_ag + j_g d_ab)."""
    cx, cy, w, b2 = oracle.lattice()
    c = np.stack([cx, cy], 1).astype(float)
    rng = np.random.default_rng(7)
    for _ in range(20):
        rho, jx, jy, pxx, pxy, pyy = rng.standard_normal(6)
        feq = oracle.equilibrium(rho, jx, jy, pxx, pxy, pyy)
        j = np.array([jx, jy])
        P = np.array([[pxx, pxy], [pxy, pyy]])
        assert np.sum(feq) == pytest.approx(rho, abs=1e-14)
        np.testing.assert_allclose(feq @ c, j, atol=1e-14)
        np.testing.assert_allclose(np.einsum("i,ia,ib->ab", feq, c, c), P, atol=1e-14)
        Q = np.einsum("i,ia,ib,ig->abg", feq, c, c, c)
        for a, b, g in itertools.product(range(2), repeat=3):
            want = b2 * (j[a] * _delta(b, g) + j[b] * _delta(a, g) + j[g] * _delta(a, b))
            assert Q[a, b, g] == pytest.approx(want, abs=1e-14)


def test_forcing_moments():
    """Eq. 11 with the solvability conditions of Eq. 22: sum S_i = 0,
    sum S_i c = S, sum S_i c c = 0."""
    cx, cy, w, b2 = oracle.lattice()
    c = np.stack([cx, cy], 1).astype(float)
    for sx, sy in [(1.0, 0.0), (0.0, 1.0), (0.3, -2.5)]:
        si = oracle.forcing(sx, sy)
        assert np.sum(si) == pytest.approx(0.0, abs=1e-15)
        np.testing.assert_allclose(si @ c, [sx, sy], atol=1e-15)
        np.testing.assert_allclose(np.einsum("i,ia,ib->ab", si, c, c), 0.0, atol=1e-15)


def test_ricker_closed_form():
    """Sec. 5 Ricker wavelet: peak 1 at t0, zeros at t0 +- 1/(pi f sqrt 2),
    zero mean, minimum -2 exp(-3/2) at t0 +- sqrt(3/2)/(pi f)."""
    f, t0 = 0.05, 30.0
    assert oracle.ricker(t0, f, t0) == pytest.approx(1.0, abs=1e-15)
    tz = 1.0 / (math.pi * f * math.sqrt(2.0))
    assert oracle.ricker(t0 + tz, f, t0) == pytest.approx(0.0, abs=1e-14)
    assert oracle.ricker(t0 - tz, f, t0) == pytest.approx(0.0, abs=1e-14)
    tm = math.sqrt(1.5) / (math.pi * f)
    assert oracle.ricker(t0 + tm, f, t0) == pytest.approx(-2 * math.exp(-1.5), abs=1e-14)
    ts = np.linspace(t0 - 200, t0 + 200, 40001)
    vals = np.array([oracle.ricker(t, f, t0) for t in ts[::10]])
    assert abs(np.trapezoid(vals, ts[::10])) < 1e-9
    # the oracle's wavelet equals the closed form kept with the theory helpers
    for t in [0.0, 12.5, 30.0, 41.0, 99.0]:
        assert oracle.ricker(t, f, t0) == pytest.approx(theory.ricker(t, f, t0), abs=1e-15)


def test_gaussian_source_field():
    """Sec. 5 source: the force of step n at a cell is
    amplitude * dir * exp(-r^2/(2 sigma^2)) * ricker(n) inside r_cut, zero
    outside; minimum-image distance on a periodic axis."""
    nx = ny = 40
    src = np.array([[3.0, 20.0, 2.0, 0.6, 0.8, 2.0, 0.05, 10.0, 6.0]])
    prob = oracle.Problem(nx=nx, ny=ny, sources=src)
    F = oracle.force(prob, 12)
    r = oracle.ricker(12, 0.05, 10.0)
    # cell (39, 21) is at minimum-image distance sqrt(16 + 1) from (3, 20)
    g = math.exp(-17.0 / 8.0)
    assert F[0, 21, 39] == pytest.approx(2.0 * 0.6 * g * r, rel=1e-14)
    assert F[1, 21, 39] == pytest.approx(2.0 * 0.8 * g * r, rel=1e-14)
    # beyond r_cut = 6
    assert F[0, 20, 10] == 0.0 and F[1, 27, 3] == 0.0
    assert F[1, 26, 3] != 0.0  # exactly at r_cut: kept
    # non-periodic x: no wrap
    prob2 = oracle.Problem(nx=nx, ny=ny, sources=src, bc_left="rigid", bc_right="rigid")
    assert oracle.force(prob2, 12)[0, 21, 39] == 0.0


def test_sponge_profile():
    """Sec. 6.4 absorbing coefficient (profile is the documented reading):
    A = A_max (d/L)^2, d = depth into the layer, zero in the interior, the
    largest value in corners, A_max = 12.8/L by default."""
    prob = oracle.Problem(nx=30, ny=20, sponge=(0, 4, 8, 5))
    A = oracle.sponge(prob)
    assert A[5, 15] == 0.0
    assert A[5, 8] == 0.0 and A[5, 7] == pytest.approx(12.8 / 8 * (1 / 8) ** 2)
    assert A[5, 0] == pytest.approx(12.8 / 8)
    assert A[19, 15] == pytest.approx(12.8 / 4)
    assert A[15, 15] == 0.0 and A[16, 15] == pytest.approx(12.8 / 4 * (1 / 4) ** 2)
    assert A[5, 29] == pytest.approx(12.8 / 5)
    assert A[19, 0] == pytest.approx(max(12.8 / 8, 12.8 / 4))
    prob = oracle.Problem(nx=30, ny=20, sponge=(3, 0, 0, 0), sponge_amax=0.5)
    A = oracle.sponge(prob)
    assert A[0, 10] == pytest.approx(0.5) and A[3, 10] == 0.0


def test_closed_forms(golden):
    """Eq. 5 and the nu limit (Sec. 4): v_P = 1 at nu = 0.25 and v_P = 2 at
    nu = 5/11; the Rayleigh root at nu = 0.25 (Sec. 7, Eq. 46)."""
    b = math.sqrt(theory.B2)
    assert theory.vp_over_vs(0.25) * b == pytest.approx(1.0, abs=1e-15)
    nl = golden["nu_limit"]
    assert theory.vp_over_vs(nl["nu_lim"]) * b == pytest.approx(nl["vP_at_limit"], abs=1e-12)
    ra = golden["rayleigh"]
    xi = theory.rayleigh_xi(0.25)
    assert xi == pytest.approx(2 - 2 / math.sqrt(3), abs=1e-12)
    assert xi == pytest.approx(ra["xi"], abs=5e-5)
    assert math.sqrt(xi * theory.B2) == pytest.approx(ra["vR_theory"], abs=5e-5)
    lam, mu = theory.lame_from_nu(0.3)
    assert theory.poisson_ratio(lam, mu) == pytest.approx(0.3, abs=1e-15)
    assert (mu - lam) / theory.B2 == pytest.approx(theory.Lambda_of_nu(0.3), abs=1e-14)
