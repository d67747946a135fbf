"""Pins of the oracle's wall treatment of the density gradient (no GPU).

The paper defines grad(rho) (Eq. 10) only as the interior centred
difference; the ghost values one cell outside a wall are a reading (rigid
wall: rho_b; free surface: the extrapolation of Eq. 39's order, 2 rho_b -
rho_in or rho_b).  Three checks that do not restate that reading pin it:

* a rigid wall (half-way bounce-back, Eq. 36) is a mirror plane: for a field
  that does not vary along the wall, the walled run equals half of a
  periodic run on the doubled domain holding the mirror image (method of
  images) — exact, whatever the material of each row;
* the divergence theorem at a free surface: summed over the solid, the
  centred differences telescope to a surface term, and the y-momentum the
  density-gradient force adds across the solid in one step must be
  Lambda b^2 times the wall
  density that the anti-bounce-back rule itself uses (Eq. 39's rho_air; the
  rule exchanges no momentum with the wall) — exact;
* the Rayleigh speed for nu != 0.25: the free-surface rule imposes P n = 0,
  which is the traction-free condition with lambda replaced by mu, so the
  surface wave travels at the root of the correspondingly modified Rayleigh
  equation (``theory.rayleigh_xi_scheme``), 3-4 % away from the elastic
  root at nu = 0.2 and 0.3.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import theory

CX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
CY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
OPP = np.array([0, 3, 4, 1, 2, 7, 8, 5, 6])
B2 = 1.0 / 3.0


def _layers(n, seed):
    """Per-row (or per-column) rho0, lambda, mu with v_S = b and nu in
    [0.15, 0.35], so Lambda differs from row to row and from zero."""
    rng = np.random.default_rng(seed)
    rho0 = rng.uniform(1.0, 2.0, n)
    nu = rng.uniform(0.15, 0.35, n)
    mu = rho0 * B2
    lam = 2.0 * mu * nu / (1.0 - 2.0 * nu)
    return rho0, lam, mu


def _momentum(fs):
    return np.array([np.einsum("iyx,i->", fs, CX), np.einsum("iyx,i->", fs, CY)])


@pytest.mark.parametrize("axis", ["y", "x"])
def test_rigid_wall_is_a_mirror_plane(axis):
    """Eq. 36 with the density-gradient force (Eq. 9): a field that does not
    vary along the walls, between two rigid walls, evolves exactly as the
    first half of a periodic domain of twice the width holding the field's
    mirror image (row y' = 2n - 1 - y carries the populations of velocity
    -c_i and the displacement -u).  This holds only if the wall's ghost
    density is the mirror value rho_b."""
    rng = np.random.default_rng(7)
    n, m, steps, tau = 9, 3, 6, 0.8
    rho0, lam, mu = _layers(n, 8)
    prof = rng.standard_normal((9, n))
    uprof = rng.standard_normal((2, n))
    img = np.concatenate([prof, prof[OPP][:, ::-1]], axis=1)
    uimg = np.concatenate([uprof, -uprof[:, ::-1]], axis=1)
    mat2 = [np.concatenate([a, a[::-1]]) for a in (rho0, lam, mu)]
    if axis == "y":
        # rows vary, columns identical; rigid top and bottom, periodic x
        fs = np.repeat(prof[:, :, None], m, 2)
        u = np.repeat(uprof[:, :, None], m, 2)
        walled = oracle.Problem(nx=m, ny=n, tau=tau, bc_top="rigid", bc_bottom="rigid",
                                rho0=rho0, lam=lam, mu=mu)
        doubled = oracle.Problem(nx=m, ny=2 * n, tau=tau, rho0=mat2[0], lam=mat2[1], mu=mat2[2])
        fs2 = np.repeat(img[:, :, None], m, 2)
        u2 = np.repeat(uimg[:, :, None], m, 2)
        half = (slice(None), slice(0, n), slice(None))
    else:
        # columns vary, rows identical; rigid left and right, periodic y
        fs = np.repeat(prof[:, None, :], m, 1)
        u = np.repeat(uprof[:, None, :], m, 1)
        cell = lambda a: np.repeat(a[None, :], m, 0)  # noqa: E731
        walled = oracle.Problem(nx=n, ny=m, tau=tau, bc_left="rigid", bc_right="rigid",
                                rho0=cell(rho0), lam=cell(lam), mu=cell(mu))
        doubled = oracle.Problem(nx=2 * n, ny=m, tau=tau, rho0=cell(mat2[0]),
                                 lam=cell(mat2[1]), mu=cell(mat2[2]))
        fs2 = np.repeat(img[:, None, :], m, 1)
        u2 = np.repeat(uimg[:, None, :], m, 1)
        half = (slice(None), slice(None), slice(0, n))
    a, _ = oracle.run(walled, steps, oracle.State(walled, fs=fs, u=u), traces=False)
    b, _ = oracle.run(doubled, steps, oracle.State(doubled, fs=fs2, u=u2), traces=False)
    np.testing.assert_allclose(a.fs, b.fs[half], rtol=0, atol=1e-12)
    np.testing.assert_allclose(a.u, b.u[half], rtol=0, atol=1e-12)
    # and the changes are not trivial: the force is at work at the walls
    assert np.abs(a.fs - fs).max() > 0.1


def _wall_density(rb, rin, fs_order):
    """rho at a free surface as the anti-bounce-back rule extrapolates it
    (Eq. 39): 1.5 rho_b - 0.5 rho_in, or rho_b for the constant reading."""
    return 1.5 * rb - 0.5 * rin if fs_order == 1 else rb


@pytest.mark.parametrize("fs_order", [0, 1])
@pytest.mark.parametrize("axis", ["y", "x"])
def test_free_surface_force_sum_is_the_surface_term(fs_order, axis):
    """Divergence theorem for the density-gradient force (Eqs. 9-10) on a
    solid between two free surfaces (Eqs. 37-42), periodic along them, with
    Lambda constant across the solid (it varies along the surfaces): in one
    step the normal momentum sum f* c changes by
    b^2 sum_along Lambda (rho_wall(far side) - rho_wall(near side)), rho_wall
    the surface density of Eq. 39 extrapolated from the streamed densities;
    the anti-bounce-back exchanges no momentum with the wall, and the
    tangential sum changes only by the interior differences along the
    surfaces."""
    rng = np.random.default_rng(11 + fs_order)
    n, m = 7, 8                      # n across the solid, m along the surfaces
    rho0, lam, mu = _layers(m, 12)
    if axis == "y":
        cell = lambda a: np.repeat(a[None, :], n, 0)  # noqa: E731  varies along x
        prob = oracle.Problem(nx=m, ny=n, tau=0.8, bc_top="free", bc_bottom="free",
                              fs_order=fs_order, rho0=cell(rho0), lam=cell(lam), mu=cell(mu))
        fs = rng.standard_normal((9, n, m))
    else:
        cell = lambda a: np.repeat(a[:, None], n, 1)  # noqa: E731  varies along y
        prob = oracle.Problem(nx=n, ny=m, tau=0.8, bc_left="free", bc_right="free",
                              fs_order=fs_order, rho0=cell(rho0), lam=cell(lam), mu=cell(mu))
        fs = rng.standard_normal((9, m, n))
    st = oracle.State(prob, fs=fs)
    rho = oracle.fields(prob, st)["rho"]          # streamed density of this step
    if axis == "x":
        rho = rho.T                               # [across][along]
    Lam = (mu - lam) / (rho0 * B2)
    near = _wall_density(rho[0], rho[1], fs_order)
    far = _wall_density(rho[-1], rho[-2], fs_order)
    expect = B2 * np.sum(Lam * (far - near))
    m0 = _momentum(fs)
    st, _ = oracle.run(prob, 1, st, traces=False)
    dm = _momentum(st.fs) - m0
    normal, tangential = (1, 0) if axis == "y" else (0, 1)
    # along the surfaces the differences are interior (periodic) ones
    along = B2 * np.sum(Lam * 0.5 * (np.roll(rho, -1, 1) - np.roll(rho, 1, 1)))
    assert abs(expect) > 0.1
    assert dm[normal] == pytest.approx(expect, abs=1e-12)
    assert dm[tangential] == pytest.approx(along, abs=1e-12)


@pytest.mark.slow
@pytest.mark.parametrize("nu", [0.2, 0.3])
def test_rayleigh_speed_off_poisson(nu, ncpu):
    """Sec. 7 generalised to nu != 0.25 (Lambda != 0, so the density-gradient
    force acts up to the surface): the surface wave between two surface
    receivers 200 cells apart travels at sqrt(xi b^2), xi the root of the
    Rayleigh equation for the boundary condition the free-surface rule
    imposes (P n = 0), within 0.4 %; it is 3-4 % from the root for a
    traction-free surface."""
    nx, ny, L = 800, 160, 40
    lam, mu = theory.lame_from_nu(nu)
    src = [160.0, 2.0, 3.0, 0.0, 1.0, 1.0, 0.05, 30.0, 24.0]
    x1, x2 = 300, 500
    prob = oracle.Problem(nx=nx, ny=ny, tau=1.0, rho0=np.ones(ny), lam=np.full(ny, lam),
                          mu=np.full(ny, mu), sources=np.atleast_2d(src),
                          receivers=np.array([[x1, 0], [x2, 0]], np.int32), nthreads=ncpu,
                          bc_top="free", bc_bottom="rigid", sponge=(0, L, L, L), fs_order=0)
    _, tr = oracle.run(prob, 760)
    v_scheme = math.sqrt(theory.rayleigh_xi_scheme(nu) * B2)
    v_elastic = math.sqrt(theory.rayleigh_xi(nu) * B2)

    def window(sig, x):
        t_arr = src[7] + (x - src[0]) / v_scheme
        w = np.zeros_like(sig)
        w[int(t_arr - 30):int(t_arr + 30)] = sig[int(t_arr - 30):int(t_arr + 30)]
        return w

    nfft, up = 1 << 14, 16
    A = np.fft.rfft(window(tr[:, 0, 3], x1), nfft)
    B = np.fft.rfft(window(tr[:, 1, 3], x2), nfft)
    lag = np.argmax(np.fft.irfft(B * np.conj(A), nfft * up)) / up
    v = (x2 - x1) / lag
    assert v == pytest.approx(v_scheme, rel=4e-3)
    assert abs(v / v_elastic - 1) > 0.02
