"""Pins of the oracle's whole time step (no GPU): conservation (Eqs. 22, 12),
linearity and the rest state, lattice symmetries, and the von Neumann
amplification matrix of Sec. 4 rebuilt independently."""
import math

import numpy as np
import pytest

import oracle
from oracle import theory, vonneumann as vn

CX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
CY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])


def _prob(nx, ny=None, nu=0.25, tau=1.0, **kw):
    ny = ny or nx
    lam, mu = theory.lame_from_nu(nu)
    return oracle.Problem(nx=nx, ny=ny, tau=tau, lam=np.full(ny, lam),
                          mu=np.full(ny, mu), rho0=np.ones(ny), **kw)


def _sums(fs):
    c = np.stack([CX, CY], 1).astype(float)
    rho = fs.sum()
    m = np.einsum("iyx,ia->a", fs, c)
    P = np.einsum("iyx,ia,ib->ab", fs, c, c)
    return rho, m, P


def test_rest_state_is_fixed_point():
    """f_i = w_i rho_r is a fixed point of Eq. 18 on a periodic grid for any
    nu (grad rho = 0, j = 0, P^n = 0); the zero state too."""
    _, _, w, _ = oracle.lattice()
    for nu in (0.25, 0.1, 0.33):
        prob = _prob(12, nu=nu, tau=0.7)
        fs = np.repeat(w[:, None, None], 12, 1).repeat(12, 2) * 1.7
        st, _ = oracle.run(prob, 5, oracle.State(prob, fs=fs), traces=False)
        np.testing.assert_allclose(st.fs, fs, atol=1e-15)
        np.testing.assert_allclose(st.u, 0.0, atol=1e-15)
    st, _ = oracle.run(prob, 3, traces=False)
    assert np.all(st.fs == 0.0)


def test_linearity():
    """With F = 0 the step is linear in (f*, u)."""
    prob = _prob(10, nu=0.2, tau=0.8, bc_top="free", bc_bottom="rigid", sponge=(0, 3, 2, 2))
    rng = np.random.default_rng(1)
    a = rng.standard_normal((9, 10, 10))
    b = rng.standard_normal((9, 10, 10))
    sa, _ = oracle.run(prob, 3, oracle.State(prob, fs=a), traces=False)
    sb, _ = oracle.run(prob, 3, oracle.State(prob, fs=b), traces=False)
    sab, _ = oracle.run(prob, 3, oracle.State(prob, fs=2 * a - 0.5 * b), traces=False)
    np.testing.assert_allclose(sab.fs, 2 * sa.fs - 0.5 * sb.fs, atol=1e-12)
    np.testing.assert_allclose(sab.u, 2 * sa.u - 0.5 * sb.u, atol=1e-12)


@pytest.mark.parametrize("nu", [0.25, 0.1, 0.3])
def test_periodic_invariants_without_force(nu):
    """Periodic grid, F = 0, uniform Lambda: sum rho and sum P are conserved
    (collision conserves both, Eq. 22; streaming permutes), and sum m too
    because the centred difference of Eq. 10 telescopes."""
    prob = _prob(16, nu=nu, tau=0.6)
    rng = np.random.default_rng(2)
    fs = 1e-2 * rng.standard_normal((9, 16, 16))
    r0, m0, P0 = _sums(fs)
    st, _ = oracle.run(prob, 7, oracle.State(prob, fs=fs), traces=False)
    r1, m1, P1 = _sums(st.fs)
    assert r1 == pytest.approx(r0, abs=1e-14)
    np.testing.assert_allclose(m1, m0, atol=1e-14)
    np.testing.assert_allclose(P1, P0, atol=1e-14)


def test_momentum_grows_by_body_force():
    """With a source, the post-collision flux sum f* c grows by the total body
    force of each step (Guo forcing: sum f* c = sum f c + S, Eqs. 18, 22)."""
    src = np.array([[7.3, 8.1, 2.0, 0.6, -0.8, 1.5, 0.05, 4.0, 6.0]])
    prob = _prob(16, nu=0.3, tau=0.9, sources=src)
    st = oracle.State(prob)
    for n in range(6):
        _, m0, _ = _sums(st.fs)
        F = oracle.force(prob, n).sum(axis=(1, 2))
        st, _ = oracle.run(prob, 1, st, traces=False)
        _, m1, _ = _sums(st.fs)
        np.testing.assert_allclose(m1 - m0, F, atol=1e-14)


def test_rigid_walls_conserve_mass():
    """Half-way bounce-back (Eq. 36) returns every population that leaves
    through a wall, so sum rho is conserved with rigid top and bottom."""
    prob = _prob(12, nu=0.25, tau=0.7, bc_top="rigid", bc_bottom="rigid")
    rng = np.random.default_rng(3)
    fs = rng.standard_normal((9, 12, 12))
    st, _ = oracle.run(prob, 9, oracle.State(prob, fs=fs), traces=False)
    assert st.fs.sum() == pytest.approx(fs.sum(), abs=1e-12)


def test_bounce_back_rule():
    """Eq. 36 on the bottom wall: the populations entering a bottom-row cell
    upward equal the downward post-collision populations of the same cell."""
    prob = _prob(6, bc_top="rigid", bc_bottom="rigid")
    rng = np.random.default_rng(4)
    fs = rng.standard_normal((9, 6, 6))
    f = oracle.stream(prob, fs)
    opp = {2: 4, 5: 7, 6: 8, 4: 2, 7: 5, 8: 6}
    for i in (4, 7, 8):          # c_y = -1: enter the bottom row from below
        np.testing.assert_array_equal(f[i][5], fs[opp[i]][5])
    for i in (2, 5, 6):          # c_y = +1: enter the top row from above
        np.testing.assert_array_equal(f[i][0], fs[opp[i]][0])
    # interior links are plain shifts
    np.testing.assert_array_equal(f[1][2], np.roll(fs[1][2], 1))
    np.testing.assert_array_equal(f[5][3], np.roll(fs[5][2], 1))


@pytest.mark.parametrize("fs_order", [0, 1])
def test_free_surface_rule_preserves_equilibrium_of_air_state(fs_order):
    """Eqs. 37-42: if the post-collision populations at the surface cell and
    the cell below are the equilibria of a state with zero flux whose stress
    has only the tangential component, the anti-bounce-back returns the
    equilibrium population itself (-f + 2 f^eq = f^eq), with either
    extrapolation to the wall."""
    prob = _prob(6, bc_top="free", bc_bottom="rigid", fs_order=fs_order)
    rho, pxx = 0.37, 0.21
    feq = oracle.equilibrium(rho, 0.0, 0.0, pxx, 0.0, 0.0)
    fs = np.zeros((9, 6, 6))
    fs[:, :, :] = feq[:, None, None]
    f = oracle.stream(prob, fs)
    for i in (2, 5, 6):
        np.testing.assert_allclose(f[i][0], feq[i], atol=1e-15)


@pytest.mark.parametrize("fs_order", [0, 1])
def test_free_surface_extrapolation(fs_order):
    """Eqs. 38-42: f_ibar = -f*_i + 2 w_i (rho_air + P^n_air : H_i / (2 b^4)),
    with P_air keeping only the tangential stress.  fs_order = 1 is the
    printed linear extrapolation rho_air = 1.5 rho_b - 0.5 rho_in (Eq. 39) and
    the same for the stress; fs_order = 0 takes the boundary cell's values."""
    _, _, w, b2 = oracle.lattice()
    prob = _prob(5, bc_top="free", bc_bottom="free", fs_order=fs_order)
    rng = np.random.default_rng(5)
    fs = rng.standard_normal((9, 5, 5))
    f = oracle.stream(prob, fs)
    c = np.stack([CX, CY], 1).astype(float)
    x = 2

    def mom(y):
        v = fs[:, y, x]
        return v.sum(), np.einsum("i,i,i", v, c[:, 0], c[:, 0])

    for (yb, yin, incoming) in ((0, 1, (2, 5, 6)), (4, 3, (4, 7, 8))):
        rb, pb = mom(yb)
        ri, pi = mom(yin)
        if fs_order == 1:
            rho_air, pxx_air = 1.5 * rb - 0.5 * ri, 1.5 * pb - 0.5 * pi
        else:
            rho_air, pxx_air = rb, pb
        Pn = np.array([[pxx_air - b2 * rho_air, 0.0], [0.0, -b2 * rho_air]])
        for i in incoming:
            k = [j for j in range(9) if CX[j] == -CX[i] and CY[j] == -CY[i]][0]
            H = np.outer(c[k], c[k]) - b2 * np.eye(2)
            want = -fs[k, yb, x] + 2 * w[k] * (rho_air + np.sum(Pn * H) / (2 * b2 * b2))
            assert f[i, yb, x] == pytest.approx(want, abs=1e-14)


def _boundary_radius(fs_order, nu, tau, ny=12, n=8, bc=("free", "rigid")):
    """Largest |eigenvalue| of the one-step operator of a channel that is
    periodic in x (plane waves exp(i k_x x), k_x = 2 pi m / n) and bounded by
    the given walls in y, built column by column from the oracle's step."""
    lam, mu = theory.lame_from_nu(nu)
    p = oracle.Problem(nx=n, ny=ny, tau=tau, bc_top=bc[0], bc_bottom=bc[1], rho0=np.ones(ny),
                       lam=np.full(ny, lam), mu=np.full(ny, mu), fs_order=fs_order)
    X = np.arange(n)
    best = 0.0
    for m in range(n // 2 + 1):
        ph = np.exp(2j * np.pi * m * X / n)
        M = np.zeros((9 * ny, 9 * ny), complex)
        for col in range(9 * ny):
            i, y = divmod(col, ny)
            out = np.zeros((9, ny, n), complex)
            for part, sc in ((ph.real, 1.0), (ph.imag, 1j)):
                fs = np.zeros((9, ny, n))
                fs[i, y, :] = part
                st, _ = oracle.run(p, 1, oracle.State(p, fs=fs), traces=False)
                out += sc * st.fs
            M[:, col] = out[:, :, 0].reshape(-1)
        best = max(best, float(np.abs(np.linalg.eigvals(M)).max()))
    return best


@pytest.mark.slow
def test_wall_stability():
    """Rigid walls (Eq. 36) and the free surface with constant extrapolation
    add no growing mode (|eig| <= 1 for every tangential wavenumber, nu = 0.2
    and 0.3 at tau = 1); the printed linear extrapolation (Eq. 39) does: its
    largest eigenvalue exceeds 1 (about 1.046 per step at nu = 0.25, tau = 1)."""
    assert _boundary_radius(0, 0.25, 1.0, bc=("rigid", "rigid")) <= 1 + 1e-12
    for nu in (0.2, 0.3):
        assert _boundary_radius(0, nu, 1.0) <= 1 + 1e-12
    r = _boundary_radius(1, 0.25, 1.0)
    assert r > 1.02


def _rotate90(fs):
    """Rotate a periodic state by +90 degrees: cell (x, y) -> (-y, x),
    velocity (cx, cy) -> (-cy, cx)."""
    n = fs.shape[1]
    out = np.empty_like(fs)
    perm = {}
    for i in range(9):
        j = [k for k in range(9) if CX[k] == -CY[i] and CY[k] == CX[i]][0]
        perm[i] = j
    ys, xs = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    nx_, ny_ = (-ys) % n, xs
    for i in range(9):
        out[perm[i], ny_, nx_] = fs[i, ys, xs]
    return out


def test_square_symmetry():
    """The scheme commutes with a 90-degree rotation of the periodic lattice
    (D2Q9 square symmetry; no source)."""
    prob = _prob(12, nu=0.15, tau=0.8)
    rng = np.random.default_rng(6)
    fs = rng.standard_normal((9, 12, 12))
    a, _ = oracle.run(prob, 2, oracle.State(prob, fs=fs), traces=False)
    b, _ = oracle.run(prob, 2, oracle.State(prob, fs=_rotate90(fs)), traces=False)
    np.testing.assert_allclose(b.fs, _rotate90(a.fs), atol=1e-13)


@pytest.mark.parametrize("nu,tau", [(0.25, 1.0), (0.1, 0.55), (0.37, 1.0), (0.0, 0.7)])
def test_amplification_matrix_brute_force(nu, tau):
    """Sec. 4, Eq. 31: one oracle step on the nine unit plane waves of an 8x8
    periodic grid equals the hand-derived matrix C(k) D(k) to 1e-13."""
    for ikx, iky in [(1, 0), (0, 3), (2, 1), (3, 3), (4, 1), (4, 4)]:
        Mb = vn.brute_force_matrix(8, ikx, iky, tau, nu)
        Ma = vn.analytic_matrix(2 * np.pi * ikx / 8, 2 * np.pi * iky / 8, tau,
                                theory.Lambda_of_nu(nu))
        assert np.abs(Mb - Ma).max() < 1e-13


def test_zero_wavenumber_spectrum():
    """At k = 0 the six conserved/forced moments give eigenvalue 1 and the
    three relaxed moments 1 - 1/tau."""
    for tau in (0.55, 1.0, 1.7):
        ev = np.sort_complex(np.linalg.eigvals(vn.analytic_matrix(0.0, 0.0, tau, 0.4)))
        want = np.sort_complex(np.array([1.0] * 6 + [1 - 1 / tau] * 3, complex))
        np.testing.assert_allclose(ev, want, atol=1e-12)


def _max_radius(nu, tau, kmax, n=41, theta=None):
    L = theory.Lambda_of_nu(nu)
    best = 0.0
    if theta is not None:
        for k in np.linspace(0, kmax, n):
            best = max(best, vn.spectral_radius(k * math.cos(theta), k * math.sin(theta), tau, L))
        return best
    for kx in np.linspace(0, kmax, n):
        for ky in np.linspace(0, kmax, n):
            if kx * kx + ky * ky <= kmax * kmax + 1e-12:
                best = max(best, vn.spectral_radius(kx, ky, tau, L))
    return best


def test_stability_claims(golden):
    """Sec. 4: nu = 0.25 is stable for every k; for the other Poisson ratios
    plotted (tau = 0.55) eigenvalues leave the unit disk along 45 degrees;
    even at nu = 0.4 every |k| <= pi/3 is stable; at nu = 0.4 all directions
    become unstable at high enough k, while nu = 0 is unstable only near 45
    degrees."""
    s = golden["stability"]
    tau = 0.55
    assert _max_radius(s["stable_nu"], tau, math.pi, n=31) <= 1 + 1e-12
    for nu in s["unstable_nu_at_45deg"]:
        assert _max_radius(nu, tau, math.pi, n=61, theta=math.pi / 4) > 1 + 1e-3
    for nu in (0.0, 0.1, 0.2, 0.3, 0.35, 0.4):
        assert _max_radius(nu, tau, s["stable_k_norm_below"], n=21) <= 1 + 1e-12
    # off the diagonal (5 and 20 degrees): nu = 0.4 unstable, nu = 0 stable
    for deg in (5.0, 20.0):
        th = math.radians(deg)
        kmax = math.pi / math.cos(th)
        assert _max_radius(s["all_directions_unstable_nu"], tau, kmax, n=121, theta=th) > 1 + 1e-3
        assert _max_radius(0.0, tau, kmax, n=121, theta=th) <= 1 + 1e-12


def test_instability_stripe_spacing(golden):
    """Sec. 4, Fig. 3: the 45-degree instability of low-nu runs shows stripes
    2.1 cells apart, i.e. the fastest-growing 45-degree wave has wavelength
    2 pi / |k| close to 2.1."""
    L = theory.Lambda_of_nu(0.0)
    ks = np.linspace(1.5, math.pi, 400)
    rad = [vn.spectral_radius(k / math.sqrt(2), k / math.sqrt(2), 0.55, L) for k in ks]
    kbest = ks[int(np.argmax(rad))]
    assert 2 * math.pi / kbest == pytest.approx(golden["stability"]["stripe_spacing_45deg"], abs=0.15)


@pytest.mark.parametrize("nu", [0.0, 0.1, 0.25, 0.3])
def test_small_k_phase_speeds(nu):
    """The propagating eigenvalues of M(k) at small k travel at v_S = b and
    v_P of Eq. 4 (Eq. 5 ratio), in every direction."""
    lam, mu = theory.lame_from_nu(nu)
    vp, vs = theory.wave_speeds(lam, mu, 1.0)
    for theta in (0.0, 0.4, math.pi / 4):
        sp = vn.phase_speeds(0.01, theta, 1.0, theory.Lambda_of_nu(nu))
        assert len(sp) == 4
        np.testing.assert_allclose(sp, [vs, vs, vp, vp], rtol=2e-4)
