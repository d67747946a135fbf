"""Von Neumann analysis of the scheme (Sec. 4) -- TEST INFRASTRUCTURE ONLY.

Two independent constructions of the one-step amplification matrix for a
plane wave f_l(x) = a_l exp(+i k.x) on a periodic lattice with F = 0, A = 0:

* :func:`analytic_collision` / :func:`analytic_matrix`: derived by hand from
  Eqs. 9-18.  For a plane wave, the centred difference of Eq. 10 gives
  grad(rho) = i s rho with s = (sin k_x, sin k_y); with j = m + S/2 and
  S = Lambda b^2 i s rho the collision acts on the amplitudes as

      C_lj = (1 - 1/tau) delta_lj
             + (w_l / tau) [1 + c_l.c_j / b^2 + H_l:H_j / (2 b^4) + (i Lambda / 2) c_l.s]
             + (1 - 1/(2 tau)) i Lambda w_l c_l.s,          H_l = c_l c_l - b^2 I,

  and pull streaming multiplies population l by exp(-i k.c_l).  This is the
  matrix of Eq. 31 with the printed last term corrected (Eq. 31 as printed
  lacks w_l and the imaginary unit and carries an extra b^2).
* :func:`brute_force_matrix`: one step of the C oracle applied to the nine unit
  plane waves on an N x N periodic grid, read back at the origin.

The analytic matrix returned is for the post-collision state that the oracle
advances (M = C D); the paper's pre-collision form D C has the same
eigenvalues.
"""
from __future__ import annotations

import numpy as np

from . import Problem, State, run
from .theory import B2, lame_from_nu

# The lattice is restated here (not imported from the C file) so that the
# brute-force comparison checks the C tables too.
CX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
CY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


def analytic_collision(kx: float, ky: float, tau: float, Lam: float) -> np.ndarray:
    s = np.array([np.sin(kx), np.sin(ky)])
    C = np.zeros((9, 9), complex)
    for l in range(9):
        cl = np.array([CX[l], CY[l]], float)
        Hl = np.outer(cl, cl) - B2 * np.eye(2)
        cs = cl @ s
        for j in range(9):
            cj = np.array([CX[j], CY[j]], float)
            Hj = np.outer(cj, cj) - B2 * np.eye(2)
            eq = 1.0 + (cl @ cj) / B2 + np.sum(Hl * Hj) / (2 * B2 * B2) + 0.5j * Lam * cs
            C[l, j] = (W[l] / tau) * eq + (1 - 1 / (2 * tau)) * 1j * Lam * W[l] * cs
        C[l, l] += 1 - 1 / tau
    return C


def streaming(kx: float, ky: float) -> np.ndarray:
    return np.diag(np.exp(-1j * (kx * CX + ky * CY)))


def analytic_matrix(kx, ky, tau, Lam, post_collision_state=True) -> np.ndarray:
    C = analytic_collision(kx, ky, tau, Lam)
    D = streaming(kx, ky)
    return C @ D if post_collision_state else D @ C


def Lambda_from_nu(nu: float) -> float:
    lam, mu = lame_from_nu(nu)
    return (mu - lam) / (1.0 * B2)


def brute_force_matrix(N: int, ikx: int, iky: int, tau: float, nu: float) -> np.ndarray:
    """Amplification matrix of the oracle's step for k = 2 pi (ikx, iky) / N.

    The step is real and linear, so the real and imaginary parts of each unit
    plane wave are stepped separately.  Also checks that the output is again a
    plane wave of the same k (raises otherwise)."""
    lam, mu = lame_from_nu(nu)
    prob = Problem(nx=N, ny=N, tau=tau,
                   rho0=np.ones(N), lam=np.full(N, lam), mu=np.full(N, mu))
    kx, ky = 2 * np.pi * ikx / N, 2 * np.pi * iky / N
    X, Y = np.meshgrid(np.arange(N), np.arange(N))
    phase = np.exp(1j * (kx * X + ky * Y))
    M = np.zeros((9, 9), complex)
    for l in range(9):
        out = np.zeros((9, N, N), complex)
        for part, scale in ((phase.real, 1.0), (phase.imag, 1j)):
            fs = np.zeros((9, N, N))
            fs[l] = part
            st, _ = run(prob, 1, State(prob, fs=fs), traces=False)
            out += scale * st.fs
        col = out[:, 0, 0]
        if not np.allclose(out, col[:, None, None] * phase[None], atol=1e-12):
            raise AssertionError("oracle step does not map a plane wave to itself")
        M[:, l] = col
    return M


def spectral_radius(kx, ky, tau, Lam) -> float:
    return float(np.max(np.abs(np.linalg.eigvals(analytic_matrix(kx, ky, tau, Lam)))))


def phase_speeds(kmag: float, theta: float, tau: float, Lam: float) -> np.ndarray:
    """|arg(eig)| / |k| of the eigenvalues with modulus near 1 and non-zero
    phase (propagating modes), sorted."""
    kx, ky = kmag * np.cos(theta), kmag * np.sin(theta)
    ev = np.linalg.eigvals(analytic_matrix(kx, ky, tau, Lam))
    sp = [abs(np.angle(e)) / kmag for e in ev if abs(abs(e) - 1) < 0.05 and abs(np.angle(e)) > 1e-3 * kmag]
    return np.sort(np.array(sp))
