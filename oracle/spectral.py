"""Fourier spectral / Crank-Nicolson Navier solver of Appendix B
(TEST INFRASTRUCTURE ONLY).

Per wavevector k the state is J = (j_x, j_y, d_t j_x, d_t j_y) (Eq. 53) and the
Navier equation for the mass flux (Eq. 54) is advanced by the Crank-Nicolson
step M J_{n+1} = N (J_n, G_x, G_y) (Eqs. 56-62), with
G = (d_t F_n + d_t F_{n+1}) / rho0 and A, B, C of Eq. 62.  The grid is periodic;
k takes the continuous-Fourier values 2 pi m / N.
"""
from __future__ import annotations

import numpy as np

from .theory import ricker, ricker_dt


def gaussian(nx, ny, xs, ys, sigma, r_cut=None):
    """g(x) = exp(-|x - x_s|^2 / (2 sigma^2)) with minimum-image distances,
    cut at r_cut like the oracle's source (Sec. 5)."""
    X, Y = np.meshgrid(np.arange(nx, dtype=float), np.arange(ny, dtype=float))
    dx = X - xs
    dy = Y - ys
    dx -= nx * np.floor(dx / nx + 0.5)
    dy -= ny * np.floor(dy / ny + 0.5)
    r2 = dx * dx + dy * dy
    g = np.exp(-r2 / (2 * sigma * sigma))
    if r_cut is not None:
        g[r2 > r_cut * r_cut] = 0.0
    return g


def crank_nicolson(nx, ny, lam, mu, rho0, src, nsteps, dt=1.0, substeps=1):
    """Mass flux j = (j_x, j_y) after ``nsteps`` time units.

    ``src`` = (x, y, sigma, dir_x, dir_y, amplitude, f_peak, t0, r_cut) like the
    oracle's sources.  ``substeps`` > 1 refines the time step (dt/substeps)."""
    xs, ys, sigma, dxs, dys, amp, fp, t0, rc = src
    g = gaussian(nx, ny, xs, ys, sigma, rc)
    gh = np.fft.fft2(g)
    kx = 2 * np.pi * np.fft.fftfreq(nx)[None, :] * np.ones((ny, 1))
    ky = 2 * np.pi * np.fft.fftfreq(ny)[:, None] * np.ones((1, nx))
    a2 = (lam + 2 * mu) / rho0
    b2 = mu / rho0
    d2 = (lam + mu) / rho0
    A = a2 * kx ** 2 + b2 * ky ** 2
    B = d2 * kx * ky
    C = a2 * ky ** 2 + b2 * kx ** 2
    h = dt / substeps
    # M and N of Eqs. 60-61, one pair per k
    M = np.zeros((ny, nx, 4, 4))
    M[..., 0, 0] = M[..., 1, 1] = M[..., 2, 2] = M[..., 3, 3] = 1.0
    M[..., 0, 2] = M[..., 1, 3] = -h / 2
    M[..., 2, 0] = A * h / 2
    M[..., 2, 1] = B * h / 2
    M[..., 3, 0] = B * h / 2
    M[..., 3, 1] = C * h / 2
    N = np.zeros((ny, nx, 4, 6))
    N[..., 0, 0] = N[..., 1, 1] = N[..., 2, 2] = N[..., 3, 3] = 1.0
    N[..., 0, 2] = N[..., 1, 3] = h / 2
    N[..., 2, 0] = -A * h / 2
    N[..., 2, 1] = -B * h / 2
    N[..., 3, 0] = -B * h / 2
    N[..., 3, 1] = -C * h / 2
    N[..., 2, 4] = h / 2
    N[..., 3, 5] = h / 2
    Minv = np.linalg.inv(M)
    T = Minv @ N  # (ny, nx, 4, 6)
    J = np.zeros((ny, nx, 4), complex)
    for n in range(nsteps * substeps):
        t0n, t1n = n * h, (n + 1) * h
        gsum = (ricker_dt(t0n, fp, t0) + ricker_dt(t1n, fp, t0)) * amp / rho0
        G = np.stack([gh * dxs * gsum, gh * dys * gsum], axis=-1)
        X = np.concatenate([J, G], axis=-1)
        J = np.einsum("yxij,yxj->yxi", T, X)
    jx = np.real(np.fft.ifft2(J[..., 0]))
    jy = np.real(np.fft.ifft2(J[..., 1]))
    return jx, jy


def misfit(j_lbm: np.ndarray, j_ref: np.ndarray) -> float:
    """Relative L2 misfit p of Eq. 34."""
    return float(np.sqrt(np.sum((j_lbm - j_ref) ** 2) / np.sum(j_ref ** 2)))
