"""Shared test helpers: turn a seeded workload into the oracle's problem and
compare arrays."""
import os

import numpy as np

import oracle


def oracle_problem(w, nthreads=None):
    return oracle.Problem(nx=w.nx, ny=w.ny, tau=w.tau, bc_top=w.bc[0], bc_bottom=w.bc[1],
                          bc_left=w.bc[2], bc_right=w.bc[3], sponge=tuple(w.sponge),
                          sponge_amax=w.sponge_amax, fs_order=w.fs_order, rho0=w.rho0, lam=w.lam, mu=w.mu,
                          sources=w.sources, receivers=w.receivers,
                          nthreads=nthreads or max(1, min(16, os.cpu_count() or 1)))


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def max_rel(a, b):
    """max |a - b| / max |b|"""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    s = np.max(np.abs(b))
    return float(np.max(np.abs(a - b)) / (s if s > 0 else 1.0))


def two_lap_speed(uy, nx, t_from, window=300, guess=0.5308, span=0.05):
    """Speed of a wave going round an nx-periodic surface from the surface
    displacement uy [T][nx]: the time lag L (within span of 2 nx / guess)
    that best aligns the window [t_from, t_from + window) of every receiver
    with the same receiver two laps later, refined by a parabola through the
    correlation peak; returns 2 nx / L (the paper's two-turn measurement)."""
    uy = np.asarray(uy, np.float64)
    lag0 = 2.0 * nx / guess
    lags = np.arange(int(lag0 * (1 - span)), int(lag0 * (1 + span)) + 1)
    a = uy[t_from:t_from + window]
    corr = np.array([float(np.sum(a * uy[t_from + L:t_from + L + window])) for L in lags])
    k = int(np.argmax(corr))
    if not 0 < k < len(lags) - 1:
        raise ValueError("correlation peak at the edge of the search range")
    c0, c1, c2 = corr[k - 1], corr[k], corr[k + 1]
    L = lags[k] + 0.5 * (c0 - c2) / (c0 - 2 * c1 + c2)
    return 2.0 * nx / L
