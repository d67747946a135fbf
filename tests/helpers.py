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
