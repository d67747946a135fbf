"""Pins of the oracle's brute-force discrete adjoint (oracle/adjoint.py)
against what does not depend on it: central finite differences of the
oracle's own misfit.  The misfit is quadratic in the source amplitudes (the
traces are affine in them), so central differences are exact there up to
rounding; in Lambda the traces are polynomials, and a small step pins the
gradient to a few parts in 1e7."""
import numpy as np
import pytest

import oracle
from oracle import adjoint as adj

B2 = 1.0 / 3.0


def _problem(fs_order=1, bc=("free", "rigid", "periodic", "periodic"), sponge=(0, 2, 0, 0)):
    nx, ny = 7, 6
    rng = np.random.default_rng(7)
    rho0 = rng.uniform(1.0, 2.0, size=(ny, nx))
    nu = rng.uniform(0.2, 0.3, size=(ny, nx))
    mu = rho0 * B2
    lam = 2 * nu * mu / (1 - 2 * nu)
    src = np.array([[3.2, 2.1, 1.0, 0.6, 0.8, 1.0, 0.3, 2.0, 3.0],
                    [5.0, 4.0, 0.8, 1.0, 0.0, 0.7, 0.25, 3.0, 2.0]])
    rec = np.array([[0, 0], [4, 1], [6, 5]], np.int32)
    return oracle.Problem(nx=nx, ny=ny, tau=0.8, bc_top=bc[0], bc_bottom=bc[1], bc_left=bc[2],
                          bc_right=bc[3], sponge=sponge, fs_order=fs_order, rho0=rho0, lam=lam,
                          mu=mu, sources=src, receivers=rec)


def _J(prob, T, data):
    _, tr = oracle.run(prob, T)
    return adj.misfit(tr, data)


def _data(prob, T):
    rng = np.random.default_rng(3)
    _, tr = oracle.run(prob, T)
    return tr + 0.3 * np.abs(tr).max() * rng.standard_normal(tr.shape)


@pytest.mark.parametrize("fs_order,bc,sponge", [
    (1, ("free", "rigid", "periodic", "periodic"), (0, 2, 0, 0)),
    (0, ("free", "free", "rigid", "rigid"), (0, 0, 2, 0)),
])
def test_amplitude_gradient_equals_central_differences(fs_order, bc, sponge):
    prob = _problem(fs_order, bc, sponge)
    T = 8
    data = _data(prob, T)
    _, tr = oracle.run(prob, T)
    _, gA = adj.gradients(prob, T, adj.misfit_trace_adjoint(tr, data), cells=[])
    for s in range(2):
        h = 1e-3
        src_p = prob.sources.copy()
        src_m = prob.sources.copy()
        src_p[s, 5] += h
        src_m[s, 5] -= h
        fd = (_J(oracle.Problem(**{**prob.__dict__, "sources": src_p}), T, data) -
              _J(oracle.Problem(**{**prob.__dict__, "sources": src_m}), T, data)) / (2 * h)
        assert abs(gA[s] - fd) <= 1e-9 * max(abs(fd), 1e-12), (s, gA[s], fd)


@pytest.mark.parametrize("fs_order,bc,sponge", [
    (1, ("free", "rigid", "periodic", "periodic"), (0, 2, 0, 0)),
    (0, ("free", "free", "rigid", "rigid"), (0, 0, 2, 0)),
])
def test_lambda_gradient_equals_central_differences(fs_order, bc, sponge):
    prob = _problem(fs_order, bc, sponge)
    T = 8
    data = _data(prob, T)
    _, tr = oracle.run(prob, T)
    cells = [(0, 0), (3, 2), (6, 5), (1, 4)]
    gL, _ = adj.gradients(prob, T, adj.misfit_trace_adjoint(tr, data), cells=cells)
    rho0 = np.asarray(prob.rho0)
    for (x, y) in cells:
        h = 1e-4
        lp = np.array(prob.lam, copy=True)
        lm = np.array(prob.lam, copy=True)
        lp[y, x] -= h * rho0[y, x] * B2   # Lambda(x) + h
        lm[y, x] += h * rho0[y, x] * B2   # Lambda(x) - h
        fd = (_J(oracle.Problem(**{**prob.__dict__, "lam": lp}), T, data) -
              _J(oracle.Problem(**{**prob.__dict__, "lam": lm}), T, data)) / (2 * h)
        assert abs(gL[y, x] - fd) <= 1e-6 * max(abs(fd), 1e-9) + 1e-12, ((x, y), gL[y, x], fd)


def test_lambda_and_mu_gradients_are_opposite():
    """Lambda = (mu - lambda)/(rho0 b^2): dJ/dmu = -dJ/dlambda = dJ/dLambda/(rho0 b^2)."""
    prob = _problem()
    g = np.random.default_rng(1).standard_normal((prob.ny, prob.nx))
    gl, gm = adj.lambda_gradients(prob, g)
    assert np.allclose(gl, -gm)
    assert np.allclose(gm * np.asarray(prob.rho0) * B2, g)


def test_step_matrix_reproduces_the_step():
    """M applied to a random state equals the oracle's step without sources."""
    prob = _problem()
    M = adj.step_matrix(prob)
    rng = np.random.default_rng(2)
    v = rng.standard_normal(M.shape[0])
    bare = adj._bare(prob)
    st, _ = oracle.run(bare, 1, adj._state(bare, v, 0), traces=False)
    assert np.allclose(M @ v, adj._vec(st), rtol=0, atol=1e-13 * np.abs(v).max())
