"""Discrete adjoint of the oracle's time step, by brute force, for tiny grids.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The step (Sec. 2, Eq. 18, with the boundaries of Sec. 6 and the sources of
Sec. 5) is affine in the state s = (f*, u):  s^{n+1} = M s^n + c^n, with M
independent of n and c^n the response to the body force of step n.  For a
fixed state it is also affine in Lambda(x) = (mu - lambda)/(rho0 b^2) at
every cell, since Lambda enters only through the force Lambda b^2 grad rho
(Eq. 9), and in each source amplitude.  This module

* builds M column by column, stepping unit states through ``oracle.run``;
* gets d s^{n+1} / d Lambda(x) as step(s^n; Lambda + e_x) - step(s^n; Lambda)
  and d s^{n+1} / d A_s as the step of the rest state with source s alone at
  unit amplitude;
* runs the reverse-mode recursion
      a^T = dJ/ds^T,   a^n = M^T a^{n+1} + dJ/ds^n,
      dJ/dLambda(x) += a^{n+1} . d s^{n+1}/d Lambda(x),
      dJ/dA_s       += a^{n+1} . d s^{n+1}/d A_s.

Every derivative comes from the forward step itself; nothing of the adjoint
is written out by hand.  The traces are tr^n = (u^{n+1}(x_r), v^n(x_r)) with
v^n = j^n / rho0 = u^{n+1}(x_r) - u^n(x_r) (the displacement rule u += j/rho0).
"""
from __future__ import annotations

from dataclasses import replace

import numpy as np

from . import Problem, State, run

B2 = 1.0 / 3.0


def _vec(st: State) -> np.ndarray:
    return np.concatenate([st.fs.ravel(), st.u.ravel()])


def _state(prob: Problem, v: np.ndarray, n: int) -> State:
    m = 9 * prob.nx * prob.ny
    return State(prob, fs=v[:m].reshape(9, prob.ny, prob.nx),
                 u=v[m:].reshape(2, prob.ny, prob.nx), n=n)


def _bare(prob: Problem) -> Problem:
    return replace(prob, sources=np.zeros((0, 9)), receivers=np.zeros((0, 2), np.int32))


def _cells(prob: Problem, a, default):
    return prob._cell_array(a, default)


def step_matrix(prob: Problem) -> np.ndarray:
    """M: the step of the state without sources, as a dense matrix."""
    bare = _bare(prob)
    N = 11 * prob.nx * prob.ny
    M = np.zeros((N, N))
    for k in range(N):
        e = np.zeros(N)
        e[k] = 1.0
        st, _ = run(bare, 1, _state(bare, e, 0), traces=False)
        M[:, k] = _vec(st)
    return M


def forward_states(prob: Problem, nsteps: int):
    """s^0 (rest) .. s^T and the traces [T][nrec][4]."""
    st = State(prob)
    out = [_vec(st)]
    trs = []
    for _ in range(nsteps):
        st, tr = run(prob, 1, st, traces=True)
        out.append(_vec(st))
        trs.append(tr[0] if tr is not None else np.zeros((0, 4)))
    return out, np.array(trs)


def misfit(traces: np.ndarray, data: np.ndarray) -> float:
    """J = 1/2 sum over steps and receivers of |u - u_data|^2 (the
    displacement components of the traces)."""
    d = traces[..., :2] - data[..., :2]
    return 0.5 * float(np.sum(d * d))


def misfit_trace_adjoint(traces: np.ndarray, data: np.ndarray) -> np.ndarray:
    g = np.zeros_like(traces)
    g[..., :2] = traces[..., :2] - data[..., :2]
    return g


def gradients(prob: Problem, nsteps: int, dtraces: np.ndarray, cells=None):
    """dJ/dLambda per cell ([ny][nx]; only ``cells`` if given, a list of
    (x, y)) and dJ/dA per source, for trace derivatives dtraces [T][nrec][4]
    of the run from rest."""
    nx, ny = prob.nx, prob.ny
    ncell = nx * ny
    N = 11 * ncell
    M = step_matrix(prob)
    states, _ = forward_states(prob, nsteps)
    rec = np.asarray(prob.receivers, np.int64).reshape(-1, 2)
    # dJ/ds^n from the traces
    dsd = [np.zeros(N) for _ in range(nsteps + 1)]
    for n in range(nsteps):
        for r, (x, y) in enumerate(rec):
            for comp in range(2):
                iu = 9 * ncell + comp * ncell + y * nx + x
                dsd[n + 1][iu] += dtraces[n, r, comp] + dtraces[n, r, 2 + comp]
                dsd[n][iu] -= dtraces[n, r, 2 + comp]
    bare = _bare(prob)
    rho0 = _cells(prob, prob.rho0, 1.0)
    lam = _cells(prob, prob.lam, None) if prob.lam is not None else rho0 / 3.0
    mu = _cells(prob, prob.mu, None) if prob.mu is not None else rho0 / 3.0
    if cells is None:
        cells = [(x, y) for y in range(ny) for x in range(nx)]
    src = np.asarray(prob.sources, np.float64).reshape(-1, 9)
    gL = np.zeros((ny, nx))
    gA = np.zeros(len(src))
    a = dsd[nsteps].copy()
    for n in range(nsteps - 1, -1, -1):
        s_n = _state(bare, states[n], n)
        base, _ = run(bare, 1, s_n, traces=False)
        base = _vec(base)
        for (x, y) in cells:
            lp = lam.copy()
            lp[y, x] -= rho0[y, x] * B2  # Lambda(x) + 1
            pert, _ = run(replace(bare, lam=lp, mu=mu, rho0=rho0), 1,
                          _state(bare, states[n], n), traces=False)
            gL[y, x] += a @ (_vec(pert) - base)
        for s in range(len(src)):
            one = src[s:s + 1].copy()
            one[0, 5] = 1.0
            c, _ = run(replace(bare, sources=one), 1, State(bare, n=n), traces=False)
            gA[s] += a @ _vec(c)
        a = M.T @ a + dsd[n]
    return gL, gA


def lambda_gradients(prob: Problem, g_Lambda: np.ndarray):
    """dJ/dlambda and dJ/dmu from dJ/dLambda (Lambda = (mu - lambda)/(rho0 b^2),
    rho0 fixed)."""
    rho0 = _cells(prob, prob.rho0, 1.0)
    return -g_Lambda / (rho0 * B2), g_Lambda / (rho0 * B2)
