"""Plain FP64 CPU oracle of the elastic-solid D2Q9 LBM step (arXiv 2009.06404).

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  The product path
(the CUDA library and its Python binding) never imports, links or runs it, and it
shares no code with that path.

Contents
--------
``lbm_oracle.c``   the time step itself (plain C, FP64): streaming, wall rules,
                   moments, density gradient, source, absorbing layer,
                   equilibrium, BGK with forcing, displacement, receivers.
``vonneumann.py``  the amplification matrix M(k) of Sec. 4 (Eq. 31), derived
                   from the scheme, and its brute-force counterpart built from
                   ``lbm_oracle.c`` on small periodic grids.
``spectral.py``    the Fourier/Crank-Nicolson Navier solver of Appendix B.
``theory.py``      closed forms: wave speeds (Eq. 4), Poisson ratio (Eq. 6),
                   Lambda(nu) (Eq. 32), the Rayleigh equation.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liblbm_oracle.so")
_lock = threading.Lock()
_lib = None

BC = {"periodic": 0, "free": 1, "rigid": 2}


def build(force: bool = False) -> str:
    """Compile ``lbm_oracle.c`` with gcc (-O2, no FP contraction); OpenMP if
    the compiler has it.  Returns the library path."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    base = ["gcc", "-std=gnu11", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
            _SRC, "-o", _LIB_PATH + ".tmp", "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_LIB_PATH + ".tmp", _LIB_PATH)
    return _LIB_PATH


class _Problem(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("tau", ctypes.c_double),
        ("bc_top", ctypes.c_int), ("bc_bottom", ctypes.c_int),
        ("bc_left", ctypes.c_int), ("bc_right", ctypes.c_int),
        ("sp_top", ctypes.c_int), ("sp_bottom", ctypes.c_int),
        ("sp_left", ctypes.c_int), ("sp_right", ctypes.c_int),
        ("sp_amax", ctypes.c_double), ("fs_order", ctypes.c_int),
        ("rho0", ctypes.c_void_p), ("lam", ctypes.c_void_p), ("mu", ctypes.c_void_p),
        ("nsrc", ctypes.c_int), ("src", ctypes.c_void_p),
        ("nrec", ctypes.c_int), ("rec", ctypes.c_void_p),
        ("nthreads", ctypes.c_int),
    ]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            # LBM_ORACLE_LIB lets the mutation tests load a deliberately broken
            # build of this oracle in a child process.
            path = os.environ.get("LBM_ORACLE_LIB") or build()
            L = ctypes.CDLL(path)
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int)
            pp = ctypes.POINTER(_Problem)
            L.oracle_lattice.argtypes = [ip, ip, dp, dp]
            L.oracle_equilibrium.argtypes = [ctypes.c_double] * 6 + [dp]
            L.oracle_forcing.argtypes = [ctypes.c_double, ctypes.c_double, dp]
            L.oracle_ricker.argtypes = [ctypes.c_double] * 3
            L.oracle_ricker.restype = ctypes.c_double
            L.oracle_run.argtypes = [pp, dp, dp, ctypes.c_long, ctypes.c_int, dp]
            L.oracle_fields.argtypes = [pp, dp, dp, ctypes.c_long, dp]
            L.oracle_stream.argtypes = [pp, dp, dp]
            L.oracle_sponge.argtypes = [pp, dp]
            L.oracle_force.argtypes = [pp, ctypes.c_long, dp]
            L.oracle_has_openmp.restype = ctypes.c_int
            _lib = L
    return _lib


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


@dataclass
class Problem:
    """One simulation set-up, in the oracle's own terms (all FP64, per cell)."""
    nx: int
    ny: int
    tau: float = 1.0
    bc_top: str = "periodic"
    bc_bottom: str = "periodic"
    bc_left: str = "periodic"
    bc_right: str = "periodic"
    sponge: Sequence[int] = (0, 0, 0, 0)  # top, bottom, left, right
    sponge_amax: float = 0.0
    fs_order: int = 1                    # free-surface extrapolation: 1 linear, 0 constant
    rho0: Optional[np.ndarray] = None    # [ny][nx] or [ny] (expanded)
    lam: Optional[np.ndarray] = None
    mu: Optional[np.ndarray] = None
    sources: np.ndarray = field(default_factory=lambda: np.zeros((0, 9)))
    receivers: np.ndarray = field(default_factory=lambda: np.zeros((0, 2), np.int32))
    nthreads: int = 1

    def _cell_array(self, a, default):
        if a is None:
            return np.full((self.ny, self.nx), default, np.float64)
        a = np.asarray(a, np.float64)
        if a.ndim == 1:
            a = np.repeat(a[:, None], self.nx, axis=1)
        return np.ascontiguousarray(a.reshape(self.ny, self.nx))

    def _struct(self):
        rho0 = self._cell_array(self.rho0, 1.0)
        # default: Poisson solid (lambda = mu = rho0/3)
        mu = self._cell_array(self.mu, None) if self.mu is not None else rho0 / 3.0
        lam = self._cell_array(self.lam, None) if self.lam is not None else rho0 / 3.0
        src = np.ascontiguousarray(np.asarray(self.sources, np.float64).reshape(-1, 9))
        rec = np.ascontiguousarray(np.asarray(self.receivers, np.int32).reshape(-1, 2))
        keep = (rho0, mu, lam, src, rec)
        s = _Problem(self.nx, self.ny, float(self.tau),
                     BC[self.bc_top], BC[self.bc_bottom], BC[self.bc_left], BC[self.bc_right],
                     *[int(v) for v in self.sponge], float(self.sponge_amax),
                     int(self.fs_order), rho0.ctypes.data, lam.ctypes.data, mu.ctypes.data,
                     src.shape[0], src.ctypes.data if src.size else None,
                     rec.shape[0], rec.ctypes.data if rec.size else None,
                     int(self.nthreads))
        return s, keep


class State:
    """Post-collision populations f* [9][ny][nx], displacement u [2][ny][nx] and
    the index n of the next step."""

    def __init__(self, prob: Problem, fs=None, u=None, n: int = 0):
        shape = (prob.ny, prob.nx)
        self.fs = (np.zeros((9,) + shape) if fs is None
                   else np.array(fs, np.float64, copy=True).reshape((9,) + shape))
        self.u = (np.zeros((2,) + shape) if u is None
                  else np.array(u, np.float64, copy=True).reshape((2,) + shape))
        self.n = int(n)


def run(prob: Problem, nsteps: int, state: Optional[State] = None,
        traces: bool = True):
    """Advance ``state`` (a fresh rest state if None) by ``nsteps`` steps.
    Returns (state, traces[nsteps][nrec][4] or None)."""
    L = lib()
    st = state if state is not None else State(prob)
    s, keep = prob._struct()
    nrec = s.nrec
    tr = np.zeros((max(nsteps, 0), nrec, 4)) if (traces and nrec) else None
    rc = L.oracle_run(ctypes.byref(s), _dptr(st.fs), _dptr(st.u), st.n, int(nsteps),
                      _dptr(tr) if tr is not None else None)
    if rc != 0:
        raise ValueError("oracle_run rejected the problem")
    st.n += max(int(nsteps), 0)
    del keep
    return st, tr


def fields(prob: Problem, state: State) -> dict:
    """ux, uy, vx, vy, rho, Pxx, Pxy, Pyy of ``state`` (each [ny][nx])."""
    L = lib()
    s, keep = prob._struct()
    out = np.zeros((8, prob.ny, prob.nx))
    rc = L.oracle_fields(ctypes.byref(s), _dptr(np.ascontiguousarray(state.fs)),
                         _dptr(np.ascontiguousarray(state.u)), state.n, _dptr(out))
    if rc != 0:
        raise ValueError("oracle_fields rejected the problem")
    del keep
    names = ["ux", "uy", "vx", "vy", "rho", "pxx", "pxy", "pyy"]
    return {k: out[i] for i, k in enumerate(names)}


def stream(prob: Problem, fs: np.ndarray) -> np.ndarray:
    L = lib()
    s, keep = prob._struct()
    fs = np.ascontiguousarray(fs, np.float64)
    out = np.zeros_like(fs)
    if L.oracle_stream(ctypes.byref(s), _dptr(fs), _dptr(out)) != 0:
        raise ValueError("oracle_stream rejected the problem")
    del keep
    return out


def sponge(prob: Problem) -> np.ndarray:
    L = lib()
    s, keep = prob._struct()
    out = np.zeros((prob.ny, prob.nx))
    L.oracle_sponge(ctypes.byref(s), _dptr(out))
    del keep
    return out


def force(prob: Problem, n: int) -> np.ndarray:
    L = lib()
    s, keep = prob._struct()
    out = np.zeros((2, prob.ny, prob.nx))
    L.oracle_force(ctypes.byref(s), int(n), _dptr(out))
    del keep
    return out


def lattice():
    L = lib()
    cx = (ctypes.c_int * 9)()
    cy = (ctypes.c_int * 9)()
    w = (ctypes.c_double * 9)()
    b2 = ctypes.c_double()
    L.oracle_lattice(cx, cy, w, ctypes.byref(b2))
    return np.array(cx[:]), np.array(cy[:]), np.array(w[:]), b2.value


def equilibrium(rho, jx, jy, pxx, pxy, pyy) -> np.ndarray:
    out = np.zeros(9)
    lib().oracle_equilibrium(rho, jx, jy, pxx, pxy, pyy, _dptr(out))
    return out


def forcing(sx, sy) -> np.ndarray:
    out = np.zeros(9)
    lib().oracle_forcing(sx, sy, _dptr(out))
    return out


def ricker(t, f, t0) -> float:
    return lib().oracle_ricker(float(t), float(f), float(t0))


def has_openmp() -> bool:
    return bool(lib().oracle_has_openmp())
