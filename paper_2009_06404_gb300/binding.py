"""ctypes binding of the C ABI in ``include/lbm_elastic.h``.

Argument marshalling only: every step of the method runs in the CUDA library.
PyTorch provides the device workspace (a uint8 CUDA tensor) and the stream.
If the library has not been built, or CUDA is unavailable, the calls raise;
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Dict, Optional, Sequence

import numpy as np

from . import build as _build

LBM_OK = 0
LBM_WARN_VS_NOT_B = 1
STATUS = {0: "LBM_OK", 1: "LBM_WARN_VS_NOT_B", -1: "LBM_ERR_ARG", -2: "LBM_ERR_UNSUPPORTED",
          -3: "LBM_ERR_WORKSPACE", -4: "LBM_ERR_CUDA", -5: "LBM_ERR_NONFINITE",
          -6: "LBM_ERR_TIMEOUT", -7: "LBM_ERR_CAPACITY"}
STORAGE = {"f64": 0, "f32": 1, "f16": 2, "bf16": 3}
BC = {"periodic": 0, "free": 1, "rigid": 2}
KERNEL = {"auto": 0, "simple": 1}

#: the exported symbols, as declared in include/lbm_elastic.h
SYMBOLS = [
    "lbm_elastic_workspace_bytes", "lbm_elastic_create", "lbm_elastic_set_material",
    "lbm_elastic_set_sources", "lbm_elastic_set_receivers", "lbm_elastic_set_sponges",
    "lbm_elastic_reset", "lbm_elastic_step", "lbm_elastic_set_steps_per_launch",
    "lbm_elastic_step_index", "lbm_elastic_read_fields",
    "lbm_elastic_traces_recorded", "lbm_elastic_read_traces", "lbm_elastic_set_state",
    "lbm_elastic_get_state", "lbm_elastic_checkpoint_bytes", "lbm_elastic_save",
    "lbm_elastic_load", "lbm_elastic_moment_sums", "lbm_elastic_sync",
    "lbm_elastic_destroy", "lbm_elastic_last_error", "lbm_elastic_status_string",
    "lbm_elastic_kernel_launches", "lbm_elastic_moment_sums_noalloc",
    "lbm_batch_workspace_bytes", "lbm_batch_create", "lbm_batch_set_launch",
    "lbm_batch_get_launch", "lbm_batch_autotune", "lbm_batch_step", "lbm_batch_sync",
    "lbm_batch_kernel_launches", "lbm_batch_cells", "lbm_batch_destroy",
    "lbm_batch_last_error",
    "lbm_adjoint_workspace_bytes", "lbm_adjoint_create", "lbm_adjoint_forward",
    "lbm_adjoint_backward", "lbm_adjoint_gradients", "lbm_adjoint_set_state",
    "lbm_adjoint_get_state", "lbm_adjoint_step_linear", "lbm_adjoint_set_fused",
    "lbm_adjoint_kernel_launches",
    "lbm_adjoint_destroy", "lbm_adjoint_last_error",
]


class LBMError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class NonFiniteError(LBMError):
    pass


class Config(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("storage", ctypes.c_int),
        ("u_fp64", ctypes.c_int), ("tau", ctypes.c_double),
        ("bc_top", ctypes.c_int), ("bc_bottom", ctypes.c_int),
        ("bc_left", ctypes.c_int), ("bc_right", ctypes.c_int),
        ("sponge_top", ctypes.c_int), ("sponge_bottom", ctypes.c_int),
        ("sponge_left", ctypes.c_int), ("sponge_right", ctypes.c_int),
        ("sponge_amax", ctypes.c_double), ("free_surface_order", ctypes.c_int),
        ("material_per_cell", ctypes.c_int),
        ("max_sources", ctypes.c_int), ("max_receivers", ctypes.c_int),
        ("max_steps_traced", ctypes.c_int), ("kernel_variant", ctypes.c_int),
        ("store_scale_log2", ctypes.c_int),
    ]


class BatchLaunch(ctypes.Structure):
    _fields_ = [
        ("mode", ctypes.c_int), ("rows", ctypes.c_int), ("order", ctypes.c_int),
        ("graph_steps", ctypes.c_int), ("steps_per_launch", ctypes.c_int),
        ("ctas_per_sm", ctypes.c_int), ("barrier_cycles", ctypes.c_longlong),
        ("barrier_extra", ctypes.c_int), ("steps_per_tile", ctypes.c_int),
    ]


BATCH_MODE = {"auto": 0, "stream": 1, "graph": 2, "persistent": 3}


class Source(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in
                ("x", "y", "sigma", "dir_x", "dir_y", "amplitude", "f_peak", "t0", "r_cut")]


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB


def load_library(build_if_missing: bool = False):
    """Loads the CUDA library (raises if it is missing and not built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_build.LIB):
            if not build_if_missing:
                raise RuntimeError(
                    "CUDA library not built: run paper_2009_06404_gb300.build.build() "
                    "(or __graft_entry__.build()) first")
            _build.build()
        L = ctypes.CDLL(_build.LIB)
        vp, dp, ip = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int
        cfgp = ctypes.POINTER(Config)
        sig = {
            "lbm_elastic_workspace_bytes": (ctypes.c_size_t, [cfgp]),
            "lbm_elastic_create": (ip, [cfgp, vp, ctypes.c_size_t, vp, ctypes.POINTER(vp)]),
            "lbm_elastic_set_material": (ip, [vp, vp, vp, vp, ip]),
            "lbm_elastic_set_sources": (ip, [vp, ctypes.POINTER(Source), ip]),
            "lbm_elastic_set_receivers": (ip, [vp, vp, ip]),
            "lbm_elastic_set_sponges": (ip, [vp, ip, ip, ip, ip, ctypes.c_double]),
            "lbm_elastic_reset": (ip, [vp]),
            "lbm_elastic_step": (ip, [vp, ip]),
            "lbm_elastic_set_steps_per_launch": (ip, [vp, ip]),
            "lbm_elastic_step_index": (ctypes.c_longlong, [vp]),
            "lbm_elastic_read_fields": (ip, [vp] + [vp] * 8 + [ip]),
            "lbm_elastic_traces_recorded": (ip, [vp]),
            "lbm_elastic_read_traces": (ip, [vp, vp, ip]),
            "lbm_elastic_set_state": (ip, [vp, vp, vp, ctypes.c_longlong, ip]),
            "lbm_elastic_get_state": (ip, [vp, vp, vp, ip]),
            "lbm_elastic_checkpoint_bytes": (ctypes.c_size_t, [vp]),
            "lbm_elastic_save": (ip, [vp, vp, ip]),
            "lbm_elastic_load": (ip, [vp, vp, ip]),
            "lbm_elastic_moment_sums": (ip, [vp, dp]),
            "lbm_elastic_sync": (ip, [vp]),
            "lbm_elastic_destroy": (ip, [vp]),
            "lbm_elastic_last_error": (ctypes.c_char_p, [vp]),
            "lbm_elastic_status_string": (ctypes.c_char_p, [ip]),
            "lbm_elastic_kernel_launches": (ctypes.c_longlong, [vp]),
            "lbm_elastic_moment_sums_noalloc": (ip, [vp, vp, ip, ip, ip, ip, ip, vp, ip, vp]),
            "lbm_batch_workspace_bytes": (ctypes.c_size_t, [ctypes.POINTER(vp), ip]),
            "lbm_batch_create": (ip, [ctypes.POINTER(vp), ip, vp, ctypes.c_size_t, vp,
                                      ctypes.POINTER(vp)]),
            "lbm_batch_set_launch": (ip, [vp, ctypes.POINTER(BatchLaunch)]),
            "lbm_batch_get_launch": (ip, [vp, ctypes.POINTER(BatchLaunch)]),
            "lbm_batch_autotune": (ip, [vp, ip, dp]),
            "lbm_batch_step": (ip, [vp, ip]),
            "lbm_batch_sync": (ip, [vp]),
            "lbm_batch_kernel_launches": (ctypes.c_longlong, [vp]),
            "lbm_batch_cells": (ctypes.c_longlong, [vp]),
            "lbm_batch_destroy": (ip, [vp]),
            "lbm_batch_last_error": (ctypes.c_char_p, [vp]),
            "lbm_adjoint_workspace_bytes": (ctypes.c_size_t, [vp, ip, ip]),
            "lbm_adjoint_create": (ip, [vp, ip, ip, vp, ctypes.c_size_t, ctypes.POINTER(vp)]),
            "lbm_adjoint_forward": (ip, [vp]),
            "lbm_adjoint_backward": (ip, [vp, vp]),
            "lbm_adjoint_gradients": (ip, [vp, vp, vp, vp, vp]),
            "lbm_adjoint_set_state": (ip, [vp, vp, vp]),
            "lbm_adjoint_get_state": (ip, [vp, vp, vp]),
            "lbm_adjoint_step_linear": (ip, [vp]),
            "lbm_adjoint_set_fused": (ip, [vp, ip]),
            "lbm_adjoint_kernel_launches": (ctypes.c_longlong, [vp]),
            "lbm_adjoint_destroy": (ip, [vp]),
            "lbm_adjoint_last_error": (ctypes.c_char_p, [vp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
        return L


def make_config(nx, ny, storage="f32", tau=1.0, bc=("periodic",) * 4, sponge=(0, 0, 0, 0),
                sponge_amax=0.0, material_per_cell=False, max_sources=16, max_receivers=256,
                max_steps_traced=0, u_fp64=False, fs_order=0, kernel="auto",
                store_scale_log2=0) -> Config:
    return Config(int(nx), int(ny), STORAGE[storage], int(bool(u_fp64)), float(tau),
                  BC[bc[0]], BC[bc[1]], BC[bc[2]], BC[bc[3]], *[int(s) for s in sponge],
                  float(sponge_amax), int(fs_order), int(bool(material_per_cell)),
                  int(max_sources), int(max_receivers), int(max_steps_traced),
                  KERNEL[kernel], int(store_scale_log2))


def _ptr(t) -> Optional[int]:
    """Address of a torch tensor or numpy array (None passes NULL)."""
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


class ElasticLBM:
    """One simulation on the current CUDA device, over a torch-owned workspace.

    All device work runs on ``stream`` (default: torch's current stream).
    Host-side arrays are numpy; device-side arrays are torch tensors.
    """

    def __init__(self, nx, ny, storage="f32", tau=1.0, bc=("periodic",) * 4,
                 sponge=(0, 0, 0, 0), sponge_amax=0.0, material_per_cell=False,
                 max_sources=16, max_receivers=256, max_steps_traced=0, u_fp64=False,
                 fs_order=0, kernel="auto", store_scale_log2=0, device=None, stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("ElasticLBM needs a CUDA device (no CPU fallback)")
        self._torch = torch
        self.L = load_library()
        self.cfg = make_config(nx, ny, storage, tau, bc, sponge, sponge_amax, material_per_cell,
                               max_sources, max_receivers, max_steps_traced, u_fp64, fs_order,
                               kernel, store_scale_log2)
        self.nx, self.ny = int(nx), int(ny)
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        nbytes = self.L.lbm_elastic_workspace_bytes(ctypes.byref(self.cfg))
        if nbytes == 0:
            raise LBMError(-1, "invalid configuration")
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            # 256 extra bytes so the start can be aligned to 256
            self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        base = self.workspace.data_ptr()
        self._ws_off = (-base) % 256
        h = ctypes.c_void_p()
        st = self.L.lbm_elastic_create(ctypes.byref(self.cfg), base + self._ws_off, nbytes,
                                       self.stream.cuda_stream, ctypes.byref(h))
        if st != LBM_OK:
            raise LBMError(st, self.L.lbm_elastic_last_error(None).decode())
        self.h = h
        self.workspace_bytes = nbytes
        self.nsrc = 0
        self.nrec = 0

    # ------------------------------------------------------------ helpers
    def _check(self, st, allow_warn=False):
        if st == LBM_OK or (allow_warn and st == LBM_WARN_VS_NOT_B):
            return st
        msg = self.L.lbm_elastic_last_error(self.h).decode()
        if st == -5:
            raise NonFiniteError(st, msg)
        raise LBMError(st, msg)

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self.L.lbm_elastic_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ------------------------------------------------------------ set-up
    def set_material(self, rho0, lam, mu):
        """rho0, lambda, mu: numpy (host) or torch CUDA tensors (device),
        [ny] per row or [ny][nx] per cell (as configured)."""
        torch = self._torch
        arrs = [rho0, lam, mu]
        on_dev = all(isinstance(a, torch.Tensor) and a.is_cuda for a in arrs)
        if on_dev:
            arrs = [a.to(torch.float64).contiguous() for a in arrs]
        else:
            arrs = [np.ascontiguousarray(np.asarray(a if not isinstance(a, torch.Tensor)
                                                    else a.cpu().numpy(), np.float64)) for a in arrs]
        want = self.ny * self.nx if self.cfg.material_per_cell else self.ny
        for a in arrs:
            if (a.numel() if on_dev else a.size) != want:
                raise ValueError(f"material arrays need {want} values")
        st = self.L.lbm_elastic_set_material(self.h, *[_ptr(a) for a in arrs], int(on_dev))
        return self._check(st, allow_warn=True)

    def set_sources(self, sources):
        """sources: array [n][9] = (x, y, sigma, dir_x, dir_y, amplitude,
        f_peak, t0, r_cut)."""
        s = np.asarray(sources, np.float64).reshape(-1, 9)
        self.nsrc = len(s)
        arr = (Source * max(1, len(s)))()
        for k, row in enumerate(s):
            arr[k] = Source(*[float(v) for v in row])
        return self._check(self.L.lbm_elastic_set_sources(self.h, arr, len(s)))

    def set_receivers(self, xy):
        a = np.ascontiguousarray(np.asarray(xy, np.int32).reshape(-1, 2))
        self.nrec = len(a)
        return self._check(self.L.lbm_elastic_set_receivers(self.h, a.ctypes.data if len(a) else None, len(a)))

    def set_sponges(self, sponge, amax: float = 0.0):
        """Replaces the absorbing layers (top, bottom, left, right thickness in
        cells) of the running simulation; the state is kept."""
        t, b, l, r = (int(v) for v in sponge)
        return self._check(self.L.lbm_elastic_set_sponges(self.h, t, b, l, r, float(amax)))

    def reset(self):
        return self._check(self.L.lbm_elastic_reset(self.h))

    # ------------------------------------------------------------ stepping
    def step(self, nsteps: int = 1):
        return self._check(self.L.lbm_elastic_step(self.h, int(nsteps)))

    def set_steps_per_launch(self, steps: int):
        """1, or 2: two time steps per kernel launch (same results bit for
        bit)."""
        return self._check(self.L.lbm_elastic_set_steps_per_launch(self.h, int(steps)))

    @property
    def step_index(self) -> int:
        return self.L.lbm_elastic_step_index(self.h)

    @property
    def kernel_launches(self) -> int:
        return self.L.lbm_elastic_kernel_launches(self.h)

    def sync(self):
        return self._check(self.L.lbm_elastic_sync(self.h))

    # ------------------------------------------------------------ outputs
    FIELD_NAMES = ("ux", "uy", "vx", "vy", "rho", "pxx", "pxy", "pyy")

    def read_fields(self, names: Sequence[str] = FIELD_NAMES, on_device: bool = True) -> Dict:
        torch = self._torch
        out = {}
        ptrs = []
        for k in self.FIELD_NAMES:
            if k in names:
                if on_device:
                    t = torch.empty((self.ny, self.nx), dtype=torch.float64, device=self.device)
                else:
                    t = np.empty((self.ny, self.nx), np.float64)
                out[k] = t
                ptrs.append(_ptr(t))
            else:
                ptrs.append(None)
        self._check(self.L.lbm_elastic_read_fields(self.h, *ptrs, int(on_device)))
        return out

    def traces_recorded(self) -> int:
        return self.L.lbm_elastic_traces_recorded(self.h)

    def read_traces(self, on_device: bool = False, out=None):
        T = self.traces_recorded()
        R = getattr(self, "nrec", 0)
        if out is None:
            if on_device:
                out = self._torch.empty((T, R, 4), dtype=self._torch.float64, device=self.device)
            else:
                out = np.empty((T, R, 4), np.float64)
        self._check(self.L.lbm_elastic_read_traces(self.h, _ptr(out) if T * R else None, int(on_device)))
        return out

    def set_state(self, f9, u2=None, step: int = 0):
        torch = self._torch
        on_dev = isinstance(f9, torch.Tensor) and f9.is_cuda
        if on_dev:
            f9 = f9.to(torch.float64).contiguous()
            u2 = None if u2 is None else u2.to(torch.float64).contiguous()
        else:
            f9 = np.ascontiguousarray(np.asarray(f9, np.float64))
            u2 = None if u2 is None else np.ascontiguousarray(np.asarray(u2, np.float64))
        n = self.nx * self.ny
        if (f9.numel() if on_dev else f9.size) != 9 * n:
            raise ValueError("f9 must hold 9*ny*nx values")
        if u2 is not None and (u2.numel() if on_dev else u2.size) != 2 * n:
            raise ValueError("u2 must hold 2*ny*nx values")
        return self._check(self.L.lbm_elastic_set_state(self.h, _ptr(f9), _ptr(u2), int(step),
                                                        int(on_dev)))

    def get_state(self, on_device: bool = False):
        shape9, shape2 = (9, self.ny, self.nx), (2, self.ny, self.nx)
        if on_device:
            torch = self._torch
            f9 = torch.empty(shape9, dtype=torch.float64, device=self.device)
            u2 = torch.empty(shape2, dtype=torch.float64, device=self.device)
        else:
            f9, u2 = np.empty(shape9), np.empty(shape2)
        self._check(self.L.lbm_elastic_get_state(self.h, _ptr(f9), _ptr(u2), int(on_device)))
        return f9, u2

    def checkpoint_bytes(self) -> int:
        return self.L.lbm_elastic_checkpoint_bytes(self.h)

    def save(self, on_device: bool = True):
        n = self.checkpoint_bytes()
        if on_device:
            buf = self._torch.empty(n, dtype=self._torch.uint8, device=self.device)
        else:
            buf = np.empty(n, np.uint8)
        self._check(self.L.lbm_elastic_save(self.h, _ptr(buf), int(on_device)))
        return buf

    def load(self, buf):
        on_dev = not isinstance(buf, np.ndarray)
        return self._check(self.L.lbm_elastic_load(self.h, _ptr(buf), int(on_dev)))

    def moment_sums(self) -> np.ndarray:
        out = (ctypes.c_double * 7)()
        self._check(self.L.lbm_elastic_moment_sums(self.h, out))
        return np.array(out[:])


class Batch:
    """Many ElasticLBM shots advanced together (one launch per step over the
    tiles of every shot, or one persistent launch for many steps).

    The shots keep their own state; after ``step`` each shot's fields, traces
    and step index are read through the shot as usual.  All work runs on
    ``stream`` (default: torch's current stream)."""

    def __init__(self, shots: Sequence["ElasticLBM"], stream=None):
        import torch
        self._torch = torch
        self.L = load_library()
        self.shots = list(shots)
        if not self.shots:
            raise LBMError(-1, "a batch needs at least one shot")
        dev = self.shots[0].device
        arr = (ctypes.c_void_p * len(self.shots))(*[s.h.value for s in self.shots])
        self._arr = arr
        nbytes = self.L.lbm_batch_workspace_bytes(arr, len(self.shots))
        if nbytes == 0:
            raise LBMError(-1, "invalid shots")
        with torch.cuda.device(dev):
            self.stream = stream if stream is not None else torch.cuda.current_stream(dev)
            self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=dev)
        base = self.workspace.data_ptr()
        off = (-base) % 256
        h = ctypes.c_void_p()
        st = self.L.lbm_batch_create(arr, len(self.shots), base + off, nbytes,
                                     self.stream.cuda_stream, ctypes.byref(h))
        if st != LBM_OK:
            raise LBMError(st, self.L.lbm_batch_last_error(None).decode())
        self.h = h

    def _check(self, st):
        if st == LBM_OK:
            return st
        msg = self.L.lbm_batch_last_error(self.h).decode()
        if st == -5:
            raise NonFiniteError(st, msg)
        raise LBMError(st, msg)

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self.L.lbm_batch_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def launch(self) -> Dict:
        l = BatchLaunch()
        self._check(self.L.lbm_batch_get_launch(self.h, ctypes.byref(l)))
        inv = {v: k for k, v in BATCH_MODE.items()}
        return {"mode": inv[l.mode], "rows": l.rows, "order": l.order,
                "graph_steps": l.graph_steps, "steps_per_launch": l.steps_per_launch,
                "ctas_per_sm": l.ctas_per_sm, "barrier_cycles": l.barrier_cycles,
                "barrier_extra": l.barrier_extra, "steps_per_tile": l.steps_per_tile}

    def set_launch(self, **kw):
        cur = self.launch
        cur.update(kw)
        l = BatchLaunch(BATCH_MODE[cur["mode"]], int(cur["rows"]), int(cur["order"]),
                        int(cur["graph_steps"]), int(cur["steps_per_launch"]),
                        int(cur["ctas_per_sm"]), int(cur["barrier_cycles"]),
                        int(cur["barrier_extra"]), int(cur["steps_per_tile"]))
        self._check(self.L.lbm_batch_set_launch(self.h, ctypes.byref(l)))

    def autotune(self, steps_per_trial: int = 3) -> float:
        """Times every launch candidate on the batch itself (this advances
        the shots) and keeps the fastest; returns its microseconds per step."""
        us = ctypes.c_double()
        self._check(self.L.lbm_batch_autotune(self.h, int(steps_per_trial), ctypes.byref(us)))
        return us.value

    def step(self, nsteps: int = 1):
        self._check(self.L.lbm_batch_step(self.h, int(nsteps)))

    def sync(self):
        self._check(self.L.lbm_batch_sync(self.h))

    @property
    def kernel_launches(self) -> int:
        return int(self.L.lbm_batch_kernel_launches(self.h))

    @property
    def cells(self) -> int:
        return int(self.L.lbm_batch_cells(self.h))


class Adjoint:
    """Reverse-mode gradients of a function of the receiver traces of one
    ElasticLBM (FP32 or FP64 storage): ``forward`` runs ``nsteps`` steps
    from the simulation's current state with a checkpoint every
    ``checkpoint_every`` steps and returns the traces it recorded;
    ``backward(dtraces)`` runs the adjoint for the trace derivatives;
    ``gradients`` returns dJ/dlambda, dJ/dmu, dJ/dLambda per cell and dJ/d
    amplitude per source.  Arrays are torch CUDA tensors (FP64)."""

    def __init__(self, sim: "ElasticLBM", nsteps: int, checkpoint_every: int = 100):
        import torch
        self._torch = torch
        self.sim = sim
        self.L = sim.L
        self.nsteps = int(nsteps)
        nbytes = self.L.lbm_adjoint_workspace_bytes(sim.h, self.nsteps, int(checkpoint_every))
        if nbytes == 0:
            raise LBMError(-1, "invalid adjoint arguments")
        with torch.cuda.device(sim.device):
            self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=sim.device)
        base = self.workspace.data_ptr()
        off = (-base) % 256
        h = ctypes.c_void_p()
        st = self.L.lbm_adjoint_create(sim.h, self.nsteps, int(checkpoint_every), base + off,
                                       nbytes, ctypes.byref(h))
        if st != LBM_OK:
            raise LBMError(st, self.L.lbm_adjoint_last_error(None).decode())
        self.h = h
        self.traced_start = 0

    def _check(self, st):
        if st != LBM_OK:
            raise LBMError(st, self.L.lbm_adjoint_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self.L.lbm_adjoint_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def forward(self):
        """Runs the forward steps; returns the traces they recorded
        ([nsteps][nrec][4] FP64 CUDA tensor, or None without receivers)."""
        self.traced_start = self.sim.traces_recorded()
        self._check(self.L.lbm_adjoint_forward(self.h))
        if self.sim.traces_recorded() == 0:
            return None
        tr = self.sim.read_traces(on_device=True)
        return tr[self.traced_start:self.traced_start + self.nsteps]

    def backward(self, dtraces=None):
        p = None
        if dtraces is not None:
            dtraces = dtraces.to(dtype=self._torch.float64).contiguous()
            p = dtraces.data_ptr()
        self._keep = dtraces
        self._check(self.L.lbm_adjoint_backward(self.h, p))

    def gradients(self) -> Dict:
        t = self._torch
        ny, nx = self.sim.ny, self.sim.nx
        dev = self.sim.device
        g = {k: t.zeros((ny, nx), dtype=t.float64, device=dev)
             for k in ("lambda", "mu", "Lambda")}
        nsrc = self.sim.nsrc
        g["amplitude"] = t.zeros(max(nsrc, 1), dtype=t.float64, device=dev)
        self._check(self.L.lbm_adjoint_gradients(self.h, g["lambda"].data_ptr(),
                                                 g["mu"].data_ptr(), g["Lambda"].data_ptr(),
                                                 g["amplitude"].data_ptr()))
        g["amplitude"] = g["amplitude"][:nsrc]
        return g

    def set_state(self, abar9, ubar2=None):
        t = self._torch
        a = abar9.to(dtype=t.float64).contiguous()
        u = None if ubar2 is None else ubar2.to(dtype=t.float64).contiguous()
        self._check(self.L.lbm_adjoint_set_state(self.h, a.data_ptr(),
                                                 None if u is None else u.data_ptr()))
        self.sim.sync()

    def get_state(self):
        t = self._torch
        ny, nx = self.sim.ny, self.sim.nx
        a = t.empty((9, ny, nx), dtype=t.float64, device=self.sim.device)
        u = t.empty((2, ny, nx), dtype=t.float64, device=self.sim.device)
        self._check(self.L.lbm_adjoint_get_state(self.h, a.data_ptr(), u.data_ptr()))
        return a, u

    def step_linear(self):
        self._check(self.L.lbm_adjoint_step_linear(self.h))

    def set_fused(self, fused: bool):
        """True (default): one fused kernel per adjoint step; False: three."""
        self._check(self.L.lbm_adjoint_set_fused(self.h, int(bool(fused))))

    @property
    def kernel_launches(self) -> int:
        return int(self.L.lbm_adjoint_kernel_launches(self.h))


def moment_sums_noalloc(f9, u2, storage="f64", u_fp64=False, nx=None, out=None,
                        stream=None):
    """Moment sums of caller-held CUDA tensors without a workspace (see
    ``lbm_elastic_moment_sums_noalloc``): f9 [9][ny][pitch], u2 [2][ny][pitch],
    the first ``nx`` (default: pitch) cells of each row summed.  With ``out``
    None the seven sums come back as a numpy array; with a CUDA float64 tensor
    of 7 elements they are written there asynchronously."""
    import torch
    L = load_library()
    ny, pitch = f9.shape[-2], f9.shape[-1]
    nx = pitch if nx is None else int(nx)
    s = (stream if stream is not None else torch.cuda.current_stream()).cuda_stream
    on_dev = out is not None
    host = (ctypes.c_double * 7)()
    st = L.lbm_elastic_moment_sums_noalloc(
        f9.data_ptr(), u2.data_ptr(), STORAGE[storage], int(bool(u_fp64)), int(nx), int(ny),
        int(pitch), out.data_ptr() if on_dev else ctypes.addressof(host), int(on_dev), s)
    if st != LBM_OK:
        raise LBMError(st, L.lbm_elastic_last_error(None).decode())
    return out if on_dev else np.array(host[:])


def from_workload(w, storage=None, max_steps_traced=None, u_fp64=False, device=None,
                  stream=None, kernel="auto", store_scale_log2=0) -> ElasticLBM:
    """An ElasticLBM set up from a :class:`workloads.Workload`."""
    sim = ElasticLBM(w.nx, w.ny, storage=storage or w.storage, tau=w.tau, bc=tuple(w.bc),
                     sponge=tuple(w.sponge), sponge_amax=w.sponge_amax,
                     material_per_cell=w.per_cell, max_sources=max(1, len(w.sources)),
                     max_receivers=max(1, len(w.receivers)),
                     max_steps_traced=w.nsteps if max_steps_traced is None else max_steps_traced,
                     u_fp64=u_fp64, fs_order=w.fs_order, kernel=kernel,
                     store_scale_log2=store_scale_log2, device=device, stream=stream)
    if w.rho0 is not None:
        sim.set_material(w.rho0, w.lam, w.mu)
    if len(w.sources):
        sim.set_sources(w.sources)
    if len(w.receivers):
        sim.set_receivers(w.receivers)
    return sim
