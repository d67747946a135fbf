"""Seeded synthetic workloads (inputs only).

This module builds the inputs that both the CUDA library and the CPU oracle are
fed: grid sizes, boundary kinds, absorbing-layer thicknesses, layered
materials (rho0, lambda, mu), Ricker x Gaussian sources, receiver positions and
random population states.  It holds none of the method's arithmetic and imports
neither the CUDA binding nor the oracle.

Materials: on the D2Q9 lattice the S-wave speed is fixed at b = 1/sqrt(3) in
lattice units, so a layer is described by its density rho0 and Poisson ratio
nu; the shear modulus is mu = rho0 / 3 (which makes v_S = 1/sqrt(3)) and
lambda = 2 mu nu / (1 - 2 nu).  Layers can therefore differ only in nu and
rho0.

Source rows are (x, y, sigma, dir_x, dir_y, amplitude, f_peak, t0, r_cut).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace
from typing import List, Sequence

import numpy as np

#: 20 cells per S wavelength at v_S = 1/sqrt(3): f_peak = v_S / 20.
F_PEAK_20 = (1.0 / math.sqrt(3.0)) / 20.0


@dataclass
class Workload:
    name: str
    nx: int
    ny: int
    nsteps: int
    tau: float = 1.0
    storage: str = "f32"                       # f64 | f32 | f16 | bf16
    bc: Sequence[str] = ("periodic",) * 4      # top, bottom, left, right
    sponge: Sequence[int] = (0, 0, 0, 0)       # top, bottom, left, right
    sponge_amax: float = 0.0                   # <= 0: 12.8 / L per layer
    fs_order: int = 0                          # free-surface extrapolation: 0 constant, 1 linear
    rho0: np.ndarray = None                    # per row [ny] or per cell [ny][nx]
    lam: np.ndarray = None
    mu: np.ndarray = None
    sources: np.ndarray = field(default_factory=lambda: np.zeros((0, 9)))
    receivers: np.ndarray = field(default_factory=lambda: np.zeros((0, 2), np.int32))
    seed: int = 0

    @property
    def cells(self) -> int:
        return self.nx * self.ny

    @property
    def per_cell(self) -> bool:
        return self.rho0 is not None and np.asarray(self.rho0).ndim == 2

    def with_(self, **kw) -> "Workload":
        return replace(self, **kw)


def lame(nu, rho0):
    """(lambda, mu) of a layer with density rho0 and Poisson ratio nu, with
    mu = rho0 / 3 (v_S = 1/sqrt(3))."""
    nu = np.asarray(nu, np.float64)
    rho0 = np.asarray(rho0, np.float64)
    mu = rho0 / 3.0
    return 2.0 * mu * nu / (1.0 - 2.0 * nu), mu


def homogeneous(ny: int, nu: float, rho0: float = 1.0):
    r = np.full(ny, float(rho0))
    lam, mu = lame(np.full(ny, nu), r)
    return r, lam, mu


def layered(ny: int, rng: np.random.Generator, nlayers: int, nu_range, rho_range):
    """Horizontally layered medium: interfaces uniform in depth, per-layer nu
    and rho0 uniform in the given ranges.  Returns per-row arrays."""
    cuts = np.sort(rng.integers(1, ny, size=nlayers - 1))
    nus = rng.uniform(*nu_range, size=nlayers)
    rhos = rng.uniform(*rho_range, size=nlayers)
    layer = np.searchsorted(cuts, np.arange(ny), side="right")
    rho0 = rhos[layer]
    lam, mu = lame(nus[layer], rho0)
    return rho0, lam, mu


def source(x, y, sigma=3.0, direction=(1.0, 0.0), amplitude=1.0,
           f_peak=F_PEAK_20, t0=None, r_cut=None):
    if t0 is None:
        t0 = 1.5 / f_peak
    if r_cut is None:
        r_cut = 8.0 * sigma
    return np.array([x, y, sigma, direction[0], direction[1], amplitude,
                     f_peak, t0, r_cut], np.float64)


def ring(cx, cy, radius, n):
    """n receivers on a circle, rounded to the nearest cell (ties upward)."""
    th = 2.0 * np.pi * np.arange(n) / n
    x = np.floor(cx + radius * np.cos(th) + 0.5).astype(np.int32)
    y = np.floor(cy + radius * np.sin(th) + 0.5).astype(np.int32)
    return np.stack([x, y], axis=1)


def surface_line(x0, x1, n, row=0):
    """n receivers on row ``row``, evenly spread over [x0, x1)."""
    x = (x0 + np.floor((np.arange(n) + 0.5) * (x1 - x0) / n)).astype(np.int32)
    return np.stack([x, np.full(n, row, np.int32)], axis=1)


# ------------------------------------------------------------------ configs

def periodic_bulk(n: int = 128, nsteps: int = 500, storage: str = "f64",
                  nu: float = 0.25, tau: float = 1.0) -> Workload:
    """Plain method, FP64: n x n periodic grid, homogeneous Poisson solid,
    +x Gaussian (sigma = 3) x Ricker (20 cells per S wavelength) source at the
    centre, 64-point receiver ring at radius 40 * n / 128."""
    rho0, lam, mu = homogeneous(n, nu)
    c = n // 2
    return Workload(
        name=f"periodic_bulk_{n}x{n}", nx=n, ny=n, nsteps=nsteps, tau=tau,
        storage=storage, rho0=rho0, lam=lam, mu=mu,
        sources=source(c, c)[None],
        receivers=ring(c, c, 40.0 * n / 128.0, 64))


def halfspace(nx: int = 2048, ny: int = 1024, nsteps: int = 4000,
              storage: str = "f32", sponge: int = 64, nrec: int = 256,
              nu: float = 0.25, tau: float = 1.0) -> Workload:
    """Half-space: free surface on the top row, absorbing layers of ``sponge``
    cells on the left, right and bottom (periodic in x and a rigid wall at the
    bottom behind them), homogeneous nu = 0.25, vertical Ricker x Gaussian force
    10 cells below the surface, ``nrec`` receivers on the surface row."""
    rho0, lam, mu = homogeneous(ny, nu)
    return Workload(
        name=f"halfspace_{nx}x{ny}", nx=nx, ny=ny, nsteps=nsteps, tau=tau,
        storage=storage, bc=("free", "rigid", "periodic", "periodic"),
        sponge=(0, sponge, sponge, sponge), rho0=rho0, lam=lam, mu=mu,
        sources=source(nx // 2, 10, direction=(0.0, 1.0))[None],
        receivers=surface_line(sponge, nx - sponge, nrec))


def layered_halfspace(nx: int, ny: int, nsteps: int, seed: int,
                      nlayers=(3, 5), nu_range=(0.2, 0.35), rho_range=(1.0, 3.0),
                      sponge: int = 32, nrec: int = 128, storage: str = "f32",
                      src_x=None, src_y=None) -> Workload:
    """Layered half-space with free top and absorbing layers elsewhere; the
    source position is drawn in the top quarter unless given."""
    rng = np.random.default_rng(seed)
    nl = int(rng.integers(nlayers[0], nlayers[1] + 1))
    rho0, lam, mu = layered(ny, rng, nl, nu_range, rho_range)
    sx = src_x if src_x is not None else float(rng.integers(sponge + 16, nx - sponge - 16))
    sy = src_y if src_y is not None else float(rng.integers(4, max(5, ny // 4)))
    return Workload(
        name=f"layered_{nx}x{ny}_s{seed}", nx=nx, ny=ny, nsteps=nsteps,
        storage=storage, bc=("free", "rigid", "periodic", "periodic"),
        sponge=(0, sponge, sponge, sponge), rho0=rho0, lam=lam, mu=mu,
        sources=source(sx, sy, direction=(0.0, 1.0))[None],
        receivers=surface_line(sponge, nx - sponge, nrec), seed=seed)


def periodic_layered_multisource(n: int = 8192, nsteps: int = 2000, seed: int = 5,
                                 nlayers: int = 8, nu_range=(0.2, 0.36),
                                 nsrc: int = 16, storage: str = "f32") -> Workload:
    """Periodic n x n grid, ``nlayers`` seeded layers, ``nsrc`` Ricker x Gaussian
    sources at seeded positions with random directions."""
    rng = np.random.default_rng(seed)
    rho0, lam, mu = layered(n, rng, nlayers, nu_range, (1.0, 3.0))
    xs = rng.uniform(0, n, size=nsrc)
    ys = rng.uniform(0, n, size=nsrc)
    th = rng.uniform(0, 2 * np.pi, size=nsrc)
    src = np.stack([source(x, y, direction=(math.cos(t), math.sin(t)))
                    for x, y, t in zip(xs, ys, th)])
    return Workload(name=f"periodic_layered_{n}x{n}_s{seed}", nx=n, ny=n,
                    nsteps=nsteps, storage=storage, rho0=rho0, lam=lam, mu=mu,
                    sources=src, seed=seed)


def random_state(nx: int, ny: int, seed: int, scale: float = 1e-3):
    """Smooth-ish random post-collision populations [9][ny][nx] and
    displacement [2][ny][nx] (for parity tests from a non-trivial state)."""
    rng = np.random.default_rng(seed)
    fs = scale * rng.standard_normal((9, ny, nx))
    u = scale * rng.standard_normal((2, ny, nx))
    return fs, u


#: grid sizes of the uneven multi-shot batch, by shot index mod 4
BATCH_SIZES = ((512, 512), (1024, 512), (1536, 768), (2048, 1024))


def batch_shots(nshots: int = 64, nsteps: int = 2000, seed: int = 3, storage: str = "f32",
                sizes=BATCH_SIZES, nrec: int = 64) -> list:
    """The uneven multi-shot batch: shot s has grid size sizes[s % len(sizes)]
    and is a 3-5-layer half-space (rho0 in [1, 3], nu in [0.2, 0.35], seeded
    per shot) with a free top, absorbing layers of 32 cells elsewhere and one
    source in the top quarter."""
    out = []
    for s in range(nshots):
        nx, ny = sizes[s % len(sizes)]
        out.append(layered_halfspace(nx, ny, nsteps, seed=seed * 1000 + s, sponge=32,
                                     nrec=nrec, storage=storage))
    return out


def fwi_blob(nx: int = 1024, ny: int = 512, nsteps: int = 3000, seed: int = 4,
             sigma: float = 25.0, dmu: float = 0.05, dlam: float = -0.05, sponge: int = 64,
             nrec: int = 128, storage: str = "f32"):
    """The inversion set-up: a 4-layer half-space (nu in [0.2, 0.3], seeded)
    with a free top, absorbing layers elsewhere, a vertical source at
    (nx / 2, 10) and nrec receivers on the surface row, and the same model
    with a Gaussian blob (width sigma, centre seeded in the interior) scaling
    mu by (1 + dmu) and lambda by (1 + dlam) at its peak.  Returns
    (base, perturbed) workloads with per-cell material."""
    rng = np.random.default_rng(seed)
    base = layered_halfspace(nx, ny, nsteps, seed=seed, nlayers=(4, 4), nu_range=(0.2, 0.3),
                             sponge=sponge, nrec=nrec, storage=storage, src_x=nx / 2,
                             src_y=10.0)
    cells = lambda a: np.repeat(np.asarray(a, np.float64)[:, None], nx, axis=1)
    rho0, lam, mu = cells(base.rho0), cells(base.lam), cells(base.mu)
    cx = rng.uniform(sponge + 2 * sigma, nx - sponge - 2 * sigma)
    cy = rng.uniform(2 * sigma, ny - sponge - 2 * sigma)
    Y, X = np.mgrid[0:ny, 0:nx]
    g = np.exp(-((X - cx) ** 2 + (Y - cy) ** 2) / (2 * sigma * sigma))
    base = base.with_(rho0=rho0, lam=lam, mu=mu, name=f"fwi_base_{nx}x{ny}")
    pert = base.with_(lam=lam * (1 + dlam * g), mu=mu * (1 + dmu * g),
                      name=f"fwi_blob_{nx}x{ny}")
    return base, pert


#: step after which the surface-wave experiment removes its lateral layers
RAYLEIGH_SWITCH_STEP = 400


def rayleigh_laps(nx: int = 300, ny: int = 100, nsteps: int = 2200, tau: float = 0.55,
                  sponge: int = 30, fs_order: int = 0, storage: str = "f64") -> Workload:
    """The paper's surface-wave experiment (Sec. 7): a Poisson solid on an
    nx-long, ny-deep grid with a free top, absorbing layers of `sponge` cells
    on the left, right and bottom (periodic lateral edges behind the lateral
    layers, rigid bottom), a vertical source (sigma = 4, period 20) near the
    upper left corner and a receiver on every surface cell.  After
    RAYLEIGH_SWITCH_STEP steps the lateral layers are to be removed
    (ElasticLBM.set_sponges), leaving the surface wave free to go round."""
    rho0, lam, mu = homogeneous(ny, 0.25)
    src = source(sponge + 15.0, 4.0, sigma=4.0, direction=(0.0, 1.0), f_peak=1.0 / 20.0,
                 t0=30.0, r_cut=32.0)
    rec = np.array([[x, 0] for x in range(nx)], np.int32)
    return Workload(name=f"rayleigh_laps_{nx}x{ny}", nx=nx, ny=ny, nsteps=nsteps, tau=tau,
                    storage=storage, bc=("free", "rigid", "periodic", "periodic"),
                    sponge=(0, sponge, sponge, sponge), fs_order=fs_order, rho0=rho0, lam=lam,
                    mu=mu, sources=src[None], receivers=rec)
