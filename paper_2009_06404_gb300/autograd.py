"""Receiver traces as a differentiable function of the material and the
source amplitudes, for full-waveform inversion.

``simulate_traces(lam, mu, amp, setup)`` runs ``setup.nsteps`` steps of a
fresh simulation with per-cell Lame parameters ``lam``, ``mu`` ([ny][nx]
CUDA tensors) and source amplitudes ``amp`` ([nsrc]) and returns the traces
[nsteps][nrec][4] (u_x, u_y after each step, v_x, v_y of the step).  Its
backward pass is the library's reverse-time adjoint (checkpoints every
``setup.checkpoint_every`` steps, each segment recomputed), not autograd
through the steps: the gradients are those of the discrete step, with rho0
held fixed.
"""
from __future__ import annotations

import numpy as np
import torch

from .binding import Adjoint, ElasticLBM


class SimulationSetup:
    """Everything except the differentiated parameters: grid, boundaries,
    absorbing layers, rho0, source positions and shapes, receivers, the
    number of steps, the checkpoint interval and the storage type (f32 or
    f64)."""

    def __init__(self, workload, nsteps=None, checkpoint_every: int = 100, storage="f32"):
        self.w = workload
        self.nsteps = int(nsteps if nsteps is not None else workload.nsteps)
        self.checkpoint_every = int(checkpoint_every)
        self.storage = storage
        rho0 = np.asarray(workload.rho0, np.float64)
        if rho0.ndim == 1:
            rho0 = np.repeat(rho0[:, None], workload.nx, axis=1)
        self.rho0 = rho0

    def make(self, lam: torch.Tensor, mu: torch.Tensor, amp: torch.Tensor) -> ElasticLBM:
        w = self.w
        sim = ElasticLBM(w.nx, w.ny, storage=self.storage, tau=w.tau, bc=tuple(w.bc),
                         sponge=tuple(w.sponge), sponge_amax=w.sponge_amax,
                         material_per_cell=True, max_sources=max(1, len(w.sources)),
                         max_receivers=max(1, len(w.receivers)), max_steps_traced=self.nsteps,
                         fs_order=w.fs_order, device=lam.device)
        rho0 = torch.as_tensor(self.rho0, dtype=torch.float64, device=lam.device)
        sim.set_material(rho0, lam.detach().to(torch.float64).contiguous(),
                         mu.detach().to(torch.float64).contiguous())
        if len(w.sources):
            src = np.array(w.sources, np.float64, copy=True)
            src[:, 5] = amp.detach().cpu().numpy()
            sim.set_sources(src)
        if len(w.receivers):
            sim.set_receivers(w.receivers)
        return sim


class TraceSimulation(torch.autograd.Function):
    @staticmethod
    def forward(ctx, lam, mu, amp, setup):
        sim = setup.make(lam, mu, amp)
        adj = Adjoint(sim, setup.nsteps, setup.checkpoint_every)
        tr = adj.forward()
        ctx.adj = adj
        return tr.clone()

    @staticmethod
    def backward(ctx, gtr):
        adj = ctx.adj
        adj.backward(gtr.contiguous())
        g = adj.gradients()
        return g["lambda"], g["mu"], g["amplitude"], None


def simulate_traces(lam: torch.Tensor, mu: torch.Tensor, amp: torch.Tensor,
                    setup: SimulationSetup) -> torch.Tensor:
    return TraceSimulation.apply(lam, mu, amp, setup)
