"""Writes tests/golden/halfspace_2048x1024_4000.npz: sampled outputs of the CPU
oracle on the full half-space workload (2048 x 1024 cells, free surface on top,
64-cell absorbing layers on the other sides, nu = 0.25, vertical Ricker x
Gaussian force 10 cells below the surface, 256 surface receivers, 4000 steps).

Calls only the oracle and the seeded workload generator.  Stored: the final
displacement and velocity sampled every 16 cells in x and y, and the traces of
every 16th receiver at every 4th step.  Run:  python tests/golden/make_halfspace_golden.py
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2009_06404_gb300 import workloads as wl  # noqa: E402

STRIDE = 16
REC_STRIDE = 16
STEP_STRIDE = 4


def main():
    w = wl.halfspace()
    prob = oracle.Problem(nx=w.nx, ny=w.ny, tau=w.tau, bc_top=w.bc[0], bc_bottom=w.bc[1],
                          bc_left=w.bc[2], bc_right=w.bc[3], sponge=tuple(w.sponge),
                          sponge_amax=w.sponge_amax, fs_order=w.fs_order, rho0=w.rho0, lam=w.lam, mu=w.mu,
                          sources=w.sources, receivers=w.receivers,
                          nthreads=os.cpu_count() or 1)
    t = time.time()
    st, tr = oracle.run(prob, w.nsteps)
    f = oracle.fields(prob, st)
    print(f"oracle: {w.nsteps} steps in {time.time() - t:.1f} s")
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "halfspace_2048x1024_4000.npz")
    np.savez_compressed(
        out,
        u=st.u[:, ::STRIDE, ::STRIDE],
        v=np.stack([f["vx"], f["vy"]])[:, ::STRIDE, ::STRIDE],
        traces=tr[STEP_STRIDE - 1::STEP_STRIDE, ::REC_STRIDE, :],
        stride=STRIDE, rec_stride=REC_STRIDE, step_stride=STEP_STRIDE,
        u_norm=np.linalg.norm(st.u), nsteps=w.nsteps)
    print("wrote", out)


if __name__ == "__main__":
    main()
