"""Full-size checks of two workloads against the FP64 references they rest on.

* The inversion set-up (1024 x 512 layered half-space with a Gaussian blob
  on mu and lambda, one Ricker source, 128 surface receivers, 3000 steps,
  checkpoints every 100 steps): the gradients of the displacement-trace
  misfit with respect to lambda and mu at 16 seeded cells, and with respect
  to the source amplitude, from the autograd Function (reverse-time adjoint)
  against central differences of the FP64 forward run.  FP64 states to
  1e-4 at every cell; FP32 states with FP64 gradient sums, the data
  modelled in FP32 too, to 1e-3 over the 16 cells (1e-2 for the amplitude).  Lambda and mu enter the
  step only through Lambda = (mu - lambda)/(rho0 b^2) (Eq. 32), so the two
  gradients are each other's negatives.
* The FP64 GPU run of the 8-layer, 16-source periodic grid at 1024 x 1024
  for 2000 steps (the reference the 16-bit and FP32 storage errors are
  measured against) equals the CPU oracle's run to 1e-12 (relative L2).
"""
import numpy as np
import pytest

import oracle
from helpers import oracle_problem, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _library():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2009_06404_gb300 import build
    build.build()


def _fd_cells(nx, ny, sponge, n=16, seed=44):
    """n seeded cells outside the absorbing layers, the surface row included."""
    rng = np.random.default_rng(seed)
    return [(int(rng.integers(sponge, nx - sponge)), int(rng.integers(0, ny - sponge)))
            for _ in range(n)]


def test_inversion_gradients_match_central_differences():
    from paper_2009_06404_gb300 import workloads as wl
    from paper_2009_06404_gb300.autograd import SimulationSetup, simulate_traces
    base, pert = wl.fwi_blob(1024, 512, 3000)
    K, dev = 100, "cuda"
    amp0 = torch.tensor(base.sources[:, 5], dtype=torch.float64, device=dev)
    lam_b = torch.as_tensor(base.lam, device=dev)
    mu_b = torch.as_tensor(base.mu, device=dev)
    lam0 = np.asarray(pert.lam, np.float64)
    setups = {s: SimulationSetup(pert, 3000, K, s) for s in ("f64", "f32")}
    # the data: traces of the model without the blob, in each precision (FP32
    # states against FP64 data would leave the FP32 error of the direct
    # surface wave in the residual, which then dominates the gradient in the
    # top rows)
    data = {}
    with torch.no_grad():
        for s in ("f64", "f32"):
            data[s] = simulate_traces(lam_b, mu_b, amp0, setups[s])[..., :2].clone()

    def J(lam, mu, amp, storage="f64"):
        tr = simulate_traces(lam, mu, amp, setups[storage])
        return 0.5 * ((tr[..., :2] - data[storage]) ** 2).sum()

    grads = {}
    for storage in ("f64", "f32"):
        lam = torch.as_tensor(pert.lam, device=dev).clone().requires_grad_(True)
        mu = torch.as_tensor(pert.mu, device=dev).clone().requires_grad_(True)
        amp = amp0.clone().requires_grad_(True)
        Jv = J(lam, mu, amp, storage)
        Jv.backward()
        grads[storage] = (lam.grad.cpu().numpy(), mu.grad.cpu().numpy(),
                          amp.grad.cpu().numpy(), float(Jv.detach()))
    gl64, gm64, ga64, J64 = grads["f64"]
    gl32, gm32, ga32, _ = grads["f32"]
    assert J64 > 0
    # lambda and mu enter only through Lambda (Eq. 32)
    np.testing.assert_allclose(gm64, -gl64, rtol=1e-12, atol=0)

    lam_t = torch.as_tensor(pert.lam, device=dev)
    mu_t = torch.as_tensor(pert.mu, device=dev)
    cells = _fd_cells(1024, 512, 64)
    fd = []
    with torch.no_grad():
        for (x, y) in cells:
            h = 1e-4 * lam0[y, x]
            lp = lam_t.clone()
            lm = lam_t.clone()
            lp[y, x] += h
            lm[y, x] -= h
            fd.append((float(J(lp, mu_t, amp0)) - float(J(lm, mu_t, amp0))) / (2 * h))
    fd = np.array(fd)
    g64 = np.array([gl64[y, x] for (x, y) in cells])
    g32 = np.array([gl32[y, x] for (x, y) in cells])
    big = np.abs(fd).max()
    assert big > 0
    # FP64 states: each cell within 1e-4 of its difference quotient (plus the
    # quotient's own round-off, ~1e-15 J / h)
    for k, (x, y) in enumerate(cells):
        h = 1e-4 * lam0[y, x]
        assert abs(g64[k] - fd[k]) <= 1e-4 * abs(fd[k]) + 1e-13 * J64 / h, ((x, y), g64[k], fd[k])
    # FP32 states, FP64 sums: within 1e-3 over the 16 cells
    assert np.linalg.norm(g32 - fd) <= 1e-3 * np.linalg.norm(fd), (g32, fd)
    # the misfit is quadratic in the amplitude: central differences are exact
    h = 1e-3
    with torch.no_grad():
        fda = (float(J(lam_t, mu_t, amp0 + h)) - float(J(lam_t, mu_t, amp0 - h))) / (2 * h)
    assert abs(ga64[0] - fda) <= 1e-6 * abs(fda), (ga64, fda)
    # FP32: the residual (2e-4 of the traces) carries the FP32 rounding of the
    # direct wave, about 0.2 % of it even with data modelled in FP32, and the
    # amplitude gradient weighs the whole residual with the direct wave
    assert abs(ga32[0] - fda) <= 1e-2 * abs(fda), (ga32, fda)


def test_fp64_precision_reference_matches_oracle():
    import paper_2009_06404_gb300 as pkg
    from paper_2009_06404_gb300 import workloads as wl
    w = wl.periodic_layered_multisource(n=1024, nsteps=2000, seed=5)
    sim = pkg.from_workload(w, storage="f64", max_steps_traced=0)
    sim.step(w.nsteps)
    f = sim.read_fields(("ux", "uy", "vx", "vy"), on_device=False)
    sim.close()
    prob = oracle_problem(w)
    st, _ = oracle.run(prob, w.nsteps, traces=False)
    fo = oracle.fields(prob, st)
    u = np.stack([f["ux"], f["uy"]])
    v = np.stack([f["vx"], f["vy"]])
    assert np.linalg.norm(st.u) > 0
    assert rel_l2(u, st.u) <= 1e-12
    assert rel_l2(v, np.stack([fo["vx"], fo["vy"]])) <= 1e-12
