"""The reverse-time adjoint of the CUDA library.

* Transpose test: for one step L of the linear part (no sources),
  <L x, y> = <x, L^T y> for random states x = (f*, u) and adjoints
  y = (a, ubar), on every boundary kind, ragged grids, absorbing layers and
  per-cell Lambda != 0, FP64 to 1e-13 and FP32 to 1e-5 (relative to the
  products' magnitude).
* Gradients against the oracle's brute-force discrete adjoint on a tiny
  grid (FP64, through checkpoints and recomputation).
* The autograd Function against central finite differences of the FP64
  forward on a layered half-space with a Gaussian blob on mu and lambda.
"""
import numpy as np
import pytest

import oracle
from oracle import adjoint as oadj
from helpers import oracle_problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

B2 = 1.0 / 3.0


@pytest.fixture(scope="module", autouse=True)
def _library():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2009_06404_gb300 import build
    build.build()


def _pkg():
    import paper_2009_06404_gb300 as pkg
    return pkg


def _wl():
    from paper_2009_06404_gb300 import workloads
    return workloads


BCS = {
    "periodic": (("periodic",) * 4, (0, 0, 0, 0)),
    "free_top_rigid_bottom": (("free", "rigid", "periodic", "periodic"), (0, 3, 0, 0)),
    "free_box": (("free", "free", "free", "free"), (2, 0, 3, 0)),
    "rigid_box": (("rigid", "rigid", "rigid", "rigid"), (0, 0, 0, 2)),
    "free_tb_rigid_lr": (("free", "free", "rigid", "rigid"), (0, 2, 2, 0)),
    "rigid_tb_free_lr": (("rigid", "rigid", "free", "free"), (0, 0, 0, 0)),
}


def _material(nx, ny, seed, nu_lo=0.2, nu_hi=0.32):
    rng = np.random.default_rng(seed)
    rho0 = rng.uniform(1.0, 2.0, size=(ny, nx))
    nu = rng.uniform(nu_lo, nu_hi, size=(ny, nx))
    mu = rho0 * B2
    lam = 2 * nu * mu / (1 - 2 * nu)
    return rho0, lam, mu


def _sim(nx, ny, storage, bc, sponge, fs_order, seed, tau=0.8, **kw):
    pkg = _pkg()
    sim = pkg.ElasticLBM(nx, ny, storage=storage, tau=tau, bc=bc, sponge=sponge,
                         material_per_cell=True, fs_order=fs_order, **kw)
    rho0, lam, mu = _material(nx, ny, seed)
    sim.set_material(rho0, lam, mu)
    return sim, (rho0, lam, mu)


@pytest.mark.parametrize("fused", [True, False])
@pytest.mark.parametrize("storage,tol", [("f64", 1e-13), ("f32", 2e-5)])
@pytest.mark.parametrize("bcname", sorted(BCS))
@pytest.mark.parametrize("nx,ny", [(13, 7), (70, 45)])
@pytest.mark.parametrize("fs_order", [0, 1])
def test_adjoint_step_is_the_transpose(storage, tol, bcname, nx, ny, fs_order, fused):
    bc, sponge = BCS[bcname]
    if fs_order == 1 and "free" not in bc:
        pytest.skip("extrapolation order only matters at a free surface")
    sim, _ = _sim(nx, ny, storage, bc, sponge, fs_order, seed=nx * 7 + ny)
    adj = _pkg().Adjoint(sim, 1, 1)
    adj.set_fused(fused)
    g = torch.Generator(device="cpu").manual_seed(nx + 100 * ny + fs_order)
    f = torch.randn((9, ny, nx), generator=g, dtype=torch.float64).cuda()
    u = torch.randn((2, ny, nx), generator=g, dtype=torch.float64).cuda()
    a = torch.randn((9, ny, nx), generator=g, dtype=torch.float64).cuda()
    ub = torch.randn((2, ny, nx), generator=g, dtype=torch.float64).cuda()
    if storage == "f32":  # exactly representable inputs
        f, u, a, ub = [t.float().double() for t in (f, u, a, ub)]
    sim.set_state(f, u, step=0)
    sim.step(1)
    f1, u1 = sim.get_state(on_device=True)
    adj.set_state(a, ub)
    adj.step_linear()
    a0, ub0 = adj.get_state()
    lhs = float((f1 * a).sum() + (u1 * ub).sum())
    rhs = float((f * a0).sum() + (u * ub0).sum())
    scale = float((f1.abs() * a.abs()).sum() + (u1.abs() * ub.abs()).sum())
    assert abs(lhs - rhs) <= tol * scale, (lhs, rhs, scale)
    assert torch.equal(ub0, ub)


def _tiny_workload(fs_order, bc, sponge, seed=7):
    wl = _wl()
    nx, ny = 9, 8
    rho0, lam, mu = _material(nx, ny, seed)
    src = np.array([[3.2, 2.1, 1.0, 0.6, 0.8, 1.0, 0.3, 2.0, 3.0],
                    [6.0, 5.0, 0.8, 1.0, 0.0, 0.7, 0.25, 3.0, 2.0]])
    rec = np.array([[0, 0], [4, 1], [8, 7], [2, 5]], np.int32)
    return wl.Workload(name="tiny", nx=nx, ny=ny, nsteps=12, tau=0.8, storage="f64", bc=bc,
                       sponge=sponge, fs_order=fs_order, rho0=rho0, lam=lam, mu=mu,
                       sources=src, receivers=rec)


@pytest.mark.parametrize("fused", [True, False])
@pytest.mark.parametrize("fs_order,bc,sponge", [
    (1, ("free", "rigid", "periodic", "periodic"), (0, 2, 0, 0)),
    (0, ("free", "free", "rigid", "rigid"), (0, 0, 2, 0)),
    (1, ("free", "free", "free", "free"), (0, 0, 0, 2)),
    (0, ("periodic",) * 4, (0, 0, 0, 0)),
])
def test_gradients_match_oracle_discrete_adjoint(fs_order, bc, sponge, fused):
    """dJ/dLambda per cell and dJ/dA per source for a misfit against noisy
    data, 12 steps with a checkpoint every 5 (FP64): the CUDA adjoint equals
    the oracle's brute-force reverse mode to 1e-10."""
    w = _tiny_workload(fs_order, bc, sponge)
    T = w.nsteps
    prob = oracle_problem(w)
    _, tr = oracle.run(prob, T)
    data = tr + 0.3 * np.abs(tr).max() * np.random.default_rng(3).standard_normal(tr.shape)
    gL_ref, gA_ref = oadj.gradients(prob, T, oadj.misfit_trace_adjoint(tr, data))
    pkg = _pkg()
    sim = pkg.from_workload(w, storage="f64", max_steps_traced=T)
    adj = pkg.Adjoint(sim, T, 5)
    adj.set_fused(fused)
    trg = adj.forward()
    assert np.allclose(trg.cpu().numpy(), tr, rtol=0, atol=1e-12 * np.abs(tr).max())
    adj.backward(torch.as_tensor(oadj.misfit_trace_adjoint(tr, data), device="cuda"))
    g = adj.gradients()
    gL = g["Lambda"].cpu().numpy()
    assert np.abs(gL - gL_ref).max() <= 1e-10 * np.abs(gL_ref).max()
    gA = g["amplitude"].cpu().numpy()
    assert np.abs(gA - gA_ref).max() <= 1e-10 * np.abs(gA_ref).max()
    gl, gm = oadj.lambda_gradients(prob, gL_ref)
    assert np.allclose(g["lambda"].cpu().numpy(), gl, rtol=1e-9, atol=1e-10 * np.abs(gl).max())
    assert np.allclose(g["mu"].cpu().numpy(), gm, rtol=1e-9, atol=1e-10 * np.abs(gm).max())
    # the handle is back where the forward run left it
    f = sim.read_fields(("ux",), on_device=False)
    st, _ = oracle.run(prob, T)
    assert np.allclose(f["ux"], st.u[0], rtol=0, atol=1e-12 * np.abs(st.u).max())


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_fused_adjoint_equals_three_kernel_form(storage):
    """The fused adjoint step and the three-kernel form compute the same
    transpose: identical dJ/dLambda and amplitude gradients (up to the order of
    the amplitude's atomic sums) on a ragged layered half-space with sources
    and receivers near the edges, through checkpoints."""
    wl = _wl()
    w = wl.layered_halfspace(70, 45, 60, seed=21, sponge=6, nrec=9, storage=storage,
                             src_x=30.0, src_y=3.0)
    w = w.with_(fs_order=1)
    out = {}
    for fused in (True, False):
        sim = _pkg().from_workload(w, storage=storage, max_steps_traced=60)
        adj = _pkg().Adjoint(sim, 60, 16)
        adj.set_fused(fused)
        tr = adj.forward()
        d = tr.clone()
        d[..., :2] -= 0.1 * tr[..., :2].abs().max()
        adj.backward(tr - d)
        g = adj.gradients()
        out[fused] = (g["Lambda"].cpu().numpy(), g["amplitude"].cpu().numpy())
    assert np.array_equal(out[True][0], out[False][0])
    assert np.allclose(out[True][1], out[False][1], rtol=1e-12, atol=0)
    assert np.abs(out[True][0]).max() > 0


def test_backward_twice_is_reproducible():
    """The first reverse sweep reuses the density gradients the forward run
    stored for its last segment; the second recomputes every segment.  Both
    give the same gradients bit for bit, and K = T (no recomputation at all)
    gives them too."""
    wl = _wl()
    w = wl.layered_halfspace(70, 45, 48, seed=22, sponge=6, nrec=9, storage="f32",
                             src_x=30.0, src_y=3.0)
    res = []
    for K in (16, 48):
        sim = _pkg().from_workload(w, storage="f32", max_steps_traced=48)
        adj = _pkg().Adjoint(sim, 48, K)
        tr = adj.forward()
        dtr = tr * 0.5
        for _ in range(2):
            adj.backward(dtr)
            res.append(adj.gradients()["Lambda"].cpu().numpy())
    assert all(np.array_equal(res[0], r) for r in res[1:])
    assert np.abs(res[0]).max() > 0


def _blob_setup(nx, ny, nsteps, storage, K):
    """Layered half-space with a Gaussian blob (+5 % on mu, -5 % on lambda)."""
    wl = _wl()
    w = wl.layered_halfspace(nx, ny, nsteps, seed=4, nlayers=(4, 4), nu_range=(0.2, 0.3),
                             sponge=16, nrec=16, storage=storage, src_x=nx / 2, src_y=6.0)
    rho0 = np.repeat(np.asarray(w.rho0)[:, None], nx, 1)
    lam = np.repeat(np.asarray(w.lam)[:, None], nx, 1)
    mu = np.repeat(np.asarray(w.mu)[:, None], nx, 1)
    Y, X = np.mgrid[0:ny, 0:nx]
    blob = np.exp(-((X - 0.45 * nx) ** 2 + (Y - 0.4 * ny) ** 2) / (2 * (0.08 * nx) ** 2))
    w = w.with_(rho0=rho0, lam=lam, mu=mu)
    from paper_2009_06404_gb300.autograd import SimulationSetup
    return SimulationSetup(w, nsteps, K, storage), lam, mu, blob


def test_autograd_function_matches_finite_differences():
    """Misfit of the traces of the blob model against those of the layered
    model; the autograd gradient (FP64 states) at 6 seeded cells and for the
    amplitude equals central differences of the FP64 forward."""
    from paper_2009_06404_gb300.autograd import simulate_traces
    nx, ny, T = 96, 64, 160
    setup, lam0, mu0, blob = _blob_setup(nx, ny, T, "f64", 40)
    dev = "cuda"
    amp = torch.tensor([1.0], dtype=torch.float64, device=dev)
    L0 = torch.as_tensor(lam0, device=dev)
    M0 = torch.as_tensor(mu0, device=dev)
    with torch.no_grad():
        d = simulate_traces(L0, M0, amp, setup)
    lam = torch.as_tensor(lam0 * (1 - 0.05 * blob), device=dev).requires_grad_(True)
    mu = torch.as_tensor(mu0 * (1 + 0.05 * blob), device=dev).requires_grad_(True)
    a = amp.clone().requires_grad_(True)

    def J(l, m, am):
        tr = simulate_traces(l, m, am, setup)
        return 0.5 * ((tr[..., :2] - d[..., :2]) ** 2).sum()

    Jv = J(lam, mu, a)
    Jv.backward()
    rng = np.random.default_rng(16)
    cells = [(int(rng.integers(20, nx - 20)), int(rng.integers(2, ny - 20))) for _ in range(6)]
    for (x, y) in cells:
        h = 1e-4 * float(lam0[y, x])
        with torch.no_grad():
            lp = lam.detach().clone()
            lm = lam.detach().clone()
            lp[y, x] += h
            lm[y, x] -= h
            fd = (float(J(lp, mu.detach(), a.detach())) - float(J(lm, mu.detach(), a.detach()))) / (2 * h)
        gl = float(lam.grad[y, x])
        gm = float(mu.grad[y, x])
        assert abs(gl - fd) <= 1e-4 * abs(fd) + 1e-11 * abs(Jv.item()) / h, ((x, y), gl, fd)
        assert abs(gm + gl) <= 1e-12 * abs(gl) + 1e-300
    h = 1e-3
    with torch.no_grad():
        fd = (float(J(lam.detach(), mu.detach(), a.detach() + h)) -
              float(J(lam.detach(), mu.detach(), a.detach() - h))) / (2 * h)
    assert abs(float(a.grad[0]) - fd) <= 1e-6 * abs(fd)


def test_fp32_adjoint_close_to_fp64():
    """FP32 states with FP64 gradient sums: the Lambda gradient field is
    within 1e-3 (relative L2) of the FP64 one on the blob problem."""
    from paper_2009_06404_gb300.autograd import simulate_traces
    nx, ny, T = 96, 64, 160
    out = {}
    for storage in ("f64", "f32"):
        setup, lam0, mu0, blob = _blob_setup(nx, ny, T, storage, 40)
        dev = "cuda"
        amp = torch.tensor([1.0], dtype=torch.float64, device=dev)
        with torch.no_grad():
            d = simulate_traces(torch.as_tensor(lam0, device=dev), torch.as_tensor(mu0, device=dev), amp, setup)
        lam = torch.as_tensor(lam0 * (1 - 0.05 * blob), device=dev).requires_grad_(True)
        mu = torch.as_tensor(mu0 * (1 + 0.05 * blob), device=dev).requires_grad_(True)
        tr = simulate_traces(lam, mu, amp, setup)
        (0.5 * ((tr[..., :2] - d[..., :2]) ** 2).sum()).backward()
        out[storage] = lam.grad.cpu().numpy()
    err = np.linalg.norm(out["f32"] - out["f64"]) / np.linalg.norm(out["f64"])
    assert err <= 1e-3, err


def test_adjoint_rejects_16bit_storage():
    pkg = _pkg()
    sim = pkg.ElasticLBM(40, 30, storage="f16")
    with pytest.raises(pkg.LBMError) as e:
        pkg.Adjoint(sim, 10, 5)
    assert e.value.status == -2
