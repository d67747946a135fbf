"""Parity of the CUDA library (called through the C ABI) with the FP64 CPU
oracle on the same seeded inputs.

Tolerances: FP64 storage and arithmetic -- relative L2 of the displacement
<= 1e-12 (element-wise checks on populations <= 1e-12 of the largest value);
FP32 -- relative L2 of the displacement <= 1e-4 after the full 4000-step
half-space run, and <= 1e-5 of the largest population value for a few steps
from a random state (a few FP32 roundings)."""
import os

import numpy as np
import pytest

import oracle
from helpers import max_rel, oracle_problem, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


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


TOL_F = {"f64": 1e-12, "f32": 1e-5}


# ------------------------------------------------------------ configs[0]

def test_periodic_bulk_128_f64_500_steps():
    """128x128 periodic, FP64, nu = 0.25, tau = 1, Gaussian x Ricker source,
    500 steps: displacement, velocity, density, stress and the 64-receiver
    ring match the oracle (rel-L2 <= 1e-12)."""
    w = _wl().periodic_bulk(128, 500, "f64")
    sim = _pkg().from_workload(w)
    sim.step(w.nsteps)
    f = sim.read_fields(on_device=False)
    tr = sim.read_traces()
    prob = oracle_problem(w)
    st, tro = oracle.run(prob, w.nsteps)
    fo = oracle.fields(prob, st)
    assert rel_l2(np.stack([f["ux"], f["uy"]]), st.u) <= 1e-12
    for k in ("vx", "vy", "rho", "pxx", "pxy", "pyy"):
        assert rel_l2(f[k], fo[k]) <= 1e-12, k
    assert tr.shape == tro.shape == (500, 64, 4)
    assert rel_l2(tr, tro) <= 1e-12
    assert sim.kernel_launches >= w.nsteps


def test_periodic_bulk_paper_variant_tau055_nu01_f64():
    """The paper's bulk-wave set-up (tau = 0.55, nu = 0.1: Lambda != 0, so the
    density-gradient force is active), 128x128, 70 steps."""
    wl = _wl()
    w = wl.periodic_bulk(128, 70, "f64", nu=0.1, tau=0.55)
    w = w.with_(sources=wl.source(64, 64, sigma=4.0, f_peak=0.05, t0=30.0, r_cut=32.0)[None])
    sim = _pkg().from_workload(w)
    sim.step(w.nsteps)
    f = sim.read_fields(on_device=False)
    prob = oracle_problem(w)
    st, _ = oracle.run(prob, w.nsteps, traces=False)
    fo = oracle.fields(prob, st)
    for k in ("vx", "vy", "rho", "pxx"):
        assert rel_l2(f[k], fo[k]) <= 1e-12, k
    assert rel_l2(np.stack([f["ux"], f["uy"]]), st.u) <= 1e-12


# ------------------------------------------------------------ all boundary kinds

BCS = {
    "periodic": (("periodic",) * 4, (0, 0, 0, 0)),
    "free_top_rigid_bottom": (("free", "rigid", "periodic", "periodic"), (0, 0, 0, 0)),
    "halfspace_sponges": (("free", "rigid", "periodic", "periodic"), (0, 3, 4, 2)),
    "rigid_box": (("rigid", "rigid", "rigid", "rigid"), (0, 0, 0, 0)),
    "free_box": (("free", "free", "free", "free"), (0, 0, 0, 0)),
    "free_tb_rigid_lr": (("free", "free", "rigid", "rigid"), (2, 0, 0, 3)),
    "periodic_sponges": (("periodic",) * 4, (2, 3, 4, 5)),
}


def _random_case(nx, ny, bc, sponge, nu_rows, per_cell, seed, storage, fs_order=0):
    wl = _wl()
    rng = np.random.default_rng(seed)
    rho0 = rng.uniform(1.0, 2.0, size=ny)
    lam, mu = wl.lame(nu_rows, rho0)
    if per_cell:
        rho0 = np.repeat(rho0[:, None], nx, 1) * rng.uniform(0.9, 1.1, size=(ny, nx))
        lam, mu = wl.lame(np.repeat(np.asarray(nu_rows)[:, None], nx, 1), rho0)
    src = np.stack([wl.source(nx * 0.4, ny * 0.5, sigma=1.5, direction=(0.6, 0.8), f_peak=0.2,
                              t0=2.0, r_cut=5.0),
                    wl.source(1.0, ny - 2.0, sigma=1.0, direction=(1.0, 0.0), f_peak=0.3,
                              t0=1.0, r_cut=3.0)])
    rec = np.array([[0, 0], [nx - 1, ny - 1], [nx // 2, ny // 3]], np.int32)
    return wl.Workload(name="random", nx=nx, ny=ny, nsteps=5, tau=0.8, storage=storage, bc=bc,
                       sponge=sponge, fs_order=fs_order, rho0=rho0, lam=lam, mu=mu, sources=src,
                       receivers=rec)


STORAGE_KERNELS = [("f64", "simple"), ("f32", "simple")]


@pytest.mark.parametrize("storage,kernel", STORAGE_KERNELS)
@pytest.mark.parametrize("bcname", sorted(BCS))
@pytest.mark.parametrize("nx,ny", [(13, 7), (70, 45), (300, 37)])
@pytest.mark.parametrize("fs_order", [0, 1])
def test_random_state_all_boundaries(storage, kernel, bcname, nx, ny, fs_order):
    """From a random state, five steps on odd grids (one partial block; several
    blocks with ragged edges) with every boundary kind, absorbing layers,
    per-row non-Poisson layers, two sources and three receivers: populations,
    displacement and traces match the oracle element by element."""
    bc, sponge = BCS[bcname]
    rng = np.random.default_rng(nx * 1000 + ny)
    nu_rows = rng.uniform(0.15, 0.33, size=ny)
    if fs_order == 1 and "free" not in bc:
        pytest.skip("extrapolation order only matters at a free surface")
    w = _random_case(nx, ny, bc, sponge, nu_rows, False, 3, storage, fs_order)
    fs0, u0 = _wl().random_state(nx, ny, seed=5)
    sim = _pkg().from_workload(w, kernel=kernel)
    sim.set_state(fs0, u0, step=3)
    sim.step(w.nsteps)
    fs, u = sim.get_state()
    tr = sim.read_traces()
    prob = oracle_problem(w)
    st, tro = oracle.run(prob, w.nsteps, oracle.State(prob, fs=fs0, u=u0, n=3))
    tol = TOL_F[storage]
    assert max_rel(fs, st.fs) <= tol
    assert max_rel(u, st.u) <= tol
    assert max_rel(tr, tro) <= tol


@pytest.mark.parametrize("storage,kernel", STORAGE_KERNELS)
def test_per_cell_material(storage, kernel):
    """Per-cell rho0 and Poisson ratio (Lambda varies cell by cell)."""
    nx, ny = 45, 33
    rng = np.random.default_rng(9)
    nu_rows = rng.uniform(0.15, 0.33, size=ny)
    w = _random_case(nx, ny, ("free", "rigid", "periodic", "periodic"), (0, 4, 3, 3), nu_rows,
                     True, 4, storage)
    fs0, u0 = _wl().random_state(nx, ny, seed=6)
    sim = _pkg().from_workload(w, kernel=kernel)
    sim.set_state(fs0, u0, step=0)
    sim.step(w.nsteps)
    fs, u = sim.get_state()
    prob = oracle_problem(w)
    st, _ = oracle.run(prob, w.nsteps, oracle.State(prob, fs=fs0, u=u0), traces=False)
    assert max_rel(fs, st.fs) <= TOL_F[storage]
    assert max_rel(u, st.u) <= TOL_F[storage]


def test_layered_halfspace_traces_f64():
    """Layered half-space (free top, absorbing layers, 4 layers with
    nu in [0.2, 0.35]) from rest, 300 steps: receiver traces and the
    displacement match the oracle (rel-L2 <= 1e-12)."""
    w = _wl().layered_halfspace(256, 96, 300, seed=4, sponge=16, nrec=32, storage="f64")
    sim = _pkg().from_workload(w)
    sim.step(w.nsteps)
    tr = sim.read_traces()
    f = sim.read_fields(("ux", "uy"), on_device=True)
    prob = oracle_problem(w)
    st, tro = oracle.run(prob, w.nsteps)
    assert rel_l2(tr, tro) <= 1e-12
    u = np.stack([f["ux"].cpu().numpy(), f["uy"].cpu().numpy()])
    assert rel_l2(u, st.u) <= 1e-12


# ------------------------------------------------------------ full size

@pytest.mark.parametrize("storage,kernel", STORAGE_KERNELS)
def test_halfspace_full_size_single_step(storage, kernel):
    """Full half-space size (2048 x 1024, free top, 64-cell layers, the bench's
    launch configuration): one step from a random state equals the oracle's
    step at every cell."""
    w = _wl().halfspace(nsteps=1, storage=storage)
    fs0, u0 = _wl().random_state(w.nx, w.ny, seed=21)
    sim = _pkg().from_workload(w, kernel=kernel)
    sim.set_state(fs0, u0, step=40)
    sim.step(1)
    fs, u = sim.get_state()
    prob = oracle_problem(w)
    st, _ = oracle.run(prob, 1, oracle.State(prob, fs=fs0, u=u0, n=40), traces=False)
    assert max_rel(fs, st.fs) <= TOL_F[storage]
    assert max_rel(u, st.u) <= TOL_F[storage]


@pytest.mark.parametrize("storage,tol", [("f64", 1e-11), ("f32", 1e-4)])
def test_halfspace_full_run_against_stored_oracle(storage, tol):
    """The full half-space workload (2048 x 1024, 4000 steps, 256 surface
    receivers) against sampled oracle outputs written by
    tests/golden/make_halfspace_golden.py: displacement (every 16th cell),
    velocity and traces (every 16th receiver, every 4th step)."""
    path = os.path.join(ROOT, "tests", "golden", "halfspace_2048x1024_4000.npz")
    g = np.load(path)
    w = _wl().halfspace(storage=storage)
    sim = _pkg().from_workload(w)
    sim.step(w.nsteps)
    f = sim.read_fields(("ux", "uy", "vx", "vy"), on_device=True)
    s = int(g["stride"])
    u = np.stack([f["ux"][::s, ::s].cpu().numpy(), f["uy"][::s, ::s].cpu().numpy()])
    v = np.stack([f["vx"][::s, ::s].cpu().numpy(), f["vy"][::s, ::s].cpu().numpy()])
    tr = sim.read_traces()
    ss, rs = int(g["step_stride"]), int(g["rec_stride"])
    tr = tr[ss - 1::ss, ::rs, :]
    assert rel_l2(u, g["u"]) <= tol
    assert rel_l2(v, g["v"]) <= tol * 10
    assert rel_l2(tr, g["traces"]) <= tol


# ------------------------------------------------------------ invariants at size

def test_invariants_large_periodic_f64():
    """Properties that hold at any size (Eqs. 12, 22): on a 1024 x 1024
    periodic grid with uniform nu = 0.3 and no source, sum rho, sum m and
    sum P are conserved over 100 steps; with a source, sum m grows by the
    summed body force."""
    wl = _wl()
    n = 1024
    rho0, lam, mu = wl.homogeneous(n, 0.3)
    sim = _pkg().ElasticLBM(n, n, storage="f64", max_sources=1, max_receivers=1)
    sim.set_material(rho0, lam, mu)
    fs0, _ = wl.random_state(n, n, seed=2)
    sim.set_state(fs0)
    m0 = sim.moment_sums()
    sim.step(100)
    m1 = sim.moment_sums()
    scale = np.abs(fs0).sum()
    assert np.all(np.abs(m1[:6] - m0[:6]) <= 1e-12 * scale)
    # source: sum of f* c grows by sum_x F each step
    src = wl.source(300.5, 700.25, sigma=3.0, direction=(0.6, -0.8), amplitude=2.0)
    sim.set_sources(src[None])
    sim.set_state(np.zeros((9, n, n)), step=40)
    xs, ys = np.meshgrid(np.arange(n), np.arange(n))
    r2 = (xs - src[0]) ** 2 + (ys - src[1]) ** 2
    g = np.where(r2 <= src[8] ** 2, np.exp(-r2 / (2 * src[2] ** 2)), 0.0).sum()
    total = np.zeros(2)
    for k in range(5):
        t = 40 + k
        a = (np.pi * src[6] * (t - src[7])) ** 2
        total += src[5] * src[3:5] * g * (1 - 2 * a) * np.exp(-a)
        sim.step(1)
    m = sim.moment_sums()
    np.testing.assert_allclose(m[1:3], total, rtol=1e-12, atol=1e-12)


# ------------------------------------------------------------ API behaviour

@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_checkpoint_resume_and_determinism_bitwise(storage):
    w = _wl().layered_halfspace(130, 70, 30, seed=7, sponge=10, nrec=8, storage=storage)
    sim = _pkg().from_workload(w)
    sim.step(20)
    ck = sim.save(on_device=True)
    ck_host = sim.save(on_device=False)
    sim.step(10)
    a, ua = sim.get_state()
    sim.load(ck)
    assert sim.step_index == 20
    sim.step(10)
    b, ub = sim.get_state()
    assert np.array_equal(a, b) and np.array_equal(ua, ub)
    sim.load(ck_host)
    sim.step(10)
    c, uc = sim.get_state()
    assert np.array_equal(a, c) and np.array_equal(ua, uc)
    # a second handle from scratch gives the same bits
    sim2 = _pkg().from_workload(w)
    sim2.step(30)
    d, ud = sim2.get_state()
    assert np.array_equal(a, d) and np.array_equal(ua, ud)


def test_read_fields_host_equals_device():
    w = _wl().layered_halfspace(600, 600, 15, seed=8, sponge=8, nrec=4, storage="f32")
    sim = _pkg().from_workload(w)
    sim.step(15)
    h = sim.read_fields(on_device=False)
    d = sim.read_fields(on_device=True)
    for k in h:
        assert np.array_equal(h[k], d[k].cpu().numpy()), k


def test_set_get_state_roundtrip():
    wl = _wl()
    fs0, u0 = wl.random_state(37, 29, seed=1)
    for storage in ("f64", "f32"):
        sim = _pkg().ElasticLBM(37, 29, storage=storage)
        sim.set_state(fs0, u0, step=5)
        fs, u = sim.get_state()
        if storage == "f64":
            assert np.array_equal(fs, fs0) and np.array_equal(u, u0)
        else:
            assert np.array_equal(fs, fs0.astype(np.float32).astype(np.float64))
        assert sim.step_index == 5
        td = torch.tensor(fs0, device="cuda")
        sim.set_state(td, None, step=0)
        fsd, ud = sim.get_state(on_device=True)
        assert np.array_equal(fsd.cpu().numpy(), fs)
        assert float(ud.abs().max()) == 0.0


def test_moment_sums_match_state():
    wl = _wl()
    sim = _pkg().ElasticLBM(64, 40, storage="f64")
    fs0, u0 = wl.random_state(64, 40, seed=3)
    sim.set_state(fs0, u0)
    m = sim.moment_sums()
    cx = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
    cy = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
    want = [fs0.sum(), np.einsum("iyx,i->", fs0, cx), np.einsum("iyx,i->", fs0, cy),
            np.einsum("iyx,i->", fs0, cx * cx), np.einsum("iyx,i->", fs0, cx * cy),
            np.einsum("iyx,i->", fs0, cy * cy), (u0 ** 2).sum()]
    np.testing.assert_allclose(m, want, rtol=1e-12, atol=1e-14)
    assert np.array_equal(m, sim.moment_sums())


def test_nonfinite_run_reports_error():
    """An unstable run (nu = 0.45 at tau = 1, Sec. 4) overflows; the step
    kernel flags it and the next synchronising call reports it."""
    wl = _wl()
    n = 64
    rho0, lam, mu = wl.homogeneous(n, 0.45)
    sim = _pkg().ElasticLBM(n, n, storage="f32")
    sim.set_material(rho0, lam, mu)
    fs0, _ = wl.random_state(n, n, seed=4, scale=1.0)
    sim.set_state(fs0)
    sim.step(400)
    with pytest.raises(_pkg().NonFiniteError):
        sim.sync()
    sim.reset()
    sim.sync()


def test_zero_and_negative_steps():
    sim = _pkg().ElasticLBM(16, 16, storage="f32")
    sim.step(0)
    assert sim.step_index == 0 and sim.kernel_launches >= 0
    with pytest.raises(_pkg().LBMError):
        sim.step(-1)


def test_vs_not_b_warning_and_capacities():
    pkg = _pkg()
    sim = pkg.ElasticLBM(16, 16, storage="f32", max_sources=1, max_receivers=2)
    st = sim.set_material(np.ones(16), np.full(16, 0.1), np.full(16, 0.5))
    assert st == 1  # LBM_WARN_VS_NOT_B
    with pytest.raises(pkg.LBMError):
        sim.set_material(np.zeros(16), np.zeros(16), np.zeros(16))
    with pytest.raises(pkg.LBMError):
        sim.set_sources(np.zeros((2, 9)) + 1.0)
    with pytest.raises(pkg.LBMError):
        sim.set_receivers([[0, 0], [1, 1], [2, 2]])
    with pytest.raises(pkg.LBMError):
        sim.set_receivers([[16, 0]])


def test_per_row_equals_per_cell_material_bitwise():
    wl = _wl()
    nx, ny = 50, 30
    rng = np.random.default_rng(2)
    rho0, lam, mu = wl.layered(ny, rng, 3, (0.2, 0.3), (1.0, 2.0))
    fs0, u0 = wl.random_state(nx, ny, seed=8)
    out = []
    for per_cell in (False, True):
        sim = _pkg().ElasticLBM(nx, ny, storage="f32", material_per_cell=per_cell,
                                bc=("free", "rigid", "periodic", "periodic"))
        if per_cell:
            sim.set_material(*[np.repeat(a[:, None], nx, 1) for a in (rho0, lam, mu)])
        else:
            sim.set_material(rho0, lam, mu)
        sim.set_state(fs0, u0)
        sim.step(7)
        out.append(sim.get_state())
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


# ------------------------------------------------------------ 16-bit storage

TOL_16 = {"f16": 3e-3, "bf16": 3e-2}  # a few roundings at 2^-11 and 2^-8


@pytest.mark.parametrize("storage,k", [("f16", 10), ("bf16", 0)])
@pytest.mark.parametrize("bcname", ["periodic", "halfspace_sponges", "free_box", "rigid_box"])
def test_16bit_storage_random_state(storage, k, bcname):
    """FP16/BF16 population storage (deviations from rest times 2^k, FP32
    arithmetic): five steps from a random state on a 70 x 45 grid match the
    FP64 oracle to a few 16-bit roundings."""
    bc, sponge = BCS[bcname]
    nx, ny = 70, 45
    rng = np.random.default_rng(11)
    nu_rows = rng.uniform(0.15, 0.33, size=ny)
    w = _random_case(nx, ny, bc, sponge, nu_rows, False, 3, storage)
    fs0, u0 = _wl().random_state(nx, ny, seed=5)
    sim = _pkg().from_workload(w, store_scale_log2=k)
    sim.set_state(fs0, u0, step=3)
    sim.step(w.nsteps)
    fs, u = sim.get_state()
    prob = oracle_problem(w)
    st, _ = oracle.run(prob, w.nsteps, oracle.State(prob, fs=fs0, u=u0, n=3), traces=False)
    assert max_rel(fs, st.fs) <= TOL_16[storage]
    assert max_rel(u, st.u) <= TOL_16[storage]


@pytest.mark.parametrize("storage,k,tol", [("f16", 10, 5e-3), ("bf16", 0, 5e-2)])
def test_16bit_halfspace_traces_first_1000_steps(storage, k, tol):
    """The full half-space with 16-bit storage: surface traces of the first
    1000 steps against the stored oracle samples.  A 16-bit run's error is
    one realization of a walk of storage roundings: changing the source
    amplitude by 1e-6 moves it between 5.5e-4 and 2.2e-3 rel-L2 (FP16) and
    between 1.8e-2 and 3.2e-2 (BF16).  The FP16 tolerance is below the
    random-walk scale of 1000 half-ulp roundings, sqrt(1000) 2^-12 = 7.7e-3."""
    g = np.load(os.path.join(ROOT, "tests", "golden", "halfspace_2048x1024_4000.npz"))
    w = _wl().halfspace(nsteps=1000, storage=storage)
    sim = _pkg().from_workload(w, store_scale_log2=k, max_steps_traced=1000)
    sim.step(1000)
    ss, rs = int(g["step_stride"]), int(g["rec_stride"])
    tr = sim.read_traces()[ss - 1::ss, ::rs, :]
    assert rel_l2(tr, g["traces"][:tr.shape[0]]) <= tol


@pytest.mark.parametrize("storage,k", [("f16", 7), ("bf16", 0)])
def test_16bit_checkpoint_and_sums(storage, k):
    wl = _wl()
    w = wl.layered_halfspace(140, 60, 20, seed=2, sponge=8, nrec=4, storage=storage)
    sim = _pkg().from_workload(w, store_scale_log2=k)
    sim.step(10)
    ck = sim.save()
    sim.step(10)
    a, ua = sim.get_state()
    sim.load(ck)
    sim.step(10)
    b, ub = sim.get_state()
    assert np.array_equal(a, b) and np.array_equal(ua, ub)
    m = sim.moment_sums()
    cx = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
    cy = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
    want = [b.sum(), np.einsum("iyx,i->", b, cx), np.einsum("iyx,i->", b, cy),
            np.einsum("iyx,i->", b, cx * cx), np.einsum("iyx,i->", b, cx * cy),
            np.einsum("iyx,i->", b, cy * cy), (ub ** 2).sum()]
    np.testing.assert_allclose(m, want, rtol=1e-10, atol=1e-12)
    # a checkpoint of another scale does not load
    other = _pkg().from_workload(w, store_scale_log2=k + 1)
    with pytest.raises(_pkg().LBMError):
        other.load(ck)
