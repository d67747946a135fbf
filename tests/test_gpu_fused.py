"""Two time steps per launch (the intermediate populations in shared memory)
against one step per launch and against the FP64 oracle.

The two-step kernel runs every cell update with the one-step arithmetic, so
states, displacements and traces must agree bit for bit with one-step
launches, for every storage type, boundary kind, grid shape (partial tiles,
grids narrower than a tile, widths that are and are not a multiple of the
16-byte chunks in which general tiles stage their inputs, so that chunks
beyond a periodic seam are copied from their image or element by element),
source placement (across seams and corners), trace-buffer end (the second
step of a launch past the last slot) and odd step count (a one-step launch
at the end)."""
import numpy as np
import pytest

import oracle
from helpers import max_rel, oracle_problem, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


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
    "halfspace_sponges": (("free", "rigid", "periodic", "periodic"), (0, 3, 4, 2)),
    "rigid_box": (("rigid",) * 4, (0, 0, 0, 0)),
    "free_box": (("free",) * 4, (0, 0, 0, 0)),
    "free_tb_rigid_lr": (("free", "free", "rigid", "rigid"), (2, 0, 0, 3)),
    "periodic_x_free_y": (("free", "free", "periodic", "periodic"), (0, 0, 0, 0)),
    "periodic_y_rigid_x": (("periodic", "periodic", "rigid", "rigid"), (3, 2, 0, 0)),
}

# (storage, u_fp64, store_scale_log2)
STORAGES = [("f64", False, 0), ("f32", False, 0), ("f32", True, 0), ("f16", False, 10),
            ("bf16", False, 0)]


def _case(nx, ny, bcname, storage, fs_order=0, per_cell=False, seed=3):
    """Lambda = 0 everywhere (nu = 0.25 in every layer, rho0 varying), two
    sources (one straddling the left seam / corner), four receivers."""
    wl = _wl()
    bc, sponge = BCS[bcname]
    if min(nx, ny) < 10:
        sponge = (0, 0, 0, 0)  # no room for the layers
    rng = np.random.default_rng(seed)
    rho0 = rng.uniform(1.0, 2.0, size=ny)
    if per_cell:
        rho0 = np.repeat(rho0[:, None], nx, 1) * rng.uniform(0.9, 1.1, size=(ny, nx))
    lam, mu = wl.lame(np.full(np.shape(rho0), 0.25), rho0)
    src = np.stack([wl.source(nx * 0.4, ny * 0.5, sigma=1.5, direction=(0.6, 0.8), f_peak=0.2,
                              t0=2.0, r_cut=5.0),
                    wl.source(0.5, 1.0, sigma=1.0, direction=(1.0, 0.0), f_peak=0.3, t0=1.0,
                              r_cut=3.0)])
    rec = np.array([[0, 0], [nx - 1, ny - 1], [nx // 2, ny // 3], [1, ny - 2]], np.int32)
    return wl.Workload(name="fused", nx=nx, ny=ny, nsteps=7, tau=0.8, storage=storage, bc=bc,
                       sponge=sponge, fs_order=fs_order, rho0=rho0, lam=lam, mu=mu,
                       sources=src, receivers=rec)


def _run(w, spl, u_fp64=False, k=0, nsteps=None, max_traced=None, seed=5):
    sim = _pkg().from_workload(w, kernel="simple", u_fp64=u_fp64, store_scale_log2=k,
                               max_steps_traced=max_traced)
    sim.set_steps_per_launch(spl)
    fs0, u0 = _wl().random_state(w.nx, w.ny, seed=seed)
    sim.set_state(fs0, u0, step=3)
    n0 = sim.kernel_launches
    sim.step(w.nsteps if nsteps is None else nsteps)
    launches = sim.kernel_launches - n0
    fs, u = sim.get_state()
    return sim, fs, u, sim.read_traces(), launches


@pytest.mark.parametrize("storage,u64,k", STORAGES)
@pytest.mark.parametrize("bcname", sorted(BCS))
@pytest.mark.parametrize("nx,ny", [(3, 3), (13, 7), (33, 17), (70, 45), (96, 40), (300, 37)])
def test_two_step_equals_one_step_bitwise(storage, u64, k, bcname, nx, ny):
    """Seven steps (three two-step launches and one one-step launch) from a
    random state; the trace buffer holds six steps, so the last pair records
    its first step only."""
    w = _case(nx, ny, bcname, storage)
    s1, fs1, u1, tr1, l1 = _run(w, 1, u64, k, max_traced=6)
    s2, fs2, u2, tr2, l2 = _run(w, 2, u64, k, max_traced=6)
    assert (l1, l2) == (7, 4)
    assert s1.step_index == s2.step_index == 10
    assert np.array_equal(fs1, fs2)
    assert np.array_equal(u1, u2)
    assert tr1.shape == tr2.shape == (6, 4, 4)
    assert np.array_equal(tr1, tr2)


@pytest.mark.parametrize("fs_order", [0, 1])
@pytest.mark.parametrize("bcname", ["halfspace_sponges", "free_box", "free_tb_rigid_lr"])
def test_two_step_free_surface_orders_bitwise(fs_order, bcname):
    """Both free-surface extrapolation orders, per-cell material."""
    w = _case(70, 45, bcname, "f64", fs_order=fs_order, per_cell=True)
    _, fs1, u1, tr1, _ = _run(w, 1)
    _, fs2, u2, tr2, _ = _run(w, 2)
    assert np.array_equal(fs1, fs2) and np.array_equal(u1, u2) and np.array_equal(tr1, tr2)


@pytest.mark.parametrize("storage,tol", [("f64", 1e-12), ("f32", 1e-5)])
@pytest.mark.parametrize("bcname", ["halfspace_sponges", "free_tb_rigid_lr", "periodic"])
def test_two_step_matches_oracle(storage, tol, bcname):
    """Six steps (three two-step launches) from a random state equal the
    oracle's element by element."""
    w = _case(70, 45, bcname, storage, fs_order=1).with_(nsteps=6)
    _, fs, u, tr, launches = _run(w, 2)
    assert launches == 3
    prob = oracle_problem(w)
    fs0, u0 = _wl().random_state(w.nx, w.ny, seed=5)
    st, tro = oracle.run(prob, 6, oracle.State(prob, fs=fs0, u=u0, n=3))
    assert max_rel(fs, st.fs) <= tol
    assert max_rel(u, st.u) <= tol
    assert max_rel(tr, tro) <= tol


@pytest.mark.parametrize("nsteps", [2, 4])
@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_two_step_full_size_halfspace(storage, nsteps):
    """The bench's workload (2048 x 1024 half-space, free top, 64-cell layers)
    from a random state, two or four steps in two-step launches: every cell
    equals the oracle's steps."""
    w = _wl().halfspace(nsteps=nsteps, storage=storage)
    fs0, u0 = _wl().random_state(w.nx, w.ny, seed=21)
    sim = _pkg().from_workload(w)
    sim.set_steps_per_launch(2)  # (the FP64 default is one step per launch)
    sim.set_state(fs0, u0, step=40)
    n0 = sim.kernel_launches
    sim.step(nsteps)
    assert sim.kernel_launches - n0 == nsteps // 2
    fs, u = sim.get_state()
    prob = oracle_problem(w)
    st, _ = oracle.run(prob, nsteps, oracle.State(prob, fs=fs0, u=u0, n=40), traces=False)
    tol = {"f64": 1e-12, "f32": 1e-5}[storage]
    assert max_rel(fs, st.fs) <= tol
    assert max_rel(u, st.u) <= tol


def test_two_step_many_sources_bitwise():
    """Sixteen sources over a periodic layered grid (source culling by the
    tile's window), 20 steps, FP32."""
    wl = _wl()
    w = wl.periodic_layered_multisource(n=256, nsteps=20, seed=5, storage="f32")
    w = w.with_(lam=w.mu.copy())  # Lambda = 0 in every layer
    outs = []
    for spl in (1, 2):
        sim = _pkg().from_workload(w, kernel="simple")
        sim.set_steps_per_launch(spl)
        sim.step(w.nsteps)
        outs.append(sim.get_state())
    for o in outs[1:]:
        assert np.array_equal(outs[0][0], o[0])
        assert np.array_equal(outs[0][1], o[1])
    assert np.abs(outs[0][1]).max() > 0


@pytest.mark.parametrize("storage,u64,k", [("f32", False, 0), ("f16", False, 10)])
@pytest.mark.parametrize("bcname", ["periodic", "halfspace_sponges", "periodic_y_rigid_x"])
@pytest.mark.parametrize("nx,ny", [(61, 29), (89, 41)])
def test_two_step_periodic_partial_tile_overlap_bitwise(storage, u64, k, bcname, nx, ny):
    """A partial tile on a periodic axis computes the full tile that ends at
    the seam and stores only its own cells: receivers and a source inside
    the cells it computes again (its neighbour's), and a partial tile one
    cell wide or tall (61 = 2 x 30 + 1, 29 = 2 x 14 + 1), leave every cell,
    displacement and trace bit for bit as one step per launch."""
    wl = _wl()
    w = _case(nx, ny, bcname, storage)
    # a cell of the last tile's overlap region: x in [nx - 30, 30 (nx // 30)),
    # y in [ny - 14, 14 (ny // 14))
    xo = (nx - 30 + 30 * (nx // 30)) // 2
    yo = (ny - 14 + 14 * (ny // 14)) // 2
    src = np.concatenate([w.sources, wl.source(xo + 0.3, yo + 0.6, sigma=1.2, direction=(0.0, 1.0),
                                               f_peak=0.25, t0=1.5, r_cut=4.0)[None]])
    rec = np.array([[xo, yo], [xo - 5, 3], [4, yo + 2], [nx - 1, ny - 1], [nx - 2, 0]], np.int32)
    w = w.with_(sources=src, receivers=rec)
    s1, fs1, u1, tr1, l1 = _run(w, 1, u64, k, max_traced=6)
    s2, fs2, u2, tr2, l2 = _run(w, 2, u64, k, max_traced=6)
    assert (l1, l2) == (7, 4)
    assert np.array_equal(fs1, fs2)
    assert np.array_equal(u1, u2)
    assert tr1.shape == tr2.shape == (6, 5, 4)
    assert np.array_equal(tr1, tr2)
    assert np.abs(tr1[:, 0]).max() > 0


def _case_lam(nx, ny, bcname, storage, fs_order=0, per_cell=False, seed=3):
    """As _case, with a Poisson ratio per row (per cell with per_cell) in
    [0.15, 0.33]: Lambda != 0, the density-gradient force is on."""
    wl = _wl()
    w = _case(nx, ny, bcname, storage, fs_order, per_cell, seed)
    nu = np.random.default_rng(seed + 1).uniform(0.15, 0.33, size=np.shape(w.rho0))
    lam, mu = wl.lame(nu, w.rho0)
    return w.with_(lam=lam, mu=mu)


@pytest.mark.parametrize("storage,u64,k", STORAGES)
@pytest.mark.parametrize("bcname", sorted(BCS))
@pytest.mark.parametrize("nx,ny", [(3, 3), (13, 7), (40, 21), (70, 45), (96, 40), (300, 37)])
def test_two_step_gradient_force_equals_one_step_bitwise(storage, u64, k, bcname, nx, ny):
    """With the density-gradient force (step n on the tile widened by two
    cells, densities on the tile widened by three): seven steps, three
    two-step launches and one one-step launch, bit for bit."""
    w = _case_lam(nx, ny, bcname, storage)
    _, fs1, u1, tr1, l1 = _run(w, 1, u64, k, max_traced=6)
    _, fs2, u2, tr2, l2 = _run(w, 2, u64, k, max_traced=6)
    assert (l1, l2) == (7, 4)
    assert np.array_equal(fs1, fs2)
    assert np.array_equal(u1, u2)
    assert np.array_equal(tr1, tr2)


@pytest.mark.parametrize("fs_order", [0, 1])
@pytest.mark.parametrize("bcname", ["halfspace_sponges", "free_box", "free_tb_rigid_lr"])
def test_two_step_gradient_force_per_cell_bitwise(fs_order, bcname):
    """Per-cell Lambda, both free-surface extrapolation orders (the wall
    ghosts of the density gradient), FP64."""
    w = _case_lam(70, 45, bcname, "f64", fs_order=fs_order, per_cell=True)
    _, fs1, u1, tr1, _ = _run(w, 1)
    _, fs2, u2, tr2, _ = _run(w, 2)
    assert np.array_equal(fs1, fs2) and np.array_equal(u1, u2) and np.array_equal(tr1, tr2)


@pytest.mark.parametrize("storage,tol", [("f64", 1e-12), ("f32", 1e-5)])
@pytest.mark.parametrize("bcname", ["halfspace_sponges", "free_tb_rigid_lr", "periodic"])
def test_two_step_gradient_force_matches_oracle(storage, tol, bcname):
    """Six steps with Lambda != 0 (three two-step launches) from a random
    state equal the oracle's element by element."""
    w = _case_lam(70, 45, bcname, storage, fs_order=1).with_(nsteps=6)
    _, fs, u, tr, launches = _run(w, 2)
    assert launches == 3
    prob = oracle_problem(w)
    fs0, u0 = _wl().random_state(w.nx, w.ny, seed=5)
    st, tro = oracle.run(prob, 6, oracle.State(prob, fs=fs0, u=u0, n=3))
    assert max_rel(fs, st.fs) <= tol
    assert max_rel(u, st.u) <= tol
    assert max_rel(tr, tro) <= tol


@pytest.mark.parametrize("storage,tol", [("f64", 1e-12), ("f32", 1e-5)])
@pytest.mark.parametrize("lam", [False, True])
def test_sources_across_seams_match_oracle(storage, tol, lam):
    """Eight sources on and near every periodic seam and corner of a grid
    whose last tiles and blocks are partial (100 x 52), receivers at tile
    corners: the host's list of the tiles a source or receiver reaches (the
    kernels skip those lookups everywhere else) must miss none, so one- and
    two-step launches agree bit for bit and both equal the oracle."""
    wl = _wl()
    w = (_case_lam if lam else _case)(100, 52, "periodic", storage)
    spots = [(0.3, 20.0, 4.0), (99.6, 40.0, 5.0), (50.0, 0.2, 4.0), (70.0, 51.7, 6.0),
             (99.5, 51.5, 3.0), (30.0, 26.0, 4.0), (14.0, 10.0, 8.0), (85.0, 33.0, 5.0)]
    src = np.stack([wl.source(x, y, sigma=1.5, direction=(0.6, 0.8), f_peak=0.25, t0=2.0,
                              r_cut=r) for x, y, r in spots])
    rec = np.array([[0, 0], [99, 51], [50, 26], [27, 11], [28, 12], [97, 3]], np.int32)
    w = w.with_(sources=src, receivers=rec, nsteps=6)
    out = {spl: _run(w, spl)[1:4] for spl in (1, 2)}
    for a, b in zip(out[1], out[2]):
        assert np.array_equal(a, b)
    prob = oracle_problem(w)
    fs0, u0 = wl.random_state(w.nx, w.ny, seed=5)
    st, tro = oracle.run(prob, 6, oracle.State(prob, fs=fs0, u=u0, n=3))
    fs, u, tr = out[2]
    assert max_rel(fs, st.fs) <= tol
    assert max_rel(u, st.u) <= tol
    assert max_rel(tr, tro) <= tol


def test_two_step_gradient_force_layered_run_bitwise():
    """A layered half-space (Lambda != 0 in every layer) from rest, 300
    steps with traces, FP32: two-step and one-step launches bit for bit."""
    w = _wl().layered_halfspace(256, 96, 300, seed=4, sponge=16, nrec=32, storage="f32")
    res = []
    for spl in (1, 2):
        sim = _pkg().from_workload(w, kernel="simple")
        sim.set_steps_per_launch(spl)
        sim.step(w.nsteps)
        res.append((sim.get_state(), sim.read_traces()))
    (a, ta), (b, tb) = res
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert np.array_equal(ta, tb)
    assert rel_l2(ta, np.zeros_like(ta)) > 0


def test_steps_per_launch_argument_and_defaults():
    """1 and 2 are accepted; until set, FP32 handles take two steps per
    launch, 16-bit handles two without and one with the gradient force, FP64
    handles one."""
    for storage, k, lam, per_launch in (("f32", 0, False, 2), ("f16", 10, False, 2),
                                        ("f64", 0, False, 1), ("f32", 0, True, 2),
                                        ("f16", 10, True, 1), ("bf16", 0, True, 1)):
        w = (_case_lam if lam else _case)(13, 7, "periodic", storage)
        sim = _pkg().from_workload(w, store_scale_log2=k)
        n0 = sim.kernel_launches
        sim.step(4)
        assert sim.kernel_launches - n0 == 4 // per_launch, storage
        for bad in (3, 0, -1):
            with pytest.raises(_pkg().LBMError):
                sim.set_steps_per_launch(bad)
        for good in (1, 2):
            sim.set_steps_per_launch(good)


def test_two_step_long_run_matches_one_step_f32():
    """400 steps of a layered half-space from rest with traces: two-step and
    one-step launches stay bit-identical."""
    wl = _wl()
    w = wl.layered_halfspace(256, 96, 400, seed=4, sponge=16, nrec=32, storage="f32")
    w = w.with_(lam=w.mu.copy())
    res = []
    for spl in (1, 2):
        sim = _pkg().from_workload(w, kernel="simple")
        sim.set_steps_per_launch(spl)
        sim.step(w.nsteps)
        res.append((sim.get_state(), sim.read_traces()))
    (a, ta) = res[0]
    for (b, tb) in res[1:]:
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
        assert np.array_equal(ta, tb)
    assert rel_l2(ta, np.zeros_like(ta)) > 0
