"""Batched stepping of many grids (one launch per step over the tiles of all
shots, a CUDA graph of such launches, or one persistent cooperative launch
with a grid barrier): every shot must give exactly what it gives when
stepped alone, for every launch form, tile height and tile order, and the
batch must match the FP64 oracle like a single grid does."""
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


def _pkg():
    import paper_2009_06404_gb300 as pkg
    return pkg


def _wl():
    from paper_2009_06404_gb300 import workloads
    return workloads


def _shot_workloads(storage, nsteps=40):
    """Uneven, ragged shots covering every boundary kind, Lambda = 0 and != 0,
    sources near edges and receivers."""
    wl = _wl()
    out = []
    # layered half-space, ragged in x and y, Lambda != 0
    out.append(wl.layered_halfspace(70, 45, nsteps, seed=11, sponge=6, nrec=9, storage=storage,
                                    src_x=30.0, src_y=5.0))
    # periodic, Lambda != 0, a source across the seam
    rho0, lam, mu = wl.homogeneous(64, 0.3)
    out.append(wl.Workload(name="per", nx=96, ny=64, nsteps=nsteps, storage=storage, rho0=rho0,
                           lam=lam, mu=mu,
                           sources=wl.source(1.0, 30.0, sigma=2.0, f_peak=0.1, t0=8.0,
                                             r_cut=8.0)[None],
                           receivers=np.array([[0, 0], [95, 63], [40, 20]], np.int32)))
    # rigid box, Lambda = 0 (nu = 0.25)
    rho0, lam, mu = wl.homogeneous(33, 0.25)
    out.append(wl.Workload(name="rigid", nx=40, ny=33, nsteps=nsteps, storage=storage,
                           bc=("rigid",) * 4, rho0=rho0, lam=lam, mu=mu,
                           sources=wl.source(20.0, 16.0, sigma=2.0, direction=(0.6, 0.8),
                                             f_peak=0.1, t0=8.0, r_cut=8.0)[None]))
    # free box with sponges, per-cell material, Lambda != 0
    rng = np.random.default_rng(5)
    rho = rng.uniform(1.0, 2.0, size=(40, 130))
    lam2, mu2 = wl.lame(rng.uniform(0.2, 0.3, size=(40, 130)), rho)
    out.append(wl.Workload(name="freebox", nx=130, ny=40, nsteps=nsteps, storage=storage,
                           bc=("free", "free", "rigid", "rigid"), sponge=(2, 0, 0, 3),
                           rho0=rho, lam=lam2, mu=mu2,
                           sources=wl.source(60.0, 3.0, sigma=1.5, direction=(0.0, 1.0),
                                             f_peak=0.15, t0=6.0, r_cut=6.0)[None],
                           receivers=wl.surface_line(2, 120, 7)))
    return out


def _make(ws, storage, max_steps_traced=200):
    return [_pkg().from_workload(w, storage=storage, max_steps_traced=max_steps_traced)
            for w in ws]


def _state(sim):
    f = sim.read_fields(("ux", "uy", "rho", "pxx"), on_device=False)
    tr = sim.read_traces() if sim.traces_recorded() else np.zeros((0,))
    return f, tr


def _assert_same(a, b, what):
    fa, ta = a
    fb, tb = b
    for k in fa:
        assert np.array_equal(fa[k], fb[k]), f"{what}: field {k} differs"
    assert np.array_equal(ta, tb), f"{what}: traces differ"


MODES = [("stream", 8, 0, 1), ("stream", 4, 1, 1), ("graph", 8, 1, 1), ("graph", 4, 0, 1),
         ("persistent", 8, 1, 1), ("persistent", 4, 0, 1),
         ("stream", 8, 1, 2), ("stream", 8, 0, 2), ("graph", 8, 0, 2), ("graph", 4, 1, 2),
         ("persistent", 8, 1, 2), ("persistent", 8, 0, 2)]


@pytest.mark.parametrize("storage", ["f64", "f32", "f16", "bf16"])
@pytest.mark.parametrize("mode,rows,order,tps", MODES)
def test_batch_equals_shots_alone(storage, mode, rows, order, tps):
    """Every launch form, tile height, order and number of time steps per
    tile gives, bit for bit, what each shot gives when stepped alone (the
    step of a cell does not depend on the tile it is in, nor on whether its
    intermediate step went through shared memory).  23 steps: with two steps
    per tile the odd one is a one-step launch; graphs of 5 launches and
    persistent launches of 7 steps leave remainders."""
    ws = _shot_workloads(storage)
    alone = _make(ws, storage)
    for s in alone:
        s.step(23)
    ref = [_state(s) for s in alone]
    shots = _make(ws, storage)
    b = _pkg().Batch(shots)
    b.set_launch(mode=mode, rows=rows, order=order, graph_steps=5, steps_per_launch=7,
                 steps_per_tile=tps)
    assert b.launch["steps_per_tile"] == tps
    b.step(23)
    b.sync()
    for i, s in enumerate(shots):
        assert s.step_index == 23 and s.traces_recorded() == alone[i].traces_recorded()
        _assert_same(_state(s), ref[i], f"shot {i} ({ws[i].name})")
    assert b.kernel_launches > 0


def test_batch_interleaved_with_single_steps():
    """Batched calls pick up steps made on a shot alone in between."""
    ws = _shot_workloads("f32")
    alone = _make(ws, "f32")
    for s in alone:
        s.step(12)
    shots = _make(ws, "f32")
    b = _pkg().Batch(shots)
    b.set_launch(mode="graph", graph_steps=3)
    b.step(5)
    shots[1].step(3)
    b.set_launch(mode="persistent", steps_per_launch=2, steps_per_tile=2)
    b.step(4)
    shots[0].step(3)
    shots[2].step(3)
    shots[3].step(3)
    b.sync()
    for i, s in enumerate(shots):
        assert s.step_index == 12
        _assert_same(_state(s), _state(alone[i]), f"shot {i}")


def test_batch_matches_oracle():
    """A batch of two small shots against the FP64 oracle (FP64 storage)."""
    ws = _shot_workloads("f64", nsteps=30)[:2]
    shots = _make(ws, "f64")
    b = _pkg().Batch(shots)
    b.set_launch(mode="persistent", rows=8, steps_per_launch=30)
    b.step(30)
    b.sync()
    for w, s in zip(ws, shots):
        prob = oracle_problem(w)
        st, tro = oracle.run(prob, 30)
        f = s.read_fields(("ux", "uy"), on_device=False)
        assert rel_l2(np.stack([f["ux"], f["uy"]]), st.u) <= 1e-12, w.name
        if len(w.receivers):
            assert rel_l2(s.read_traces(), tro) <= 1e-12, w.name


def test_batch_autotune_advances_and_matches():
    """The autotuner times every candidate on the batch itself: the shots
    advance by (2 + trial, rounded up to even) x 18 steps and still equal
    shots stepped alone."""
    ws = _shot_workloads("f32", nsteps=80)
    shots = _make(ws, "f32")
    b = _pkg().Batch(shots)
    us = b.autotune(1)
    b.sync()
    assert us > 0
    assert b.launch["mode"] in ("stream", "graph", "persistent")
    assert b.launch["steps_per_tile"] in (1, 2)
    n = shots[0].step_index
    assert n == 72 and all(s.step_index == n for s in shots)
    alone = _make(ws, "f32")
    for s in alone:
        s.step(n)
    for i, s in enumerate(shots):
        _assert_same(_state(s), _state(alone[i]), f"shot {i}")


def test_batch_auto_mode_tunes_on_long_calls():
    ws = _shot_workloads("f32", nsteps=110)[:2]
    shots = _make(ws, "f32")
    b = _pkg().Batch(shots)
    assert b.launch["mode"] == "auto"
    b.step(100)
    b.sync()
    assert all(s.step_index == 100 for s in shots)
    alone = _make(ws, "f32")
    for s in alone:
        s.step(100)
    for i, s in enumerate(shots):
        _assert_same(_state(s), _state(alone[i]), f"shot {i}")


def test_batch_barrier_timeout_is_reported_and_recoverable():
    """A grid barrier that can never complete (it waits for one arrival more
    than the grid has) gives up after its cycle limit: the kernel returns,
    sync reports LBM_ERR_TIMEOUT and the context stays usable."""
    pkg = _pkg()
    ws = _shot_workloads("f32")[:2]
    shots = _make(ws, "f32")
    b = pkg.Batch(shots)
    b.set_launch(mode="persistent", barrier_extra=1, barrier_cycles=2_000_000,
                 steps_per_launch=3)
    b.step(3)
    with pytest.raises(pkg.LBMError) as e:
        b.sync()
    assert e.value.status == -6
    # a fresh batch on fresh shots runs normally afterwards
    shots2 = _make(ws, "f32")
    b2 = pkg.Batch(shots2)
    b2.set_launch(mode="persistent", barrier_extra=0, barrier_cycles=0)
    b2.step(5)
    b2.sync()
    alone = _make(ws, "f32")
    for s in alone:
        s.step(5)
    for i, s in enumerate(shots2):
        _assert_same(_state(s), _state(alone[i]), f"shot {i}")


def test_batch_rejects_mixed_storage_and_bad_launch():
    pkg = _pkg()
    ws = _shot_workloads("f32")[:2]
    a = pkg.from_workload(ws[0], storage="f32")
    c = pkg.from_workload(ws[1], storage="f64")
    with pytest.raises(pkg.LBMError) as e:
        pkg.Batch([a, c])
    assert e.value.status == -1
    b = pkg.Batch([a])
    for bad in ({"rows": 16}, {"order": 2}, {"graph_steps": 0}, {"steps_per_launch": 0},
                {"steps_per_tile": 3}, {"steps_per_tile": 0}):
        with pytest.raises(pkg.LBMError):
            b.set_launch(**bad)
