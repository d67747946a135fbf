"""Throughput benchmark of the elastic-solid D2Q9 LBM step on GB300.

Workload (one benchmark step = one full shot): the 2048 x 1024 half-space --
free surface on the top row, 64-cell absorbing layers on the left, right and
bottom, homogeneous Poisson solid (nu = 0.25), vertical Ricker x Gaussian force
10 cells below the surface, 256 surface receivers -- advanced 4000 time steps
in FP32 from rest, receivers recorded every step.  Metric: MLUPS (million
lattice-cell updates per second) = cells x time steps / time.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

One JSON line is printed by rank 0.  Timing: CUDA events on the library's
stream, a barrier and a synchronise on both sides of the K timed shots, the
maximum over ranks; L2 is flushed (a 256 MiB write) before every shot.  With N
GPUs each rank runs its own shot (independent replicas, weak scaling).
``--impl reference`` times the FP64 CPU oracle on the host cores instead, on
bounded samples of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "D2Q9 elastic-LBM MLUPS & % HBM roofline: plain vs batched/FP16-store/adjoint"
UNIT = "MLUPS"
# Algorithmic bytes per cell of one step-kernel launch without per-cell
# material: 9 populations read + 9 written + the displacement read + written
# (FP32: 9 x 4 x 2 + 2 x 4 x 2).  A one-step launch does this per time step; a
# two-step launch (intermediate populations in shared memory) per two.
BYTES_PER_CELL = {"f32": 9 * 4 * 2 + 2 * 4 * 2, "f64": 9 * 8 * 2 + 2 * 8 * 2}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi while running."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.t = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.gpu)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            if self.t is not None:
                self.t.join(timeout=2)

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def aggregate(elapsed_ms: float, units_per_rank: float, dist=None, device="cpu"):
    """Whole-job throughput of independent replicas: the slowest rank's time
    (max over ranks) and the units all ranks processed.  Returns
    (max_elapsed_ms, units_per_second)."""
    import torch
    world = dist.get_world_size() if dist is not None else 1
    t = torch.tensor([elapsed_ms], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    tmax = float(t.item())
    return tmax, world * units_per_rank / (tmax / 1e3)


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def cpu_oracle_sample(nsteps_sample: int, nthreads: int):
    """Times the FP64 CPU oracle on ``nsteps_sample`` steps of the half-space
    workload, starting from rest at step 40 (the source is firing).  Returns
    (MLUPS, seconds)."""
    import oracle
    from paper_2009_06404_gb300 import workloads as wl
    w = wl.halfspace()
    prob = oracle.Problem(nx=w.nx, ny=w.ny, tau=w.tau, bc_top=w.bc[0], bc_bottom=w.bc[1],
                          bc_left=w.bc[2], bc_right=w.bc[3], sponge=tuple(w.sponge),
                          sponge_amax=w.sponge_amax, fs_order=w.fs_order, rho0=w.rho0, lam=w.lam, mu=w.mu,
                          sources=w.sources, receivers=w.receivers, nthreads=nthreads)
    st = oracle.State(prob, n=40)
    t = time.perf_counter()
    oracle.run(prob, nsteps_sample, st)
    dt = time.perf_counter() - t
    return w.cells * nsteps_sample / dt / 1e6, dt


def run_reference(args):
    world, rank, _ = _dist()
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    nthreads = os.cpu_count() or 1
    sample = args.ref_sample_steps
    for _ in range(args.warmup):
        cpu_oracle_sample(sample, nthreads)
    vals, secs = [], []
    for _ in range(args.steps):
        v, dt = cpu_oracle_sample(sample, nthreads)
        vals.append(v)
        secs.append(dt)
    from paper_2009_06404_gb300 import workloads as wl
    w = wl.halfspace()
    total = w.cells * sample * args.steps / sum(secs) / 1e6
    desc = (f"FP64 oracle, {sample} time steps of the {w.nx}x{w.ny} half-space per step, "
            f"OpenMP over rows, {nthreads} threads")
    line = {
        "impl": "reference", "metric": METRIC, "value": total, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * sum(secs) / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "halfspace_2048x1024_fp32_4000steps", "nx": w.nx, "ny": w.ny,
                   "time_steps_per_step": sample, "note": "bounded sample of the workload"},
        "cpu_baseline": {"value": total, "unit": UNIT, "cores": nthreads, "kind": "oracle",
                         "sample": desc},
        "e2e": {"value": total, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_gpu(args):
    import torch
    import paper_2009_06404_gb300 as pkg
    from paper_2009_06404_gb300 import workloads as wl
    from paper_2009_06404_gb300 import build as _build

    world, rank, local = _dist()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    if not _build.up_to_date():
        if rank == 0:
            _build.build()
        if dist is not None:
            dist.barrier()
    pkg.load_library()

    storage = args.storage
    w = wl.halfspace(nsteps=args.time_steps, storage=storage)
    stream = torch.cuda.current_stream()
    sim = pkg.from_workload(w, max_steps_traced=w.nsteps, stream=stream)
    spl = args.steps_per_launch
    sim.set_steps_per_launch(spl)
    # step-kernel launches per shot (Lambda = 0 here, so two-step launches apply)
    step_launches = w.nsteps // spl + w.nsteps % spl
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def shot(ev_pair=None):
        sim.reset()
        if ev_pair is not None:
            ev_pair[0].record(stream)
        sim.step(w.nsteps)
        if ev_pair is not None:
            ev_pair[1].record(stream)

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # --------------------------------------------------- device-resident timing
    for _ in range(args.warmup):
        flush.fill_(1)
        shot()
    barrier()
    launches0 = sim.kernel_launches
    step_events = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                   for _ in range(args.steps)]
    t_start = torch.cuda.Event(enable_timing=True)
    t_stop = torch.cuda.Event(enable_timing=True)
    gpu_index = local
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        try:
            gpu_index = int(vis.split(",")[local])
        except ValueError:
            pass
    with ClockSampler(gpu_index) as clk:
        barrier()
        elapsed = 0.0
        kernel_ms = 0.0
        for k in range(args.steps):
            flush.fill_(k & 0xFF)  # L2 flush, outside the shot's events
            e0, e1 = step_events[k]
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            shot((e0, e1))
            b.record(stream)
            torch.cuda.synchronize()
            elapsed += a.elapsed_time(b)
            kernel_ms += e0.elapsed_time(e1)
        barrier()
    sim.sync()
    gpu_launches = sim.kernel_launches - launches0
    cells_steps = w.cells * w.nsteps
    elapsed_max, rate = aggregate(elapsed, cells_steps * args.steps, dist, "cuda")
    value = rate / 1e6

    # --------------------------------------------------- end to end (host buffers)
    rho0, lam, mu = (np.ascontiguousarray(a) for a in (w.rho0, w.lam, w.mu))
    src = np.ascontiguousarray(w.sources)
    rec = np.ascontiguousarray(w.receivers)
    tr_host = torch.empty((w.nsteps, len(rec), 4), dtype=torch.float64).pin_memory()
    u_host = [torch.empty((w.ny, w.nx), dtype=torch.float64).pin_memory() for _ in range(2)]
    h2d = rho0.nbytes + lam.nbytes + mu.nbytes + src.nbytes + rec.nbytes
    d2h = tr_host.numel() * 8 + sum(u.numel() * 8 for u in u_host)

    def e2e_shot():
        sim.set_material(rho0, lam, mu)
        sim.set_sources(src)
        sim.set_receivers(rec)
        sim.reset()
        sim.step(w.nsteps)
        sim.read_traces(out=tr_host.numpy())
        f = sim.L.lbm_elastic_read_fields(sim.h, u_host[0].data_ptr(), u_host[1].data_ptr(),
                                          None, None, None, None, None, None, 0)
        sim._check(f)

    for _ in range(max(1, args.warmup // 2)):
        flush.fill_(3)
        e2e_shot()
    barrier()
    e2e_ms = 0.0
    for k in range(args.steps):
        flush.fill_(k & 0xFF)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        e2e_shot()
        b.record(stream)
        torch.cuda.synchronize()
        e2e_ms += a.elapsed_time(b)
    _, e2e_rate = aggregate(e2e_ms, cells_steps * args.steps, dist, "cuda")
    e2e_value = e2e_rate / 1e6

    # --------------------------------------------------- the one-step kernel, same shots
    one_step_ms, one_step_shots = None, min(args.steps, 3)
    if spl == 2:
        sim.set_steps_per_launch(1)
        flush.fill_(2)
        shot()
        one_step_ms = 0.0
        for k in range(one_step_shots):
            flush.fill_(k & 0xFF)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            shot((e0, e1))
            torch.cuda.synchronize()
            one_step_ms += e0.elapsed_time(e1)
        sim.set_steps_per_launch(spl)

    # --------------------------------------------------- roofline of the step kernel
    peak, peak_kind = _peaks()
    # a launch moves every population and the displacement once each way,
    # whether it advances one time step or two
    avg_launch_s = kernel_ms / 1e3 / (args.steps * step_launches)
    bytes_launch = BYTES_PER_CELL[storage] * w.cells
    achieved = bytes_launch / avg_launch_s / 1e9
    kname = "step2_kernel" if spl == 2 else "step_kernel"
    one_step = None
    if one_step_ms is not None:
        l1_s = one_step_ms / 1e3 / (one_step_shots * w.nsteps)
        one_step = {"kernel": "step_kernel", "shots": one_step_shots,
                    "mlups": w.cells / l1_s / 1e6, "avg_launch_us": l1_s * 1e6,
                    "achieved": bytes_launch / l1_s / 1e9, "frac": bytes_launch / l1_s / 1e9 / peak}
    traffic = None
    prof = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(prof):
        try:
            with open(prof) as f:
                d = json.load(f)
            key = f"{'step2' if spl == 2 else 'step'}_{storage}_{w.nx}x{w.ny}"
            if key in d and d[key].get("kernel_hash") == _build.source_hash(_build.STEP_SOURCES):
                traffic = d[key]["dram_bytes_per_launch"]
        except Exception:
            traffic = None

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0

    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        nthreads = os.cpu_count() or 1
        v, dt = cpu_oracle_sample(args.cpu_sample_steps, nthreads)
        cpu = {"value": v, "unit": UNIT, "cores": nthreads, "kind": "oracle",
               "sample": f"{args.cpu_sample_steps} time steps of the {w.nx}x{w.ny} half-space "
                         f"(FP64 oracle, OpenMP over rows), {dt:.1f} s"}

    forms = None
    if world == 1 and not args.no_forms:
        forms = measure_forms(torch, pkg, wl)
        forms["plain"] = {"workload": "halfspace_2048x1024, FP32", "mlups": value}

    clocks = clk.summary()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": elapsed_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if storage == "f32" else storage, "data": "synthetic",
        "config": {"workload": "halfspace_2048x1024_fp32_4000steps", "nx": w.nx, "ny": w.ny,
                   "time_steps_per_step": w.nsteps, "storage": storage,
                   "free_surface": "top",
                   "free_surface_extrapolation": ("constant (the paper's linear form, "
                                                  "Eq. 39, grows without bound at tau = 1)"
                                                  if w.fs_order == 0 else "linear (Eq. 39)"),
                   "absorbing_layers": "left,right,bottom x64",
                   "receivers": len(w.receivers), "parallelism": f"replicas x{world}",
                   "l2": "flushed before every timed shot (256 MiB write)"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "peak_kind": peak_kind, "kernel": kname,
                     "steps_per_launch": spl,
                     "bytes_per_cell_per_launch": BYTES_PER_CELL[storage],
                     "bytes_per_cell_step": BYTES_PER_CELL[storage] / spl,
                     "avg_launch_us": avg_launch_s * 1e6,
                     # the same launches counted at the one-step figure of
                     # BYTES_PER_CELL per cell and time step (above 1: the
                     # two-step kernel moves fewer bytes than one step would)
                     "frac_at_one_step_bytes": achieved * spl / peak,
                     "one_step_kernel": one_step},
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": UNIT,
                "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
        "clocks": clocks,
        "gpu_launches": int(gpu_launches),
        "forms": forms,
    }
    print(json.dumps(line), flush=True)
    sim.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


def _ev(torch):
    return torch.cuda.Event(enable_timing=True)


def _timed(torch, fn) -> float:
    """Milliseconds of fn() on the current stream (synchronised both sides)."""
    torch.cuda.synchronize()
    a, b = _ev(torch), _ev(torch)
    a.record()
    fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b)


def _rel_l2(a, b) -> float:
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


# Error budget of a storage format: relative L2 error of u and of v against
# the FP64 run after 2000 steps.  A tenth of the smallest discretisation error
# the paper reports for the method itself (Table 1: 0.0349 relative L2 of j
# at 512^2), so that storage rounding adds under 1 % to the method's own
# error (in quadrature).
ERROR_BUDGET_REL_L2 = 3.5e-3


def form_precision(torch, pkg, wl, n=8192, steps=2000, time_steps=2000, err_n=1024):
    """FP16 / BF16 population storage (FP32 arithmetic) against FP32 storage
    on the periodic 8-layer, 16-source grid: MLUPS over time_steps steps at
    n x n, and the relative L2 error of u and v after `steps` steps against
    an FP64 run of the same generator at err_n x err_n (that FP64 run equals
    the CPU oracle's to 1e-12, tests/test_gpu_fullsize.py), with a verdict
    against ERROR_BUDGET_REL_L2."""
    scale = {"f32": 0, "f16": 10, "bf16": 0, "f64": 0}
    w = wl.periodic_layered_multisource(n=n, nsteps=time_steps)
    mlups, alt = {}, {}
    for st in ("f32", "f16", "bf16"):
        sim = pkg.from_workload(w, storage=st, store_scale_log2=scale[st], max_steps_traced=0)
        sim.step(20)
        ms = _timed(torch, lambda: sim.step(time_steps))
        mlups[st] = w.cells * time_steps / ms / 1e3
        if st == "f16":
            # the other launch form of 16-bit storage with Lambda != 0 (the
            # library's default for it is one step per launch)
            sim.set_steps_per_launch(2)
            sim.step(20)
            ms = _timed(torch, lambda: sim.step(min(time_steps, 400)))
            alt["f16_two_steps_per_launch"] = w.cells * min(time_steps, 400) / ms / 1e3
        sim.sync()
        sim.close()
        del sim
    we = wl.periodic_layered_multisource(n=err_n, nsteps=steps)
    fields = {}
    for st in ("f64", "f32", "f16", "bf16"):
        sim = pkg.from_workload(we, storage=st, store_scale_log2=scale[st], max_steps_traced=0)
        sim.step(steps)
        f = sim.read_fields(("ux", "uy", "vx", "vy"), on_device=False)
        fields[st] = (np.stack([f["ux"], f["uy"]]), np.stack([f["vx"], f["vy"]]))
        sim.close()
    err_u = {st: _rel_l2(fields[st][0], fields["f64"][0]) for st in ("f32", "f16", "bf16")}
    err_v = {st: _rel_l2(fields[st][1], fields["f64"][1]) for st in ("f32", "f16", "bf16")}
    ok = {st: bool(err_u[st] <= ERROR_BUDGET_REL_L2 and err_v[st] <= ERROR_BUDGET_REL_L2)
          for st in ("f32", "f16", "bf16")}
    return {"workload": f"periodic_layered_{n}x{n}_8layers_16src", "time_steps": time_steps,
            "mlups": mlups, "mlups_other_launch_form": alt,
            "speedup_vs_f32": {k: mlups[k] / mlups["f32"] for k in ("f16", "bf16")},
            "error": {"vs": f"FP64 GPU run, same generator at {err_n}x{err_n}, {steps} steps "
                            "(equal to the CPU oracle to 1e-12)",
                      "rel_l2_u": err_u, "rel_l2_v": err_v,
                      "budget_rel_l2": ERROR_BUDGET_REL_L2, "within_budget": ok},
            "store_scale_log2": {k: scale[k] for k in ("f16", "bf16")}}


def form_batched(torch, pkg, wl, nshots=64, time_steps=2000):
    """64 uneven layered shots (65.0 M cells) advanced together, against the
    same shots stepped one after another."""
    ws = wl.batch_shots(nshots, nsteps=2000)
    shots = [pkg.from_workload(w, max_steps_traced=0) for w in ws]
    cells = sum(w.cells for w in ws)

    def plain(nt):
        for sh in shots:
            sh.step(nt)

    plain(20)
    plain_ms = _timed(torch, lambda: plain(time_steps))
    b = pkg.Batch(shots)
    best_us = b.autotune(10)  # 18 candidates x 12 steps
    launch = b.launch
    b.step(20)
    batch_ms = _timed(torch, lambda: b.step(time_steps))
    b.sync()
    launches = b.kernel_launches
    plain_m = cells * time_steps / plain_ms / 1e3
    batch_m = cells * time_steps / batch_ms / 1e3
    out = {"workload": f"{nshots} layered half-space shots, sizes 512^2..2048x1024, "
                       f"{cells} cells, FP32", "time_steps": time_steps,
           "mlups": batch_m, "plain_mlups": plain_m, "speedup_vs_plain": batch_m / plain_m,
           "launch": {k: launch[k] for k in ("mode", "rows", "order", "steps_per_tile")},
           "autotune_best_us_per_step": best_us, "kernel_launches": launches,
           "error": "bit-identical to the shots stepped alone (tested)"}
    b.close()
    for sh in shots:
        sh.close()
    return out


def form_adjoint(torch, pkg, wl, nx=1024, ny=512, steps=3000, every=100,
                 storages=("f64", "f32")):
    """Gradient of the trace misfit of the blob model against the layered
    model with respect to lambda, mu per cell and the source amplitude:
    forward with checkpoints plus reverse sweep, FP32 states with FP64
    gradient sums, against the plain FP32 forward; error of the FP32 lambda
    gradient against the FP64 one."""
    from paper_2009_06404_gb300.autograd import SimulationSetup, simulate_traces
    base, pert = wl.fwi_blob(nx, ny, steps)
    res = {}
    grads = {}
    # FP64 first: it also loads torch's backward kernels for the misfit, so
    # the FP32 timing sees no one-time module loading; last, FP32 with one
    # segment (every gradient record kept in HBM: no recomputation)
    runs = [(st, every) for st in storages] + [("f32_all", steps)]
    for key, every_k in runs:
        st = key[:3]
        setup = SimulationSetup(pert, steps, every_k, st)
        dev = "cuda"
        amp = torch.ones(1, dtype=torch.float64, device=dev)
        with torch.no_grad():
            d = simulate_traces(torch.as_tensor(base.lam, device=dev),
                                torch.as_tensor(base.mu, device=dev), amp, setup)
        lam = torch.as_tensor(pert.lam, device=dev).requires_grad_(True)
        mu = torch.as_tensor(pert.mu, device=dev).requires_grad_(True)
        tr = [None]

        def fwd():
            tr[0] = simulate_traces(lam, mu, amp, setup)

        t_f = _timed(torch, fwd)
        J = 0.5 * ((tr[0][..., :2] - d[..., :2]) ** 2).sum()
        t_b = _timed(torch, J.backward)
        grads[key] = lam.grad.cpu().numpy()
        res[key] = (t_f, t_b)
        del setup, lam, mu, tr, J
        torch.cuda.empty_cache()
    sim = pkg.from_workload(pert, storage="f32", max_steps_traced=steps)
    sim.step(100)
    plain_ms = _timed(torch, lambda: sim.step(steps))
    sim.close()
    cells = nx * ny
    t_f, t_b = res["f32"]
    adj_m = cells * steps / (t_f + t_b) / 1e3
    plain_m = cells * steps / plain_ms / 1e3
    err = (_rel_l2(grads["f32"], grads["f64"]) if "f64" in grads else None)
    t_f2, t_b2 = res["f32_all"]
    all_m = cells * steps / (t_f2 + t_b2) / 1e3
    return {"workload": f"fwi_blob_{nx}x{ny}, {steps} steps, checkpoints every {every}, "
                        "128 receivers, FP32 states, FP64 gradient sums",
            "mlups": adj_m, "plain_mlups": plain_m, "speedup_vs_plain": adj_m / plain_m,
            "forward_ms": t_f, "backward_ms": t_b,
            "error": {"rel_l2_grad_lambda_f32_vs_f64": err},
            "no_recompute": {"checkpoint_every": steps, "mlups": all_m,
                             "speedup_vs_plain": all_m / plain_m,
                             "forward_ms": t_f2, "backward_ms": t_b2,
                             "gradient_equal_bitwise": bool(np.array_equal(grads["f32_all"],
                                                                           grads["f32"]))}}


def form_plain_large(torch, pkg, wl, n=8192, time_steps=2000):
    """The plain FP32 step (the library's default launch form) on an n x n
    periodic grid whose 5.9 GB of state is far beyond L2: the 8-layer,
    16-source generator as it is (Lambda != 0, density-gradient force) and
    with every layer a Poisson solid (Lambda = 0).  MLUPS and the fraction
    of the measured HBM peak at 88 algorithmic bytes per cell and time step."""
    peak, peak_kind = _peaks()
    out = {"workload": f"periodic {n}x{n}, 8 layers, 16 sources, FP32, {time_steps} steps",
           "peak": peak, "peak_kind": peak_kind,
           "bytes_per_cell_step": BYTES_PER_CELL["f32"]}
    w = wl.periodic_layered_multisource(n=n, nsteps=time_steps)
    for key, wk in (("lambda_nonzero", w),
                    ("lambda_zero", w.with_(lam=np.asarray(w.mu, np.float64).copy()))):
        sim = pkg.from_workload(wk, storage="f32", max_steps_traced=0)
        sim.step(20)
        ms = _timed(torch, lambda: sim.step(time_steps))
        sim.sync()
        mlups = wk.cells * time_steps / ms / 1e3
        gbs = BYTES_PER_CELL["f32"] * mlups * 1e6 / 1e9
        out[key] = {"mlups": mlups, "ms": ms, "achieved_gbs_at_88B": gbs,
                    "frac_at_88B": gbs / peak,
                    "kernel": "step2_kernel" if key == "lambda_zero" else "step2_lam_kernel"}
        sim.close()
        del sim
        torch.cuda.empty_cache()
    return out


def measure_forms(torch, pkg, wl):
    out = {}
    for name, fn in (("plain_large", form_plain_large), ("batched", form_batched),
                     ("precision", form_precision), ("adjoint", form_adjoint)):
        try:
            out[name] = fn(torch, pkg, wl)
        except Exception as e:  # a failing form must not cost the headline line
            out[name] = {"error": f"{type(e).__name__}: {e}"}
        torch.cuda.empty_cache()
    return out


def run_form(args):
    """One form alone (its JSON object), e.g. for a profiler capture."""
    import torch
    import paper_2009_06404_gb300 as pkg
    from paper_2009_06404_gb300 import workloads as wl
    from paper_2009_06404_gb300 import build as _build
    if not _build.up_to_date():
        _build.build()
    pkg.load_library()
    if args.form == "batched":
        out = form_batched(torch, pkg, wl, nshots=args.nshots, time_steps=args.form_steps or 2000)
    elif args.form == "plain_large":
        out = form_plain_large(torch, pkg, wl, n=args.prec_n, time_steps=args.form_steps or 2000)
    elif args.form == "precision":
        out = form_precision(torch, pkg, wl, n=args.prec_n, steps=args.prec_err_steps,
                             time_steps=args.form_steps or 2000, err_n=args.prec_err_n)
    else:
        out = form_adjoint(torch, pkg, wl, nx=args.adj_nx, ny=args.adj_ny,
                           steps=args.form_steps or 3000, every=args.adj_every,
                           storages=tuple(args.adj_storages.split(",")))
    print(json.dumps({"form": args.form, **out}), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--storage", default="f32", choices=["f32", "f64"])
    ap.add_argument("--time-steps", type=int, default=4000)
    ap.add_argument("--steps-per-launch", type=int, default=2, choices=[1, 2],
                    help="time steps per step-kernel launch (2: the two-step kernel)")
    ap.add_argument("--cpu-sample-steps", type=int, default=100)
    ap.add_argument("--ref-sample-steps", type=int, default=10)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the 8192^2 plain / batched / 16-bit / adjoint form measurements")
    ap.add_argument("--form", choices=["plain_large", "batched", "precision", "adjoint"],
                    help="measure only this form and print its JSON object")
    ap.add_argument("--form-steps", type=int, default=0,
                    help="time steps of the form (0: its default)")
    ap.add_argument("--nshots", type=int, default=64)
    ap.add_argument("--prec-n", type=int, default=8192)
    ap.add_argument("--prec-err-n", type=int, default=1024)
    ap.add_argument("--prec-err-steps", type=int, default=2000)
    ap.add_argument("--adj-nx", type=int, default=1024)
    ap.add_argument("--adj-ny", type=int, default=512)
    ap.add_argument("--adj-every", type=int, default=100)
    ap.add_argument("--adj-storages", default="f64,f32",
                    help="storage types of the adjoint form, f32 last (f64,f32 or f32)")
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    if args.form:
        return run_form(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
