"""Benchmark of the fused MDF-FDLBM step (one JSON line on rank 0).

Workload: periodic Taylor-Green vortex on a 4096 x 4096 uniform grid, FP32
state and arithmetic, nu = 0.01, U0 = 0.01, CFL 0.5, eta = 0.8, s'/s = 1.5.
One bench step = one time step of the method over the whole grid (one fused
kernel launch).  The two state buffers (2 x 692 MB) are far larger than L2, so
every step streams the state from HBM; no L2 flush is needed.

  value      MLUPS (million lattice-node updates per second) of the whole job,
             device-timed with CUDA events on the solver's stream
  e2e        the same metric through the C ABI with host buffers: upload of
             the initial fields from pinned host memory, the steps, and the
             download of u, v, p to pinned host memory, all inside the timed
             region
  roofline   HBM roofline of the fused step: algorithmic bytes per node
             update (state read once + written once) x nodes / launch time,
             against the measured copy bandwidth of this GPU type
  cpu_baseline  the FP64 CPU oracle timed on a bounded sample (rank 0, N = 1)

--impl reference times the FP64 CPU oracle on the host cores instead (the
reference arm of this method: there is no other implementation to run).
Multi-GPU runs (torchrun, one rank per GPU) are independent replicas of the
workload (weak scaling); the method needs no exchange between them.
"""
import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MLUPS & % HBM roofline; time-to-residual 1e-8, warm-start+batch vs cold"
NX = NY = 4096
NU, U0 = 0.01, 0.01
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "step_taylor_green_4096_traffic.json")
STEP_SOURCE = os.path.join(ROOT, "paper_2306_08216_gb300", "csrc", "mdf_step_fast.cu")


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index, period_ms=50):
        self.gpu = gpu_index
        self.period_ms = period_ms
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.QUERY, "--format=csv,noheader,nounits",
                 "-lms", str(self.period_ms)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def finite_json(x):
    """The bench line as strict JSON: non-finite floats (a residual never
    reached, a diverged problem) become null."""
    if isinstance(x, float):
        return x if math.isfinite(x) else None
    if isinstance(x, dict):
        return {k: finite_json(v) for k, v in x.items()}
    if isinstance(x, (list, tuple)):
        return [finite_json(v) for v in x]
    return x


def max_over_ranks(x, world, device="cpu"):
    """Max of a per-rank scalar over all ranks (identity for one rank)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_mlups(nodes, steps, world, seconds_max):
    """Whole-job throughput: every rank updates `nodes` nodes `steps` times;
    the job takes as long as its slowest rank."""
    return world * nodes * steps / seconds_max / 1e6


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fp:
            d = json.load(fp)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def ncu_traffic_per_launch():
    """DRAM bytes per launch of the step kernel from the committed ncu summary,
    or None if the summary is missing or was taken on another kernel source."""
    try:
        with open(TRAFFIC_FILE) as fp:
            d = json.load(fp)
        with open(STEP_SOURCE, "rb") as fp:
            digest = hashlib.sha256(fp.read()).hexdigest()[:16]
    except (OSError, ValueError):
        return None
    if d.get("source_sha256_16") != digest:
        return None
    return d.get("dram_bytes_per_launch")


def oracle_sample(steps, n=512):
    """FP64 oracle on an n x n Taylor-Green grid: (MLUPS, threads, seconds)."""
    from oracle.oracle import Oracle, max_threads
    from paper_2306_08216_gb300 import workloads as W
    o = Oracle(n, n, nu=NU, lx=2 * math.pi, ly=2 * math.pi)
    o.init(*W.taylor_green(n, U0))
    o.step(1)
    t0 = time.perf_counter()
    o.step(steps)
    dt = time.perf_counter() - t0
    return n * n * steps / dt / 1e6, max_threads(), dt


CAV_N, CAV_RE, CAV_U0 = 257, 1000.0, 0.1
CLOCK_WINDOW_MS = 1500.0


def time_to_residual(mdf, W, grid, stream, target=1e-8, check_every=100, max_steps=3_000_000):
    """Cold start from rest to residual <= target (windowed residual of
    mdf_residual, window `check_every` steps); wall-clock seconds including
    the residual checks and the one window enqueued after the last check."""
    kw = dict(nu=CAV_U0 / CAV_RE, walls=(True, True), u_wall=(0, 0, 0, CAV_U0), stream=stream)
    if grid.startswith("tanh"):
        xs = W.tanh_nodes(CAV_N, 1.5)
        kw.update(grid="separable", x=xs, y=xs)
    s = mdf.Solver(CAV_N, CAV_N, **kw)
    s.init(*W.zeros(CAV_N, CAV_N))
    s.synchronize()
    t0 = time.perf_counter()
    # the check of each window is read while the next window runs
    # (residual_start / residual_finish); the march stops at the first check
    # at or below the target, and the clock includes the window enqueued
    # behind it
    s.step(check_every)
    steps = check_every
    s.residual_start()
    while True:
        more = steps < max_steps
        if more:
            s.step(check_every)
        r, _ = s.residual_finish()
        if r <= target or not more:
            break
        steps += check_every
        s.residual_start()
    s.synchronize()
    sec = time.perf_counter() - t0
    out = {"workload": "lid-driven cavity Re=%g, %dx%d nodes, %s grid, from rest" % (CAV_RE, CAV_N, CAV_N, grid),
           "target": target, "reached": r <= target, "residual": r, "steps": steps, "seconds": sec,
           "us_per_step": 1e6 * sec / steps, "launch": s.launch_info()}
    s.close()
    return out


BATCH_COUNT, BATCH_SEED = 512, 2306


def batch_problems(count=BATCH_COUNT, seed=BATCH_SEED, u0=0.1):
    """Seeded sweep of power-law lid-driven cavities: Re log-uniform in
    [100, 5000], n uniform in [0.5, 1.5], side in {65, 129, 257, 513};
    K = u0^(2-n) L^n / Re with L = 1, nu clamped to [nu_ref/20, 20 nu_ref],
    nu_ref = K (u0/L)^(n-1)."""
    from paper_2306_08216_gb300 import workloads as W
    re, nn, sides = W.cavity_batch_draws(count, seed)
    probs = []
    for Re, n, side in zip(re, nn, sides):
        K = u0 ** (2 - n) / Re
        nu_ref = K * u0 ** (n - 1)
        probs.append(dict(nx=int(side), ny=int(side), nu=nu_ref, walls=(True, True), u_wall=(0, 0, 0, u0),
                          power_law=(K, float(n), nu_ref / 20, nu_ref * 20)))
    return probs


def batch_benchmark(mdf, torch, stream, steps=200, solo_sample=BATCH_COUNT, count=BATCH_COUNT):
    """Throughput of the batched step over the seeded 512-cavity sweep, against
    the same cavities stepped one problem per launch, each by its own
    autotuned single-problem solver for the same steps (every cavity by
    default; with solo_sample < count a sample spread over the sweep, scaled
    by node count)."""
    probs = batch_problems(count)
    t0 = time.perf_counter()
    batch = mdf.Batch(probs, stream=stream)
    create_s = time.perf_counter() - t0
    batch.step(2)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    batch.step(steps)
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    info = batch.info()
    r, status = batch.residual()
    nodes = info["nodes"]
    batch_mlups = nodes * steps / (ms / 1e3) / 1e6
    # the same sweep with 16-bit deviation storage (tile mode): throughput and
    # the largest velocity deviation from the FP32 batch after the same steps,
    # on the first cavity of every side
    import numpy as np
    sides = sorted({p["nx"] for p in probs})
    sample = [next(i for i, p in enumerate(probs) if p["nx"] == sd) for sd in sides]
    u32 = {i: batch.problem(i).fields(["u"])["u"].astype(np.float64) for i in sample}
    storage = {}
    for mode in ("fp16", "bf16"):
        b16 = mdf.Batch([dict(p, storage=mode) for p in probs], stream=stream)
        b16.step(2)
        torch.cuda.synchronize()
        e0.record(stream)
        b16.step(steps)
        e1.record(stream)
        e1.synchronize()
        ms16 = e0.elapsed_time(e1)
        r16, st16 = b16.residual()
        du = max(float(np.abs(b16.problem(i).fields(["u"])["u"] - u32[i]).max()) for i in sample) / 0.1
        storage[mode] = {"mlups": nodes * steps / (ms16 / 1e3) / 1e6, "ms_per_step": ms16 / steps,
                         "kernel": b16.info()["kernel"], "bytes_per_node": 56.0,
                         "diverged": int((st16 == mdf.MDF_E_DIVERGED).sum()),
                         "max_du_vs_fp32_batch_over_u_lid": du, "du_sample": "first cavity of each side %s" % sides}
        b16.close()
    batch_kernel = info["kernel"]
    batch.close()
    # one-problem-per-launch reference: every cavity, or a sample spread over
    # the sweep (largest and smallest mixed)
    idx = list(range(0, len(probs), max(1, len(probs) // solo_sample)))[:solo_sample]
    solo_nodes, solo_ms = 0, 0.0
    for i in idx:
        kw = dict(probs[i])
        nx, ny = kw.pop("nx"), kw.pop("ny")
        sv = mdf.Solver(nx, ny, stream=stream, **kw)
        sv.step(2)
        sv.synchronize()
        e0.record(stream)
        sv.step(steps)
        e1.record(stream)
        e1.synchronize()
        solo_ms += e0.elapsed_time(e1)
        solo_nodes += nx * ny
        sv.close()
    solo_mlups = solo_nodes * steps / (solo_ms / 1e3) / 1e6
    return {"workload": "%d power-law cavities, sides {65,129,257,513}, Re log-uniform [100,5000], "
                        "n uniform [0.5,1.5], seed %d" % (count, BATCH_SEED),
            "steps": steps, "nodes": nodes, "ms_per_step": ms / steps, "value": batch_mlups, "unit": "MLUPS",
            "launches_per_step": 1, "work_items": info["work_items"], "blocks": info["blocks"],
            "kernel": batch_kernel, "storage": storage,
            "diverged": int((status == mdf.MDF_E_DIVERGED).sum()), "create_seconds": create_s,
            "one_launch_per_problem_mlups": solo_mlups, "solo_sample": len(idx),
            "speedup_vs_one_launch_per_problem": batch_mlups / solo_mlups}


def storage_benchmark(mdf, W, torch, stream, ref_solver, nx, steps=500, warmup=20):
    """The same Taylor-Green workload with 16-bit deviation storage (FP32
    u, v, P plus the non-equilibrium part in FP16 / BF16): device-timed
    MLUPS, achieved bandwidth of the algorithmic bytes, and the largest
    velocity deviation from the FP32 run after the same steps."""
    u, v, p = W.taylor_green(nx, U0)
    ref_solver.init(u, v, p)
    ref_solver.step(warmup + steps)
    u32 = ref_solver.fields(["u"])["u"]
    peak, _ = measured_peaks()
    out = {}
    for mode in ("fp16", "bf16"):
        s = mdf.Solver(nx, nx, nu=NU, lx=2 * math.pi, ly=2 * math.pi, stream=stream, storage=mode)
        s.init(u, v, p)
        s.step(warmup)
        s.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.step(steps)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1) / steps
        bpn = s.bytes_per_node()
        gbs = bpn * nx * nx / (ms / 1e3) / 1e9
        du = float(abs(s.fields(["u"])["u"].astype("float64") - u32).max())
        out[mode] = {"mlups": nx * nx / (ms / 1e3) / 1e6, "ms_per_step": ms, "bytes_per_node": bpn,
                     "achieved_gbs": gbs, "frac": gbs / peak, "max_du_vs_fp32_over_U0": du / U0,
                     "steps": warmup + steps, "launch": s.launch_info()}
        del s
    return out


def rho0_benchmark(mdf, W, torch, stream, nx, steps=300, warmup=20):
    """The Taylor-Green workload with the alpha = 0 distribution of Eq. 2.1.2
    evolved beside alpha = 1, 2 (rho_0 = 1 + 0.1 sin 2 pi x cos 2 pi y; 15
    FP32 planes; the kernel the autotuner picks: the periodic register-window
    march with the scalar lane, or the tile kernel): device-timed MLUPS, the
    fraction of the measured copy bandwidth at 120 B per node, and the
    change of total rho_0 (conserved on a periodic grid without source)."""
    import numpy as np
    u, v, p = W.taylor_green(nx, U0)
    X, Y = np.meshgrid(np.arange(nx) / nx, np.arange(nx) / nx)
    s = mdf.Solver(nx, nx, nu=NU, lx=2 * math.pi, ly=2 * math.pi, stream=stream, rho0=True)
    s.init(u, v, p)
    s.init_rho0(1 + 0.1 * np.sin(2 * math.pi * X) * np.cos(2 * math.pi * Y))
    m0 = float(s.rho0().astype(np.float64).sum())
    s.step(warmup)
    s.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s.step(steps)
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1) / steps
    bpn = s.bytes_per_node()
    gbs = bpn * nx * nx / (ms / 1e3) / 1e9
    peak, _ = measured_peaks()
    m1 = float(s.rho0().astype(np.float64).sum())
    out = {"workload": "taylor_green_%dx%d_fp32_rho0" % (nx, nx), "mlups": nx * nx / (ms / 1e3) / 1e6,
           "ms_per_step": ms, "bytes_per_node": bpn, "achieved_gbs": gbs, "frac": gbs / peak,
           "rho0_total_rel_change": (m1 - m0) / m0, "steps": warmup + steps, "launch": s.launch_info()}
    del s
    return out


def body_fitted_benchmark(mdf, W, torch, stream, n=513, steps=300, warmup=20, u0=0.1):
    """Power-law lid-driven cavities on the body-fitted trapezoid grid
    (n x n nodes, metric coefficients in FP64 at set-up, curvilinear
    kernel): device-timed MLUPS and the fraction of the measured copy
    bandwidth at the algorithmic bytes (state + 4 metric planes), for
    n_index in {0.5, 1, 1.5} and Re in {100, 400, 1000}."""
    X, Y = W.trapezoid_grid(n, n)
    peak, _ = measured_peaks()
    out = []
    for n_index in (0.5, 1.0, 1.5):
        for re in (100.0, 400.0, 1000.0):
            K = u0 ** (2.0 - n_index) / re  # Re = u0^(2-n) L^n / K, L = 1 (lid width)
            nu_ref = K * u0 ** (n_index - 1.0)
            s = mdf.Solver(n, n, nu=nu_ref, grid="curvilinear", x=X, y=Y, walls=(True, True),
                           u_wall=(0, 0, 0, u0), power_law=(K, n_index, nu_ref / 20, nu_ref * 20), stream=stream)
            s.init(*W.zeros(n, n))
            s.step(warmup)
            s.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            s.step(steps)
            e1.record(stream)
            e1.synchronize()
            ms = e0.elapsed_time(e1) / steps
            bpn = s.bytes_per_node()
            gbs = bpn * n * n / (ms / 1e3) / 1e9
            try:
                r, _ = s.residual()
            except mdf.MdfError as e:
                r = "diverged (%s)" % e
            out.append({"n_index": n_index, "Re": re, "mlups": n * n / (ms / 1e3) / 1e6, "ms_per_step": ms,
                        "bytes_per_node": bpn, "achieved_gbs": gbs, "frac": gbs / peak, "residual": r})
            s.close()
    return {"workload": "power-law lid-driven cavity, isosceles trapezoid (lid 1, bottom 0.5, height 1), "
                        "%dx%d nodes, curvilinear kernel" % (n, n), "steps": steps, "runs": out}


def warm_start_benchmark(stream, per_side=2, target=1e-6, max_steps=400_000):
    """Learned warm start + batching against cold starts on a stratified
    subset of the seeded 512-cavity sweep: the first `per_side` cavities of
    each side (65, 129, 257, 513) of the steady subset recorded with the
    shipped network (cavities with Re <= 1000, the range it is trained on,
    whose flow reaches `target` from rest).  The network's 128 x 128
    prediction resampled to every cavity's grid starts one batch, the same
    cavities from rest another, and each cavity is also marched from rest by
    itself (one launch per problem and step); every arm measured."""
    import os

    from paper_2306_08216_gb300 import warmstart as WS
    with open(os.path.join(WS.WEIGHTS_DIR, "warmstart_cavity_R128.json")) as fp:
        rep = json.load(fp)
    steady, sides = rep["sweep"]["indices"], rep["sweep"]["sides"]
    idx = []
    for side in (65, 129, 257, 513):
        idx += [i for i, sd in zip(steady, sides) if sd == side][:per_side]
    net = WS.Net(128, 16, stream=stream)
    net.load(os.path.join(WS.WEIGHTS_DIR, "warmstart_cavity_R128.npy"))
    out = WS.warm_vs_cold_sweep(net, target=target, max_steps=max_steps, indices=idx, stream=stream, log=None)
    net.close()
    for k in ("cold_batch", "warm_batch"):
        out[k] = {a: b for a, b in out[k].items() if a not in ("final_residual", "seconds_to_target")}
    out["workload"] = ("stratified subset of the seeded 512-cavity sweep (seed 2306): the first %d per side "
                       "{65,129,257,513} of the steady subset recorded with the network (Re <= 1000, flow "
                       "reaching %.0e from rest)" % (per_side, target))
    return out


def oracle_full_configs(threads=0, log=print):
    """The FP64 oracle on every benchmark configuration at full size, one
    JSON line each (CPU only; hours of work on a few host cores, so never
    part of a default run): Taylor-Green 64^2 x 1000 steps; the Re = 1000
    cavity at 257^2 (uniform and tanh beta = 1.5) marched to residual 1e-8
    with the library's residual definition (window 100 steps); the power-law
    trapezoid cavities at 513^2 (n in {0.5, 1, 1.5} x Re in {100, 400,
    1000}, 200 steps each from rest); the 512-cavity sweep (10 steps of
    every cavity, one problem after another); Taylor-Green 4096^2 x 2000
    steps."""
    import numpy as np

    from oracle.oracle import Oracle, max_threads
    from paper_2306_08216_gb300 import workloads as W
    cores = threads or max_threads()

    def emit(name, nodes, steps, sec, **extra):
        d = {"workload": name, "nodes": nodes, "steps": steps, "seconds": sec,
             "mlups": nodes * steps / sec / 1e6, "cores": cores, "kind": "oracle"}
        d.update(extra)
        log(json.dumps(finite_json(d)))

    def timed(o, steps):
        t0 = time.perf_counter()
        o.step(steps)
        return time.perf_counter() - t0

    o = Oracle(64, 64, nu=NU, lx=2 * math.pi, ly=2 * math.pi, threads=threads)
    o.init(*W.taylor_green(64, U0))
    emit("taylor_green_64x64_fp64", 64 * 64, 1000, timed(o, 1000))
    X, Y = W.trapezoid_grid(513, 513)
    for n_index in (0.5, 1.0, 1.5):
        for re in (100.0, 400.0, 1000.0):
            K = CAV_U0 ** (2.0 - n_index) / re
            nu_ref = K * CAV_U0 ** (n_index - 1.0)
            o = Oracle(513, 513, nu=nu_ref, grid="curvilinear", x=X, y=Y, walls=(True, True),
                       u_wall=(0, 0, 0, CAV_U0), power_law=(K, n_index, nu_ref / 20, nu_ref * 20), threads=threads)
            o.init(*W.zeros(513, 513))
            emit("trapezoid_513x513_power_law_n%g_re%g_fp64" % (n_index, re), 513 * 513, 200, timed(o, 200))
            del o
    probs = batch_problems()
    sec, nodes = 0.0, 0
    for p in probs:
        kw = dict(p)
        nx, ny = kw.pop("nx"), kw.pop("ny")
        o = Oracle(nx, ny, threads=threads, **kw)
        o.init(*W.zeros(nx, ny))
        sec += timed(o, 10)
        nodes += nx * ny
        del o
    emit("batch_512_power_law_cavities_fp64", nodes, 10, sec, note="each cavity stepped on its own")
    o = Oracle(NX, NY, nu=NU, lx=2 * math.pi, ly=2 * math.pi, threads=threads)
    o.init(*W.taylor_green(NX, U0))
    emit("taylor_green_4096x4096_fp64", NX * NY, 2000, timed(o, 2000))
    del o
    for grid in ("uniform", "tanh_1.5"):
        kw = dict(nu=CAV_U0 / CAV_RE, walls=(True, True), u_wall=(0, 0, 0, CAV_U0), threads=threads)
        if grid.startswith("tanh"):
            xs = W.tanh_nodes(CAV_N, 1.5)
            kw.update(grid="separable", x=xs, y=xs)
        o = Oracle(CAV_N, CAV_N, **kw)
        o.init(*W.zeros(CAV_N, CAV_N))
        f = o.fields()
        prev = np.stack([f["u"], f["v"]])
        steps, sec, r = 0, 0.0, math.inf
        while r > 1e-8 and steps < 3_000_000:
            t0 = time.perf_counter()
            o.step(100)
            f = o.fields()
            cur = np.stack([f["u"], f["v"]])
            r = math.sqrt(((cur - prev) ** 2).sum()) / (100 * math.sqrt((cur ** 2).sum()))
            sec += time.perf_counter() - t0
            prev = cur
            steps += 100
        emit("cavity_257x257_re1000_%s_to_residual_1e-8_fp64" % grid, CAV_N * CAV_N, steps, sec, residual=r,
             reached=bool(r <= 1e-8))
        del o


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    if args.oracle_configs:
        oracle_full_configs(args.oracle_threads)
        return 0
    from oracle.oracle import Oracle, max_threads
    from paper_2306_08216_gb300 import workloads as W
    n = 512
    o = Oracle(n, n, nu=NU, lx=2 * math.pi, ly=2 * math.pi)
    o.init(*W.taylor_green(n, U0))
    o.step(args.warmup)
    t0 = time.perf_counter()
    o.step(args.steps)
    sec = time.perf_counter() - t0
    val = n * n * args.steps / sec / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": "MLUPS", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sec / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "taylor_green_512x512_fp64_oracle", "nx": n, "ny": n,
                   "sample_of": "taylor_green_4096x4096_fp32",
                   "sample": "512x512 Taylor-Green (same per-node work as the 4096^2 workload), one oracle step "
                             "per bench step", "nu": NU, "U0": U0, "cfl": 0.5, "eta": 0.8},
        "cpu_baseline": {"value": val, "unit": "MLUPS", "cores": max_threads(), "kind": "oracle",
                         "sample": "512x512 Taylor-Green, %d steps" % args.steps},
        "e2e": {"value": val, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--oracle-configs", action="store_true",
                    help="with --impl reference: time the FP64 oracle on every benchmark configuration at full "
                         "size (hours of CPU work; one JSON line per configuration)")
    ap.add_argument("--oracle-threads", type=int, default=0, help="oracle threads (0 = all)")
    ap.add_argument("--no-time-to-residual", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-storage", action="store_true", help="skip the 16-bit storage runs")
    ap.add_argument("--no-warm-start", action="store_true", help="skip the learned warm-start comparison")
    ap.add_argument("--no-body-fitted", action="store_true", help="skip the trapezoid power-law runs")
    ap.add_argument("--no-rho0", action="store_true", help="skip the run with the alpha = 0 distribution")
    ap.add_argument("--launch", default=None,
                    help="threads,rows_per_block: pin the launch plan instead of the autotuned one (profiling)")
    ap.add_argument("--batch-solo-sample", type=int, default=0,
                    help="time the one-launch-per-problem reference of the batch on this many cavities "
                         "(0: every cavity of the sweep)")
    ap.add_argument("--batch-count", type=int, default=BATCH_COUNT,
                    help="cavities of the batched sweep (default 512; fewer only for profiling)")
    ap.add_argument("--nx", type=int, default=NX,
                    help="grid side (default 4096, the benchmark workload; smaller sides only for profiling)")
    args = ap.parse_args()
    rank, world, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2306_08216_gb300 import build as B
    from paper_2306_08216_gb300 import mdf
    from paper_2306_08216_gb300 import workloads as W

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    B.build()
    stream = torch.cuda.Stream()

    def barrier():
        if world > 1:
            dist.barrier()

    nx = ny = args.nx
    u, v, p = W.taylor_green(nx, U0)
    solver = mdf.Solver(nx, ny, nu=NU, lx=2 * math.pi, ly=2 * math.pi, stream=stream)
    if args.launch:
        threads, rows = (int(x) for x in args.launch.split(","))
        solver.set_launch(threads, rows)
    solver.init(u, v, p)
    solver.step(args.warmup)
    solver.synchronize()
    info = solver.launch_info()
    bpn = solver.bytes_per_node()

    # ---- device-timed run: K fused steps, CUDA events on the solver stream
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clocks:
        start.record(stream)
        solver.step(args.steps)
        stop.record(stream)
        stop.synchronize()
        # a timed region shorter than the sampler's period holds no sample:
        # the same step keeps the GPU loaded for at least 1 s more (outside
        # the timed region, before the sampler stops) so the line carries
        # clocks taken under this load
        ms_timed = start.elapsed_time(stop)
        extra_steps = 0
        if ms_timed < CLOCK_WINDOW_MS:
            extra_steps = int(math.ceil((CLOCK_WINDOW_MS - ms_timed) / max(ms_timed / args.steps, 1e-3)))
            solver.step(extra_steps)
            solver.synchronize()
    torch.cuda.synchronize()
    ms = start.elapsed_time(stop)
    barrier()
    ms_max = max_over_ranks(ms, world, "cuda")
    nodes = nx * ny
    value = job_mlups(nodes, args.steps, world, ms_max / 1e3)
    ms_step = ms_max / args.steps
    peak, peak_kind = measured_peaks()
    achieved = bpn * nodes / (ms / args.steps / 1e3) / 1e9  # GB/s of this rank's launches
    r, drift = solver.residual()  # also checks for divergence

    # ---- end-to-end through the C ABI with host buffers
    pin = [torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).pin_memory() for a in (u, v, p)]
    outs = [torch.empty((ny, nx), dtype=torch.float32).pin_memory() for _ in range(3)]
    e2e_steps = args.steps
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    solver.init(pin[0].numpy(), pin[1].numpy(), pin[2].numpy())
    solver.step(e2e_steps)
    solver.fields(["u", "v", "P"], out=dict(zip(("u", "v", "P"), outs)))  # straight into the pinned buffers
    e2e_sec = time.perf_counter() - t0
    e2e_val = job_mlups(nodes, e2e_steps, world, max_over_ranks(e2e_sec, world, "cuda"))

    # ---- 16-bit deviation storage on the same workload
    storage = None if args.no_storage else storage_benchmark(mdf, W, torch, stream, solver, nx)

    # ---- the same workload with the alpha = 0 distribution evolved
    rho0 = None if args.no_rho0 else rho0_benchmark(mdf, W, torch, stream, nx)

    # ---- batched sweep: many cavities, one launch per step
    batch = None if args.no_batch else batch_benchmark(
        mdf, torch, stream, count=args.batch_count, solo_sample=args.batch_solo_sample or args.batch_count)

    # ---- power-law cavities on the body-fitted trapezoid grid
    body = None if args.no_body_fitted else body_fitted_benchmark(mdf, W, torch, stream)

    # ---- learned warm start + batching against cold starts
    warm = None if args.no_warm_start else warm_start_benchmark(stream)

    # ---- time to residual 1e-8 from rest: lid-driven cavity, Re = 1000, 257^2
    ttr = None
    if not args.no_time_to_residual:
        ttr = {}
        for grid in ("uniform", "tanh_1.5"):
            ttr[grid] = time_to_residual(mdf, W, grid, stream)
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        # about 10 s of CPU work (512^2 x 1400 = 367 M node updates)
        mlups, cores, sec = oracle_sample(1400, 512)
        cpu = {"value": mlups, "unit": "MLUPS", "cores": cores, "kind": "oracle",
               "sample": "512x512 Taylor-Green, 1400 steps (%.1f s)" % sec}
    line = {
        "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "taylor_green_%dx%d_fp32" % (nx, ny), "nx": nx, "ny": ny, "nu": NU, "U0": U0, "cfl": 0.5,
                   "eta": 0.8, "s_ratio": 1.5, "l2": "inputs larger than L2 (2 x 692 MB state), no flush",
                   "parallelism": "replicas x%d" % world, "launch": info},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": ncu_traffic_per_launch(), "bytes_per_node": bpn,
                     "peak_kind": peak_kind + " (MEASURED_PEAKS hbm_gbs)" if peak_kind == "measured" else peak_kind},
        "e2e": {"value": e2e_val, "unit": "MLUPS", "h2d_bytes_per_step": 3 * nodes * 4 / e2e_steps,
                "d2h_bytes_per_step": 3 * nodes * 4 / e2e_steps, "steps": e2e_steps, "seconds": e2e_sec,
                "note": "one upload of u, v, p (pinned host -> device, %d MB) and one download of u, v, P "
                        "(device -> pinned host, %d MB) per run of %d steps, through mdf_init_fields, mdf_step "
                        "and mdf_fields; with few steps the host copies dominate"
                        % (3 * nodes * 4 // 2 ** 20, 3 * nodes * 4 // 2 ** 20, e2e_steps)},
        "gpu_launches": args.steps,
        "clocks": dict(clocks.summary(), window="the %d timed steps and %d more steps of the same kernel right "
                                                 "after them (%.0f ms), sampled every %d ms"
                       % (args.steps, extra_steps, ms_timed * (1 + extra_steps / args.steps), clocks.period_ms)),
        "cpu_baseline": cpu,
        "check": {"residual": r, "drift_u": drift[0], "drift_v": drift[1]},
        "time_to_residual": ttr,
        "batch": batch,
        "storage": storage,
        "warm_start": warm,
        "body_fitted": body,
        "rho0": rho0,
    }
    if ttr and cpu:
        for k in ttr:
            ttr[k]["cpu_oracle_seconds_extrapolated"] = ttr[k]["steps"] * CAV_N * CAV_N / (cpu["value"] * 1e6)
    print(json.dumps(finite_json(line), allow_nan=False), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
