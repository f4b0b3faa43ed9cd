"""Benchmark of the fused double-MRT thermal LBM step on GB300.

Workload: a 128^3 cavity of Type 2 (hot / cold y walls, linear-profile x and z
walls), Ra = 1e5, Pr = 0.71, Ma = 0.1, starting from rest.  One benchmark
step = 100 fused LBM time steps + the convergence residual + the hot-wall
Nusselt numbers, i.e. one pass of the whole hot path.  Throughput is MLUPS
(million coupled D3Q19 + D3Q7 cell updates per second).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl dmrt|reference]
                    [--storage f32|bf16|f16] [--grid N --wall T --ra RA]

The defaults measure the 128^3 Type 2 cavity in FP32 storage; --grid 256
--wall 3 --ra 1e6 --storage bf16 (or f16) measures the 256^3 Type 3 cavity with
16-bit population storage.

With N > 1 (launched by torchrun) every rank runs an independent replica of
the same cavity ("replicas only": a single cavity is not sharded); the
reported value is the total cell updates of all ranks over the slowest
rank's time.  Rank 0 prints one JSON line.
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GRID = (128, 128, 128)
WALL = 2
RA, PR, MA = 1e5, 0.71, 0.1
LBM_STEPS_PER_STEP = 100
STORAGES = {"f32": 0, "bf16": 1, "f16": 2}
METRIC = "MLUPS and % HBM roofline per coupled step"
# GB300 HBM3e nominal bandwidth (GB/s); the roofline fraction is taken against
# the measured copy bandwidth, and against this figure beside it
NOMINAL_HBM_GBS = 7900.0
WALL_NAMES = {1: "Type 1 (adiabatic side walls)", 2: "Type 2 (linear side walls)",
              3: "Type 3 (linear x walls, adiabatic z walls)"}


STREAMINGS = {"ab": 0, "inplace": 1}


def workload(args) -> str:
    n = args.grid
    scheme = "" if args.streaming == "ab" else ", in-place streaming (one population buffer)"
    return (f"{n}^3 cavity, {WALL_NAMES[args.wall]}, Ra={args.ra:g}, Pr={PR}, Ma={MA}, from rest, "
            f"{args.storage} population storage{scheme}; one step = {args.inner} fused LBM steps + "
            f"residual + hot-wall Nu")


_BODY = ["paper_1511_04633_gb300/csrc/step_body.cuh", "paper_1511_04633_gb300/csrc/lattice.cuh",
         "paper_1511_04633_gb300/csrc/vec2.cuh", "paper_1511_04633_gb300/csrc/residual.cuh"]
# sources of each step kernel: one cell per thread (two buffers), two cells
# per thread (two buffers; direct or TMA-staged loads), in place
KERNEL_SOURCES = {"ab": ["paper_1511_04633_gb300/csrc/step.cu"] + _BODY,
                  "pair": ["paper_1511_04633_gb300/csrc/step_pair.cu",
                           "paper_1511_04633_gb300/csrc/pair_body.cuh"] + _BODY,
                  "pair_tma": ["paper_1511_04633_gb300/csrc/step_pair.cu",
                               "paper_1511_04633_gb300/csrc/pair_body.cuh",
                               "paper_1511_04633_gb300/csrc/umma.cuh"] + _BODY,
                  "inplace": ["paper_1511_04633_gb300/csrc/step_inplace.cu"] + _BODY,
                  "inplace_pair": ["paper_1511_04633_gb300/csrc/step_pair.cu",
                                   "paper_1511_04633_gb300/csrc/pair_body.cuh"] + _BODY}
STEP_KERNEL_SOURCES = KERNEL_SOURCES["ab"]


# ---------------------------------------------------------------- distributed plumbing

def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, local, world


def init_dist(world: int, backend: str):
    if world <= 1:
        return None
    import torch.distributed as dist
    os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
    dist.init_process_group(backend=backend)
    return dist


def barrier(dist):
    if dist is not None:
        dist.barrier()


def reduce_max(dist, value: float, device=None) -> float:
    """Maximum of `value` over all ranks (the slowest rank's time)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate(units_per_rank: float, world: int, seconds_max: float) -> float:
    """Whole-job throughput in MLUPS: all ranks' cell updates / slowest time."""
    return units_per_rank * world / seconds_max / 1e6


# ---------------------------------------------------------------- clocks and peaks

class ClockSampler:
    """nvidia-smi clock / throttle-reason samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None or not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        max_mhz = max(r[1] for r in rows)
        loaded = [r for r in rows if r[0] > 0.5 * max_mhz] or rows
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in loaded for k, v in enumerate(r[2]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in loaded), "sm_max_mhz": max_mhz,
                "reasons": reasons, "samples": len(loaded)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def step_kernel_digest(scheme: str = "ab") -> str:
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES[scheme]:
        with open(os.path.join(ROOT, rel), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(storage: str = "f32", wall: int = 2, scheme: str = "ab"):
    """DRAM bytes per step-kernel launch from the committed ncu summary, only
    if it was taken on the current kernel sources for this storage, wall and
    kernel scheme ("ab", "pair", "pair_tma", "inplace" or "inplace_pair")."""
    path = os.path.join(ROOT, "profiles", "step_kernel_traffic.json")
    try:
        with open(path) as fh:
            t = json.load(fh)
    except (OSError, ValueError):
        return None
    recs = t if isinstance(t, list) else [t]
    for rec in recs:
        if (rec.get("source_digest") == step_kernel_digest(scheme)
                and rec.get("storage", "f32") == storage and rec.get("wall", 2) == wall
                and rec.get("scheme", "ab") == scheme):
            return rec.get("dram_bytes_per_launch")
    return None


# ---------------------------------------------------------------- CPU oracle legs

def oracle_sample(grid, wall, ra, seconds: float = 12.0, max_steps: int = 400):
    """Time the FP64 oracle on the benchmark cavity: steps from rest until
    `seconds` of CPU work (at least 2).  Returns (MLUPS, cores, steps)."""
    import oracle
    o = oracle.Oracle.physical(grid, wall, ra, PR, MA)
    o.step(1)  # first touch of the buffers
    cells = grid[0] * grid[1] * grid[2]
    n = 0
    t0 = time.perf_counter()
    while n < 2 or (time.perf_counter() - t0 < seconds and n < max_steps):
        o.step(1)
        n += 1
    dt = time.perf_counter() - t0
    o.close()
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return cells * n / dt / 1e6, cores, n


def run_reference(args, rank, world):
    """The oracle as the reference arm: each benchmark step is a bounded
    sample of the same workload (a few oracle LBM steps) on the host cores."""
    if rank != 0:
        return
    import oracle
    grid = (args.grid,) * 3
    o = oracle.Oracle.physical(grid, args.wall, args.ra, PR, MA)
    cells = grid[0] * grid[1] * grid[2]
    per_step = args.ref_lbm_steps
    for _ in range(args.warmup):
        o.step(per_step)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o.step(per_step)
    dt = time.perf_counter() - t0
    o.close()
    value = cells * per_step * args.steps / dt / 1e6
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    sample = f"{per_step} FP64 oracle LBM step(s) of the {args.grid}^3 Type {args.wall} cavity per benchmark step"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "MLUPS",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload(args), "grid": list(grid), "wall_type": args.wall,
                   "Ra": args.ra, "parallelism": "replicas"},
        "cpu_baseline": {"value": value, "unit": "MLUPS", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- GPU arm

def run_dmrt(args, rank, local, world):
    import torch
    from paper_1511_04633_gb300 import dmrt

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    dist = init_dist(world, "nccl")
    device = torch.device("cuda", local)
    # a dedicated stream: the library launches on it and the events below are
    # recorded on it (torch's default stream is the legacy NULL stream)
    stream = torch.cuda.Stream(device)
    torch.cuda.set_stream(stream)
    dmrt.load()

    grid = (args.grid,) * 3
    cells = grid[0] * grid[1] * grid[2]
    storage = STORAGES[args.storage]
    cav = dmrt.Cavity(grid, args.ra, PR, MA, args.wall, storage=storage,
                      streaming=STREAMINGS[args.streaming], cells_per_thread=args.cells_per_thread,
                      pair_loads=args.pair_loads)
    dmrt.dmrt_set_stream(cav.h, stream)
    inner = args.inner
    cpt = cav.params["cells_per_thread"]
    if args.streaming == "inplace":
        scheme = {1: "inplace", 2: "inplace_pair"}[cpt]
    else:
        scheme = {1: "ab", 2: ("pair_tma" if cav.params["pair_loads"] == 2 else "pair")}[cpt]

    def one_step():
        dmrt.dmrt_step(cav.h, inner)
        return dmrt.dmrt_nusselt(cav.h, 0)

    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()

    # timed region: device-resident state, CUDA events on the launch stream
    dmrt.dmrt_get_stats(cav.h, reset=True)
    dmrt.dmrt_set_timing(cav.h, True)
    barrier(dist)
    torch.cuda.synchronize()
    with ClockSampler(local) as clocks:
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(args.steps):
            one_step()
        ev1.record(stream)
        torch.cuda.synchronize()
    barrier(dist)
    ms = ev0.elapsed_time(ev1)
    stats = dmrt.dmrt_get_stats(cav.h, reset=True)
    dmrt.dmrt_set_timing(cav.h, False)
    secs = reduce_max(dist, ms / 1e3, device)
    units = cells * inner * args.steps
    value = aggregate(units, world, secs)

    # roofline of the dominant kernel (the fused step), from its own events
    launch_s = stats["step_ms"] / 1e3 / max(stats["timed_steps"], 1)
    bytes_per_cell = stats["bytes_per_cell"]
    achieved = bytes_per_cell * cells / launch_s / 1e9
    peak, peak_src = measured_peaks()
    traffic = profiled_traffic(args.storage, args.wall, scheme)

    # end to end through the C ABI with host buffers: upload the start fields
    # from pinned memory, step, read the fields and Nu back
    rho_h = torch.ones(grid[::-1], dtype=torch.float32).pin_memory()
    u_h = torch.zeros((3,) + grid[::-1], dtype=torch.float32).pin_memory()
    th_h = torch.zeros(grid[::-1], dtype=torch.float32).pin_memory()
    rho_o = torch.empty_like(rho_h).pin_memory()
    u_o = torch.empty_like(u_h).pin_memory()
    th_o = torch.empty_like(th_h).pin_memory()
    dmrt.dmrt_fields(cav.h, rho_h, u_h, th_h)  # the current state as the start fields

    def e2e_step():
        dmrt.dmrt_init_fields(cav.h, rho_h, u_h, th_h)
        dmrt.dmrt_step(cav.h, inner)
        dmrt.dmrt_fields(cav.h, rho_o, u_o, th_o)
        return dmrt.dmrt_nusselt(cav.h, 0)

    for _ in range(2):
        e2e_step()
    e2e_steps = max(3, args.steps // 4)
    barrier(dist)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        e2e_step()
    torch.cuda.synchronize()
    e2e_secs = reduce_max(dist, time.perf_counter() - t0, device)
    e2e_value = aggregate(cells * inner * e2e_steps, world, e2e_secs)
    h2d = 5 * 4 * cells
    d2h = 5 * 4 * cells + 3 * 8

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    nbuf = 2 if args.streaming == "ab" else 1
    steady = None if args.no_steady else run_to_steady(dmrt, torch, stream, grid, storage, args, launch_s)
    warm = None if args.warm_start_cases <= 0 else run_warm_start(args.warm_start_cases)
    configs = None if args.no_configs else run_configs(dmrt, torch, stream, local)
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        mlups, cores, n = oracle_sample(grid, args.wall, args.ra, args.cpu_seconds)
        cpu = {"value": mlups, "unit": "MLUPS", "cores": cores, "kind": "oracle",
               "sample": f"{n} FP64 oracle LBM steps of the {args.grid}^3 Type {args.wall} "
                         f"cavity from rest"}

    line = {
        "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": secs / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": workload(args), "grid": list(grid), "wall_type": args.wall,
                   "Ra": args.ra, "Pr": PR, "Ma": MA, "lbm_steps_per_step": inner,
                   "storage": f"{args.storage} deviations from rest equilibrium"
                              + ("" if storage == 0 else ", stochastic rounding"),
                   "streaming": "two population buffers (A-B)" if args.streaming == "ab"
                                else "in place: one population buffer, two alternating kernels",
                   "l2": f"inputs larger than L2 ({nbuf} x {bytes_per_cell / 2 * cells / 1e6:.0f} MB "
                         f"population buffer)" if bytes_per_cell / 2 * cells > 129e6
                         else "inputs fit in L2: not a DRAM measurement",
                   "cells_per_thread": cpt, "pair_loads": cav.params["pair_loads"],
                   "parallelism": f"replicas x{world}"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "peak_source": peak_src,
                     "nominal_peak": NOMINAL_HBM_GBS, "frac_nominal": achieved / NOMINAL_HBM_GBS,
                     "kernel": {"ab": f"step_kernel<{args.wall}, {args.storage}>",
                                "pair": f"step_pair_kernel<{args.wall}, {args.storage}>",
                                "pair_tma": f"step_pair_tma_kernel<{args.wall}, {args.storage}>",
                                "inplace": f"step_inplace_kernel<{args.wall}, {args.storage}> "
                                           "(both phases)",
                                "inplace_pair": f"step_inplace_pair_kernel<{args.wall}, {args.storage}> "
                                                "(both phases)"}[scheme],
                     "bytes_per_cell": bytes_per_cell, "launch_us": launch_s * 1e6},
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": "MLUPS", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": stats["total_launches"],
        "clocks": clocks.summary(),
        "steady": steady,
        "warm_start": warm,
        "configs": configs,
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


# Convergence residual per storage format: 1e-7 for FP32; 16-bit storage with
# stochastic rounding has a noise floor near 3e-5 (BF16) and 3e-6 (FP16), so
# its state counts as steady at 1e-4 and 1e-5.
STEADY_TOL = {0: 1e-7, 1: 1e-4, 2: 1e-5}


def run_to_steady(dmrt, torch, stream, grid, storage, args, launch_s, seconds=40.0):
    """Outside the timed region: a fresh cavity of the workload run from rest
    to the convergence residual of its storage format (within a step budget of
    about `seconds` of kernel time), then a 1000-step window timed on the
    converged state."""
    tol = STEADY_TOL[storage]
    cav = dmrt.Cavity(grid, args.ra, PR, MA, args.wall, storage=storage, streaming=STREAMINGS[args.streaming],
                      cells_per_thread=args.cells_per_thread, pair_loads=args.pair_loads)
    dmrt.dmrt_set_stream(cav.h, stream)
    budget = max(10_000, int(seconds / max(launch_s, 1e-7)) // 100 * 100)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ok, steps, r = cav.run_to_steady(tol, budget)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    nu = cav.nusselt(0)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    cav.step(1000)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    cells = grid[0] * grid[1] * grid[2]
    cav.close()
    return {"tol": tol, "converged": bool(ok), "steps": steps, "residual": r, "seconds": wall,
            "nu_hot_wall": list(nu), "window_steps": 1000,
            "window_mlups": cells * 1000 / (ms / 1e3) / 1e6}


WARM_GRID = 128  # the warm-started cavities of the learned warm start (64^3 network, resampled)


def run_warm_start(count):
    """Outside the timed region: the learned warm start on `count` cavities
    of the network's seeded draws that it was not trained on, at 128^3.  The
    network is read from the parameters file that
    ``python -m paper_1511_04633_gb300.surrogate --save-params`` wrote (no
    training here).  Each cavity is solved from rest to the convergence
    residual and on to 1e-9 for the reference Nu, and from the network's
    prediction to the convergence residual; steps and wall-clock seconds
    until the hot-wall Nu_3D stays within 1e-3 of the reference, and until
    the residual falls below 1e-7, are reported for both."""
    from paper_1511_04633_gb300 import surrogate as S

    sur, info = S.load_surrogate()
    cases = []
    t0 = time.perf_counter()
    for d in S.held_out_draws(count):
        r = S.compare_warm_start(sur, WARM_GRID, d["Ra"], d["wall"], tol=1e-7, nu_rtol=1e-3)
        cold, warm = r["from_rest"], r["warm"]

        def ratio(a, b):
            return None if a is None or b is None or b <= 0 else a / b

        cases.append({"Ra": d["Ra"], "wall": d["wall"], "nu_reference": r["nu_reference"],
                      "nu_warm_rel_err": r["nu_rel_diff"],
                      "from_rest": {k: cold[k] for k in ("steps_to_nu", "seconds_to_nu",
                                                         "steps_to_residual", "seconds_to_residual")},
                      "warm": {k: warm[k] for k in ("steps_to_nu", "seconds_to_nu", "steps_to_residual",
                                                    "seconds_to_residual", "predict_seconds")},
                      "gain_steps_to_nu": ratio(cold["steps_to_nu"], warm["steps_to_nu"]),
                      "gain_seconds_to_nu": ratio(cold["seconds_to_nu"], warm["seconds_to_nu"]),
                      "gain_seconds_to_residual": ratio(cold["seconds_to_residual"], warm["seconds_to_residual"])})
    sur.close()
    gains = [c["gain_seconds_to_nu"] for c in cases if c["gain_seconds_to_nu"] is not None]
    return {"grid": WARM_GRID, "network": {"grid": info.get("grid"), "channels": info.get("channels"),
                                           "trained_on": info.get("train"), "seed": info.get("seed")},
            "nu_rtol": 1e-3, "residual_tol": 1e-7, "nu_reference": "from-rest solve continued to r < 1e-9",
            "cases": cases, "min_gain_seconds_to_nu": min(gains) if gains else None,
            "max_nu_warm_rel_err": max(c["nu_warm_rel_err"] for c in cases),
            "seconds": time.perf_counter() - t0}


def measure_ensemble(dmrt, inputs, torch, stream, gpu, *, members, seed, storage, streaming, inner, steps,
                     warmup, dist=None, device=None, world=1):
    """The batched ensemble of seeded cavities (a few launches per time step
    over all of them, autotuned) timed with CUDA events on `stream`, and the same
    cavities as separate handles stepped one after another.  Returns the
    measurement as a dict (MLUPS over all ranks)."""
    draws = inputs.ensemble_draws(members, seed=seed)
    cav = [{"grid": (d["n"],) * 3, "Ra": d["Ra"], "wall": d["wall"]} for d in draws]
    ens = dmrt.Ensemble(cav, storage=storage, streaming=streaming)
    ens_kernel = ("ensemble_pair_kernel" if ens.params(0)["cells_per_thread"] == 2
                  else "ensemble_step_kernel") + (" (in place, both phases)" if streaming else "")
    dmrt.dmrt_ensemble_set_stream(ens.e, stream)
    report = ens.autotune(trials=3)
    cells = ens.cells

    def one_step():
        ens.step(inner)
        return ens.nusselt(0)

    for _ in range(warmup):
        one_step()
    dmrt.dmrt_ensemble_get_stats(ens.e, reset=True)
    dmrt.dmrt_ensemble_set_timing(ens.e, True)
    barrier(dist)
    torch.cuda.synchronize()
    with ClockSampler(gpu) as clocks:
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(steps):
            one_step()
        ev1.record(stream)
        torch.cuda.synchronize()
    barrier(dist)
    secs = reduce_max(dist, ev0.elapsed_time(ev1) / 1e3, device)
    stats = dmrt.dmrt_ensemble_get_stats(ens.e, reset=True)
    value = aggregate(cells * inner * steps, world, secs)
    launch_s = stats["step_ms"] / 1e3 / max(stats["timed_steps"], 1)
    achieved = stats["bytes_per_cell"] * cells / launch_s / 1e9
    peak, peak_src = measured_peaks()
    taus = [ens.params(k)["tau_nu"] for k in range(len(cav))]
    ens.close()

    # the same cavities as separate handles, stepped one after another
    singles = [dmrt.Cavity(c["grid"], c["Ra"], wall_type=c["wall"], storage=storage, streaming=streaming)
               for c in cav]
    for h in singles:
        dmrt.dmrt_set_stream(h.h, stream)
        h.step(inner)
        h.nusselt(0)
    sep_steps = max(2, steps // 4)
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(sep_steps):
        for h in singles:
            h.step(inner)
            h.nusselt(0)
    ev1.record(stream)
    torch.cuda.synchronize()
    sep_secs = reduce_max(dist, ev0.elapsed_time(ev1) / 1e3, device)
    separate = aggregate(cells * inner * sep_steps, world, sep_secs)
    for h in singles:
        h.close()
    names = {v: k for k, v in STORAGES.items()}
    return {
        "value": value, "unit": "MLUPS", "steps": steps, "warmup": warmup, "ms_per_step": secs / steps * 1e3,
        "workload": f"ensemble of {len(cav)} seeded cavities (edge in 32/48/64/96, log10 Ra in [3, 6], "
                    f"types 1-3, seed {seed}), {names[storage]} storage"
                    + ("" if streaming == 0 else ", in-place streaming")
                    + f"; one step = {inner} LBM steps of all members + residuals + hot-wall Nu of all",
        "cells": cells, "min_tau_nu": min(taus), "autotune": report,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": None, "peak_source": peak_src,
                     "nominal_peak": NOMINAL_HBM_GBS, "frac_nominal": achieved / NOMINAL_HBM_GBS,
                     "kernel": ens_kernel, "bytes_per_cell": stats["bytes_per_cell"],
                     "launch_us": launch_s * 1e6},
        "separate_runs": {"value": separate, "unit": "MLUPS",
                          "what": f"the same {len(cav)} cavities as separate handles, stepped one after another"},
        "gpu_launches": stats["total_launches"], "clocks": clocks.summary(),
    }


def measure_cavity(dmrt, torch, stream, gpu, *, grid, wall, ra, storage, inner, steps, warmup):
    """One cavity from rest: `steps` benchmark steps of `inner` LBM steps,
    a residual and a hot-wall Nu each, timed with CUDA events on `stream`;
    the step kernels' own events give the roofline."""
    cav = dmrt.Cavity(grid, ra, PR, MA, wall, storage=storage)
    dmrt.dmrt_set_stream(cav.h, stream)
    for _ in range(warmup):
        cav.step(inner)
        cav.nusselt(0)
    dmrt.dmrt_get_stats(cav.h, reset=True)
    dmrt.dmrt_set_timing(cav.h, True)
    torch.cuda.synchronize()
    with ClockSampler(gpu) as clocks:
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(steps):
            dmrt.dmrt_step(cav.h, inner)
            dmrt.dmrt_nusselt(cav.h, 0)
        ev1.record(stream)
        torch.cuda.synchronize()
    secs = ev0.elapsed_time(ev1) / 1e3
    stats = dmrt.dmrt_get_stats(cav.h, reset=True)
    cells = grid[0] * grid[1] * grid[2]
    launch_s = stats["step_ms"] / 1e3 / max(stats["timed_steps"], 1)
    achieved = stats["bytes_per_cell"] * cells / launch_s / 1e9
    peak, peak_src = measured_peaks()
    params = cav.params
    cav.close()
    names = {v: k for k, v in STORAGES.items()}
    kernel = "step_pair_kernel" if params["cells_per_thread"] == 2 else "step_kernel"
    traffic = profiled_traffic(names[storage], wall, "pair" if params["cells_per_thread"] == 2 else "ab")
    return {
        "value": cells * inner * steps / secs / 1e6, "unit": "MLUPS", "steps": steps, "warmup": warmup,
        "ms_per_step": secs / steps * 1e3,
        "workload": f"{grid[0]}^3 cavity, {WALL_NAMES[wall]}, Ra={ra:g}, Pr={PR}, Ma={MA}, from rest, "
                    f"{names[storage]} population storage" + ("" if storage == 0 else ", stochastic rounding")
                    + f"; one step = {inner} fused LBM steps + residual + hot-wall Nu",
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "peak_source": peak_src,
                     "nominal_peak": NOMINAL_HBM_GBS, "frac_nominal": achieved / NOMINAL_HBM_GBS,
                     "kernel": f"{kernel}<{wall}, {names[storage]}>", "bytes_per_cell": stats["bytes_per_cell"],
                     "launch_us": launch_s * 1e6},
        "gpu_launches": stats["total_launches"], "clocks": clocks.summary(),
    }


def run_configs(dmrt, torch, stream, gpu, steps=5, warmup=3):
    """Outside the timed region: short CUDA-event-timed measurements of the
    reduced-storage 256^3 cavity (Type 3, Ra = 1e6, BF16 and FP16) and of the
    64-member seeded ensemble (FP32 and BF16 with two buffers, BF16 in place,
    against the same cavities as separate handles), each with its own clock
    samples."""
    from paper_1511_04633_gb300 import inputs

    out = {}
    for name in ("bf16", "f16"):
        out[f"256cube_type3_ra1e6_{name}"] = measure_cavity(
            dmrt, torch, stream, gpu, grid=(256,) * 3, wall=3, ra=1e6, storage=STORAGES[name],
            inner=LBM_STEPS_PER_STEP, steps=steps, warmup=warmup)
    for name, streaming in (("f32", "ab"), ("bf16", "ab"), ("bf16", "inplace")):
        key = f"ensemble64_{name}" + ("_inplace" if streaming == "inplace" else "")
        out[key] = measure_ensemble(
            dmrt, inputs, torch, stream, gpu, members=64, seed=1234, storage=STORAGES[name],
            streaming=STREAMINGS[streaming], inner=LBM_STEPS_PER_STEP, steps=steps, warmup=warmup)
    return out


def run_ensemble(args, rank, local, world):
    """The batched ensemble of seeded cavities as the benchmark line."""
    import torch
    from paper_1511_04633_gb300 import dmrt, inputs

    torch.cuda.set_device(local)
    dist = init_dist(world, "nccl")
    device = torch.device("cuda", local)
    stream = torch.cuda.Stream(device)
    torch.cuda.set_stream(stream)
    m = measure_ensemble(dmrt, inputs, torch, stream, local, members=args.members, seed=args.seed,
                         storage=STORAGES[args.storage], streaming=STREAMINGS[args.streaming],
                         inner=args.inner, steps=args.steps, warmup=args.warmup, dist=dist, device=device,
                         world=world)
    if rank == 0:
        line = {
            "metric": METRIC, "value": m["value"], "unit": "MLUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": m["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": m["workload"], "cells": m["cells"], "min_tau_nu": m["min_tau_nu"],
                       "autotune": m["autotune"], "parallelism": f"replicas x{world}"},
            "roofline": m["roofline"], "separate_runs": m["separate_runs"],
            "gpu_launches": m["gpu_launches"], "clocks": m["clocks"],
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["dmrt", "reference"], default="dmrt")
    ap.add_argument("--inner", type=int, default=LBM_STEPS_PER_STEP,
                    help="LBM time steps per benchmark step")
    ap.add_argument("--ref-lbm-steps", type=int, default=1,
                    help="oracle LBM steps per reference benchmark step")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--storage", choices=sorted(STORAGES), default="f32")
    ap.add_argument("--streaming", choices=sorted(STREAMINGS), default="ab",
                    help="two population buffers, or one updated in place")
    ap.add_argument("--grid", type=int, default=GRID[0], help="cubic cavity edge")
    ap.add_argument("--cells-per-thread", type=int, choices=[0, 1, 2], default=0,
                    help="step kernel: 0 = the library's choice, 1 or 2 cells per thread")
    ap.add_argument("--pair-loads", type=int, choices=[0, 1, 2], default=0,
                    help="two-cell two-buffer kernel: 0 = the library's choice, 1 = direct loads, "
                         "2 = TMA-staged")
    ap.add_argument("--wall", type=int, choices=[1, 2, 3], default=WALL)
    ap.add_argument("--ra", type=float, default=RA)
    ap.add_argument("--ensemble", action="store_true",
                    help="measure the batched ensemble of seeded cavities instead")
    ap.add_argument("--members", type=int, default=64)
    ap.add_argument("--seed", type=int, default=1234)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-steady", action="store_true",
                    help="skip the run to steady state after the timed region")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the 256^3 16-bit and 64-member ensemble measurements after the timed region")
    ap.add_argument("--warm-start-cases", type=int, default=3,
                    help="held-out 128^3 cavities of the learned warm start measured after the timed "
                         "region (0: none)")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    rank, local, world = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.ensemble:
        run_ensemble(args, rank, local, world)
        return
    run_dmrt(args, rank, local, world)


if __name__ == "__main__":
    main()
