#!/usr/bin/env python3
"""Throughput of the porous-media D3Q27 collide-stream step on B300.

Workload (default): the periodic 256^3 porous box -- Gaussian-random-field
porosity (correlation length 16, seed 2) mapped to [0.35, 1], Carman-Kozeny
permeability with d = 2, Ergun Forchheimer coefficient, nu = 0.02, body force
b = 6e-4 along x (Re = <|v|> 16 / nu ~ 5-8 on a 64^3 oracle pilot) -- with FP32 population storage and FP32 arithmetic.
A step is one time step over every node: by default the three split kernels
(moments, velocity, collide-and-push into a second population array), or with
--kernel fused one z-marching kernel.  The same kernels streaming in place
(one population array) are timed too.  Populations (1.8 GB) exceed the 126 MB
L2, so no flush is needed between steps.

Prints ONE JSON line (rank 0).  Under torchrun every rank advances its own
replica of the box (weak scaling, no collective on the data path).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "porous D3Q27 GLUPS & % HBM roofline per storage dtype; serving p50/p99 ms"
UNIT = "GLUPS"
WORKLOADS = {
    "porous_box_256": dict(shape=(256, 256, 256), ell=16.0, seed=2, nu=0.02, b=(6e-4, 0.0, 0.0)),
    "porous_box_128": dict(shape=(128, 128, 128), ell=16.0, seed=2, nu=0.02, b=(6e-4, 0.0, 0.0)),
    "porous_box_640": dict(shape=(640, 640, 640), ell=16.0, seed=5, nu=0.02, b=(6e-4, 0.0, 0.0)),
    # the 640^3 box cut by a free slot 64 nodes wide in y: the slot carries a
    # Brinkman channel flow whose centre speed b 64^2 / (8 nu) ~ 0.05 sets b
    "slot_box_640": dict(shape=(640, 640, 640), ell=16.0, seed=5, nu=0.02, b=(2e-6, 0.0, 0.0), slot=64),
}
STORAGE_BYTES = {"fp64": 8, "fp32": 4, "fp16": 2, "bf16": 2}


def algorithmic_bytes(storage, Q=27):
    """Populations read once and written once, porosity and permeability read
    once: the least traffic of one node update (the whole step)."""
    sb = STORAGE_BYTES[storage]
    tb = 8 if storage == "fp64" else 4
    return 2 * Q * sb + 2 * tb


def kernel_bytes(kernel, storage, Q=27):
    """Per-kernel bytes per node that each kernel of a step must move by its
    design (its inputs read once, its outputs written once).  Split step:
    K1 populations + eps + kappa -> rho, m; K2 rho, m + eps + kappa -> v, a;
    K3 populations + rho, v, a + eps -> populations."""
    sb = STORAGE_BYTES[storage]
    if kernel == "fused":
        return {"k_fused_d3q27": 2 * Q * sb + 8}
    return {"k_split_moments": Q * sb + 8 + 16, "k_split_velocity": 16 + 8 + 24,
            "k_split_collide": 2 * Q * sb + 28 + 4}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.samples = []
        self._stop = threading.Event()
        self._t = None

    def _run(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                      "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=5)
                if out.returncode == 0 and out.stdout.strip():
                    self.samples.append([s.strip() for s in out.stdout.strip().split(",")])
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *exc):
        self._stop.set()
        if self._t:
            self._t.join(timeout=10)

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for s in self.samples:
            try:
                sm.append(float(s[0]))
                mx = float(s[1])
            except ValueError:
                continue
            for k, name in enumerate(names):
                if len(s) > 3 + k and s[3 + k].lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if os.environ.get("BENCH_BACKEND", "nccl") == "nccl" else "gloo")
        pg = dist
    return world, rank, local, pg


def max_over_ranks(x, pg, device=None):
    """Largest value of x over all ranks (the slowest rank sets the job time)."""
    if pg is None:
        return float(x)
    import torch

    on_gpu = pg.get_backend() == "nccl"
    t = torch.tensor([float(x)], dtype=torch.float64, device=f"cuda:{device}" if on_gpu else "cpu")
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def aggregate_glups(n_nodes, steps, ms_max, world):
    """Whole-job throughput: every rank advanced its own n_nodes box `steps` times
    within the slowest rank's ms_max."""
    return world * n_nodes * steps / (ms_max * 1e-3) / 1e9


def make_inputs(name):
    from paper_2606_29619_b300 import workloads

    w = WORKLOADS[name]
    if "slot" in w:
        eps, kap = workloads.slot_box(w["shape"][0], ell=w["ell"], seed=w["seed"], slot=w["slot"])
    else:
        eps, kap = workloads.porous_box(w["shape"], ell=w["ell"], seed=w["seed"])
    return eps, kap, w


def traffic_from_profile(kernel_tag, source="lbm_split.cuh"):
    """DRAM bytes per launch from the committed ncu summary, if the summary was
    taken on the current kernel source (its hash must match)."""
    import hashlib

    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        src = os.path.join(ROOT, "paper_2606_29619_b300", "csrc", source)
        h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        e = d.get(kernel_tag)
        if e and e.get("source_sha") == h:
            return float(e["dram_bytes_per_launch"])
    except Exception:
        pass
    return None


def time_storage(lbm, eps, kap, w, storage, steps, warmup, device, barrier, kernel="split", keep_v=False,
                 streaming="auto", tune_cache=None, autotune=True):
    """Device-timed GLUPS of one storage form; returns dict with ms per step
    and the mean device time of each kernel of a step (CUDA events around
    every launch of the timed region, on the stream the kernels run on)."""
    import torch

    stream = torch.cuda.Stream(device=device)
    # the split kernels' tile height: timed by the autotuner at creation (before the timed region)
    sim = lbm.Simulation(lbm.D3Q27, eps, kap, viscosity=w["nu"], force=w["b"], forchheimer=lbm.F_ERGUN,
                         storage=storage, kernel=kernel, stream=stream, device=device, streaming=streaming,
                         autotune=kernel == "split" and autotune, tune_cache=tune_cache)
    N = sim.N
    tuning = sim.tuning()
    sim.step(warmup)
    sim.sync()
    barrier()
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(device)
    start.record(stream)
    kernel_ms = sim.time_kernels(steps)
    end.record(stream)
    end.synchronize()
    torch.cuda.synchronize(device)
    ms = start.elapsed_time(end)
    sim.sync()
    info = sim.info()
    stats = sim.reduce()
    v = sim.moments()[1] if keep_v else None
    sim.close()
    del sim
    torch.cuda.empty_cache()
    names = list(kernel_bytes(info["kernel"], storage))
    return {"ms": ms, "ms_per_step": ms / steps, "N": N, "launches_per_step": info["launches_per_step"],
            "mean_vx": stats["mean_v"][0], "kernel": info["kernel"], "in_place": info["in_place"], "v": v,
            "kernel_ms": dict(zip(names, kernel_ms)), "tuning": tuning}


def cpu_baseline(seconds=15.0, name="porous_box_256"):
    """The oracle as it stands, on a bounded sample of the workload: the 48^3
    copy of the same porous box (same correlation length and seed), stepped
    until about `seconds` of CPU time."""
    import oracle
    from paper_2606_29619_b300 import workloads

    w = WORKLOADS[name]
    shape = (48, 48, 48)
    eps, kap = workloads.porous_box(shape, ell=w["ell"], seed=w["seed"])
    o = oracle.Oracle(oracle.D3Q27, eps, kap, nu_f=w["nu"], b=w["b"], forch=-1.0).init()
    N = eps.size
    t0 = time.perf_counter()
    steps = 0
    while time.perf_counter() - t0 < seconds:
        o.step(1)
        steps += 1
    dt = time.perf_counter() - t0
    cores = oracle.threads()
    # the same sample on one core, for a third of the time
    oracle.set_threads(1)
    t1 = time.perf_counter()
    steps1 = 0
    while time.perf_counter() - t1 < seconds / 3:
        o.step(1)
        steps1 += 1
    dt1 = time.perf_counter() - t1
    oracle.set_threads(cores)
    return {"value": N * steps / dt / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"D3Q27 48^3 copy of {name} (same GRF recipe), {steps} FP64 oracle steps in {dt:.1f} s",
            "one_core": {"value": N * steps1 / dt1 / 1e9, "unit": UNIT, "cores": 1,
                         "sample": f"{steps1} steps of the same copy in {dt1:.1f} s"}}


def e2e_run(lbm, eps, kap, w, steps, device, kernel="split", tune_cache=None, autotune=True):
    """Whole job through the public API with host buffers: lbm_create copies the
    host porosity / permeability to the device (and initialises the
    populations), `steps` steps run, and the result (rho and v in FP64) comes
    back to host memory.  The three parts are timed separately too."""
    import torch

    torch.cuda.synchronize(device)
    t0 = time.perf_counter()
    sim = lbm.Simulation(lbm.D3Q27, eps, kap, viscosity=w["nu"], force=w["b"], forchheimer=lbm.F_ERGUN,
                         storage="fp32", kernel=kernel, device=device, autotune=kernel == "split" and autotune,
                         tune_cache=tune_cache)
    t1 = time.perf_counter()
    sim.step(steps)
    sim.sync()
    t2 = time.perf_counter()
    rho, v = sim.moments()
    t3 = time.perf_counter()
    N = sim.N
    sim.close()
    return {"value": N * steps / (t3 - t0) / 1e9, "unit": UNIT, "steps": steps,
            "h2d_bytes_per_step": int(round(2 * 8 * N / steps)), "d2h_bytes_per_step": int(round(4 * 8 * N / steps)),
            "create_s": t1 - t0, "steps_s": t2 - t1, "readback_s": t3 - t2,
            "note": "one job at the workload's step count: host inputs to device, steps, rho and v back to host"}


def _serve(lbm, requests, cap_bytes, arrivals, storage="fp16", check_every=100, tol=1e-7, max_steps=200000):
    """Runs the request stream through one server: request k (3 cases, force
    1e-6 along x, y, z) is submitted at arrivals[k] seconds; returns per-request
    latency (last case finished - arrival), node updates and wall time."""
    srv = lbm.Server(storage=storage, hbm_cap_bytes=cap_bytes, check_every=check_every)
    owner, pending, finished = {}, list(range(len(requests))), {}
    left = {k: 3 for k in range(len(requests))}
    t0 = time.perf_counter()
    statuses = {}
    while len(finished) < len(requests):
        now = time.perf_counter() - t0
        while pending and arrivals[pending[0]] <= now:
            k = pending.pop(0)
            req = requests[k]
            for ax in range(3):
                b = [0.0, 0.0, 0.0]
                b[ax] = 1e-6
                cid = srv.submit(req["eps"], req["kappa"], viscosity=0.02, force=b, tol=tol, max_steps=max_steps)
                owner[cid] = (k, ax)
        res, active, queued = srv.run(batches=1)
        for r in res:
            k, ax = owner[r["id"]]
            statuses[r["status"]] = statuses.get(r["status"], 0) + 1
            requests[k].setdefault("k_app", [0.0, 0.0, 0.0])[ax] = r["k_app"]
            requests[k].setdefault("status", [None, None, None])[ax] = r["status"]
            left[k] -= 1
            if left[k] == 0:
                finished[k] = time.perf_counter() - t0 - arrivals[k]
        if not res and active == 0 and queued == 0 and pending:
            time.sleep(max(0.0, min(0.01, arrivals[pending[0]] - (time.perf_counter() - t0))))
    wall = time.perf_counter() - t0
    st = srv.stats()
    srv.close()
    lat = np.array([finished[k] for k in range(len(requests))])
    return {"wall_s": wall, "node_updates": st["node_updates"], "glups": st["node_updates"] / wall / 1e9,
            "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "kernel_launches": st["kernel_launches"], "statuses": {str(k): v for k, v in statuses.items()}}


def _plain_serial(lbm, requests, storage="fp16", check_every=100, tol=1e-7, max_steps=200000):
    """The same requests without the server: one case at a time, each a
    Simulation stepped with plain launches (three kernels per step, no graph),
    its residual and mean flow checked every check_every steps with the
    server's retirement rule."""
    t0 = time.perf_counter()
    updates = 0
    for req in requests:
        for ax in range(3):
            b = [0.0, 0.0, 0.0]
            b[ax] = 1e-6
            sim = lbm.Simulation(lbm.D3Q27, req["eps"], req["kappa"], viscosity=0.02, force=b,
                                 forchheimer=lbm.F_ERGUN, storage=storage, kernel="split", streaming="in_place")
            hist, means, steps = [], [], 0
            sim.reduce(snapshot=True)
            while True:
                sim.step(check_every)
                steps += check_every
                st = sim.reduce(snapshot=True)
                hist.append(st["residual"])
                means.append(st["mean_v"][ax])
                floor = len(hist) >= 10 and min(hist[-5:]) > 0.9 * min(hist[-10:-5])
                settled = len(means) >= 2 and abs(means[-1] - means[-2]) <= 10 * tol * abs(means[-1])
                if hist[-1] < tol or (floor and settled) or steps >= max_steps:
                    break
            updates += steps * sim.N
            sim.close()
    wall = time.perf_counter() - t0
    return {"wall_s": wall, "node_updates": updates, "glups": updates / wall / 1e9}


def serving_benchmark(lbm, n_requests, sides, seed=7):
    """Config of the serving workload: periodic D3Q27 cubes (sides drawn from
    `sides`), porosity clip(m + 0.1 g, 0.1, 1) with m ~ U[0.4, 0.9] and
    correlation length ~ U[4, 24], Carman-Kozeny permeability, nu = 0.02,
    force 1e-6 along each axis (3 cases per request, K_app diagonal), FP16
    storage, retirement at a 1e-7 change over 100 steps or at the storage noise
    floor, 60 GB admission cap.  First the same requests run one case at a time
    with plain launches (the baseline); their service rate sets the Poisson
    arrival rate of the batched run to twice that rate."""
    from paper_2606_29619_b300 import workloads

    reqs = [workloads.serving_request(k, sides=sides) for k in range(n_requests)]
    plain = _plain_serial(lbm, [dict(r) for r in reqs])
    rate = 2.0 * n_requests / plain["wall_s"]
    rng = np.random.default_rng(seed)
    arrivals = list(np.cumsum(rng.exponential(1.0 / rate, n_requests)))
    served = [dict(r) for r in reqs]
    batched = _serve(lbm, served, 60e9, arrivals)
    saturated = _serve(lbm, [dict(r) for r in reqs], 60e9, [0.0] * n_requests)
    # K_app of every request against the same request served with FP32 storage
    ref = [dict(r) for r in reqs]
    _serve(lbm, ref, 60e9, [0.0] * n_requests, storage="fp32")
    # over the cases that retired (converged or at the storage floor with a settled mean flow) in both runs
    errs, capped = [], 0
    for q, r in zip(served, ref):
        for a, b, sa, sb in zip(q["k_app"], r["k_app"], q["status"], r["status"]):
            if sa in (0, 1) and sb in (0, 1) and b != 0:
                errs.append(abs(a - b) / abs(b))
            else:
                capped += 1
    return {"requests": n_requests, "sides": list(sides), "arrival_rate_per_s": rate,
            "p50_ms": batched["p50_ms"], "p99_ms": batched["p99_ms"],
            "batched_poisson": batched, "batched_all_queued": saturated,
            "one_at_a_time_plain_launches": plain,
            "speedup_glups": saturated["glups"] / plain["glups"],
            "k_app_rel_err_vs_fp32": {"max": float(max(errs)) if errs else None,
                                      "median": float(np.median(errs)) if errs else None, "cases": len(errs),
                                      "not_retired": capped,
                                      "note": "FP16 served K_app against the same request served with FP32 "
                                              "storage; cases at the step cap in either run are counted apart"},
            "note": "batched_all_queued: every request queued at t=0 (throughput); "
                    "one_at_a_time_plain_launches: each case a Simulation stepped with plain launches, one after "
                    "another (the baseline; speedup_glups = batched_all_queued / it); batched_poisson: Poisson "
                    "arrivals at 2x the one-at-a-time service rate (latency)"}


def channel_case(lbm, storage, kernel, steps, shape=(256, 256, 512), side=128, U=0.05, nu=0.064, device=0):
    """The porous-cube channel: velocity inlet U at x = 0, pressure outlet rho = 1
    at x = nx - 1, bounce-back walls in y and z, centred cube of side `side`
    (eps = 0.4, Da = 1e-4 on the cube side, F = 0.55), Re = U side / nu."""
    import torch
    from paper_2606_29619_b300 import workloads

    nz, ny, nx = shape
    eps, kap = workloads.cube_channel(nx, ny, nz, side=side, eps_cube=0.4, Da=1e-4)
    stream = torch.cuda.Stream(device=device)
    sim = lbm.Simulation(lbm.D3Q27, eps, kap, viscosity=nu, forchheimer=0.55, storage=storage, kernel=kernel,
                         bc=("inflow_outflow", "wall", "wall"), inlet_v=(U, 0, 0), outlet_rho=1.0, stream=stream,
                         device=device)
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    start.record(stream)
    sim.step(steps)
    end.record(stream)
    end.synchronize()
    sim.sync()
    st = sim.reduce()
    rho, v = sim.moments()
    x0, y0, z0 = (nx - side) // 2, (ny - side) // 2, (nz - side) // 2
    xm = nx // 2
    vx = v[0, :, :, xm]
    total = vx.sum()
    frac = float(vx[z0:z0 + side, y0:y0 + side].sum() / total) if total != 0 else float("nan")
    sim.close()
    return {"storage": storage, "kernel": kernel, "steps": steps, "ms_per_step": start.elapsed_time(end) / steps,
            "glups": eps.size * steps / (start.elapsed_time(end) * 1e-3) / 1e9, "drag_x": st["drag"][0],
            "flow_fraction": frac, "mean_vx": st["mean_v"][0], "v": v}


def channel_benchmark(lbm, steps, kernel="split", storages=("fp64", "fp32", "fp16", "bf16")):
    """The channel's storage forms for `steps` steps from rest.  The inflow
    reaches the cube only after about 2,000 steps, so the FP64 reference and the
    drag, flow-fraction and velocity errors against it are taken from that many
    steps on; shorter runs report GLUPS only."""
    out = {}
    ref = None
    if steps < 2000:
        storages = tuple(s for s in storages if s != "fp64")
        out["note"] = "fewer than 2,000 steps: the flow has not reached the cube; GLUPS only"
    for stg in storages:
        r = channel_case(lbm, stg, "sweep" if stg == "fp64" else kernel, steps)
        v = r.pop("v")
        if steps < 2000:
            for k in ("drag_x", "flow_fraction", "mean_vx"):
                r.pop(k, None)
        elif ref is None:
            ref = (v, r)
        else:
            rv, rr = ref
            r["v_err_vs_fp64"] = float(np.max(np.sqrt(((v - rv) ** 2).sum(0))) / np.max(np.sqrt((rv ** 2).sum(0))))
            r["drag_rel_err_vs_fp64"] = abs(r["drag_x"] - rr["drag_x"]) / abs(rr["drag_x"])
            r["flow_fraction_abs_err_vs_fp64"] = abs(r["flow_fraction"] - rr["flow_fraction"])
        out[stg] = r
    return out


def slot_box_benchmark(lbm, steps, warmup, device, barrier, peak):
    """Config 5: the 640^3 slot box (porous box, seed 5, cut by a free slot 64
    nodes wide) with in-place streaming, FP32 and FP16 storage: GLUPS, the step
    against the HBM roofline, and FP16's velocity error against FP32 after the
    same steps."""
    eps, kap, w = make_inputs("slot_box_640")
    out, vs = {}, {}
    for st in ("fp32", "fp16"):
        r = time_storage(lbm, eps, kap, w, st, steps, warmup, device, barrier, kernel="split", keep_v=True,
                         streaming="in_place")
        vs[st] = r.pop("v")
        ach = algorithmic_bytes(st) * r["N"] / (r["ms_per_step"] * 1e-3) / 1e9
        out[st] = {"glups": r["N"] / (r["ms_per_step"] * 1e-3) / 1e9, "ms_per_step": r["ms_per_step"],
                   "roofline_frac": ach / peak, "kernel_ms": r["kernel_ms"], "in_place": r["in_place"]}
    vr = vs["fp32"]
    out["fp16"]["v_err_vs_fp32"] = float(np.max(np.sqrt(((vs["fp16"] - vr) ** 2).sum(axis=0)))
                                         / np.max(np.sqrt((vr ** 2).sum(axis=0))))
    out["grid"] = list(w["shape"])
    out["steps"] = steps
    return out


def run_reference(args, world, rank):
    """Reference arm: the FP64 CPU oracle on the host cores."""
    if rank != 0:
        return
    import oracle
    from paper_2606_29619_b300 import workloads

    name = args.workload
    w = WORKLOADS[name]
    shape = (32, 32, 32)
    eps, kap = workloads.porous_box(shape, ell=w["ell"], seed=w["seed"])
    o = oracle.Oracle(oracle.D3Q27, eps, kap, nu_f=w["nu"], b=w["b"], forch=-1.0).init()
    N = eps.size
    o.step(args.warmup)
    t0 = time.perf_counter()
    o.step(args.steps)
    dt = time.perf_counter() - t0
    cores = oracle.threads()
    value = N * args.steps / dt / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{name}_fp32", "grid": list(w["shape"]), "lattice": "D3Q27", "storage": "fp64",
                       "sample": "32^3 copy per step", "note": "the oracle computes and stores in FP64"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"D3Q27 32^3 copy of {name}, one FP64 oracle step per bench step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="porous_box_256", choices=sorted(WORKLOADS))
    ap.add_argument("--storages", default="fp32,fp16,bf16")
    ap.add_argument("--kernel", default="split", choices=["split", "fused"])
    ap.add_argument("--serving-requests", type=int, default=24)
    ap.add_argument("--channel-steps", type=int, default=200,
                    help="also run the 512x256x256 porous-cube channel for this many steps per storage form")
    ap.add_argument("--serving-sides", default="32,48,64,96")
    ap.add_argument("--slot-box-steps", type=int, default=100,
                    help="also run the 640^3 slot box in place (FP32 and FP16) for this many steps")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--e2e-steps", type=int, default=5000, help="steps of the end-to-end job (the workload's 5,000)")
    ap.add_argument("--in-place", default="fp32,fp16", help="storage forms also timed with in-place streaming")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default tile height (profiling runs)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    world, rank, local, pg = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
        return

    import torch

    import paper_2606_29619_b300 as lbm

    device = local
    torch.cuda.set_device(device)
    lbm.load_library()

    def barrier():
        if pg is not None:
            pg.barrier()

    eps, kap, w = make_inputs(args.workload)
    storages = [s for s in args.storages.split(",") if s]
    if storages[0] != "fp32":
        storages = ["fp32"] + [s for s in storages if s != "fp32"]
    peak, peak_kind = measured_peaks()
    results = {}
    # the autotuner's choices for this run (timed once per storage and streaming form, then read by the
    # end-to-end run's creation)
    tune_cache = os.path.join(tempfile.mkdtemp(prefix="lbm_tune_"), "tune.jsonl")
    inplace_forms = [s for s in args.in_place.split(",") if s] if args.kernel == "split" else []
    inplace = {}
    with ClockSampler(device) as clk:
        for st in storages:
            results[st] = time_storage(lbm, eps, kap, w, st, args.steps, args.warmup, device, barrier,
                                       kernel=args.kernel, keep_v=(rank == 0 and len(storages) > 1),
                                       streaming="two_arrays" if args.kernel == "split" else "auto",
                                       tune_cache=tune_cache, autotune=not args.no_autotune)
        for st in inplace_forms:
            inplace[st] = time_storage(lbm, eps, kap, w, st, args.steps, args.warmup, device, barrier,
                                       kernel="split", streaming="in_place", tune_cache=tune_cache,
                                       autotune=not args.no_autotune)
            inplace[st].pop("v")
    # velocity of each reduced storage form against the FP32 form after the same steps
    vref = results["fp32"].pop("v")
    for st in storages[1:]:
        vs = results[st].pop("v")
        if vref is not None and vs is not None:
            results[st]["v_err_vs_fp32"] = float(np.max(np.sqrt(((vs - vref) ** 2).sum(axis=0)))
                                                 / np.max(np.sqrt((vref ** 2).sum(axis=0))))
    del vref
    clocks = clk.summary()
    head = results["fp32"]
    ms = max_over_ranks(head["ms"], pg, device)
    N = head["N"]
    value = aggregate_glups(N, args.steps, ms, world)
    per_launch_s = head["ms_per_step"] * 1e-3 / head["launches_per_step"]

    def kernel_rooflines(st):
        r = results[st]
        kb = kernel_bytes(r["kernel"], st)
        src = "lbm_fused.cuh" if r["kernel"] == "fused" else "lbm_split.cuh"
        out = {}
        for name, ms_launch in r["kernel_ms"].items():
            achieved = kb[name] * r["N"] / (ms_launch * 1e-3) / 1e9
            out[name] = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "peak_source": f"{peak_kind} hbm_gbs", "algorithmic_bytes_per_node": kb[name],
                         "ms_per_launch": ms_launch,
                         "traffic": traffic_from_profile(f"{name}_{st}_{args.workload}", src)}
        return out

    def dominant_kernel(st):
        """The kernel with the largest share of the step, against its own bytes."""
        ks = kernel_rooflines(st)
        name = max(ks, key=lambda k: ks[k]["ms_per_launch"])
        return dict(ks[name], kernel=name)

    def roofline(st, r=None):
        """The whole step against the least traffic of a node update (populations
        read and written once, porosity and permeability read once); traffic: the
        DRAM bytes of the step's kernels per step, from the committed ncu summary."""
        r = results[st] if r is None else r
        achieved = algorithmic_bytes(st) * r["N"] / (r["ms_per_step"] * 1e-3) / 1e9
        traffic = None
        if r["kernel"] == "split":
            # in place: the moments and collide kernels are the in-place ones (lbm_inplace.cuh)
            parts = [("k_ip" + name[7:] if r.get("in_place") and name != "k_split_velocity" else name,
                      "lbm_inplace.cuh" if r.get("in_place") and name != "k_split_velocity" else "lbm_split.cuh")
                     for name in r["kernel_ms"]]
            t = [traffic_from_profile(f"{name}_{st}_{args.workload}", src) for name, src in parts]
            traffic = sum(t) if all(x is not None for x in t) else None
        return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "peak_source": f"{peak_kind} hbm_gbs", "algorithmic_bytes_per_node": algorithmic_bytes(st),
                "kernel": "the whole step (" + ", ".join(r["kernel_ms"]) + ")", "traffic": traffic}

    e2e = (e2e_run(lbm, eps, kap, w, args.e2e_steps, device, args.kernel, tune_cache, not args.no_autotune)
           if rank == 0 and args.e2e_steps > 0 else None)
    channel = channel_benchmark(lbm, args.channel_steps, args.kernel) if rank == 0 and args.channel_steps > 0 else None
    slot = (slot_box_benchmark(lbm, args.slot_box_steps, args.warmup, device, lambda: None, peak)
            if rank == 0 and args.slot_box_steps > 0 and args.kernel == "split" else None)
    serving = None
    if rank == 0 and args.serving_requests > 0:
        serving = serving_benchmark(lbm, args.serving_requests, [int(x) for x in args.serving_sides.split(",")])
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.cpu_seconds, args.workload)
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{args.workload}_fp32", "grid": list(w["shape"]), "lattice": "D3Q27",
                       "storage": "fp32", "nu": w["nu"], "force": list(w["b"]), "kernel": head["kernel"],
                       "tile_y": head["tuning"]["tile_y"],
                       "parallelism": f"replicas{world}", "l2": "populations exceed L2 (no flush needed)"},
            "roofline": roofline("fp32"),
            "dominant_kernel": dominant_kernel("fp32"),
            "storage_forms": {st: {"glups": results[st]["N"] / (results[st]["ms_per_step"] * 1e-3) / 1e9,
                                   "ms_per_step": results[st]["ms_per_step"], "roofline": roofline(st),
                                   "dominant_kernel": dominant_kernel(st), "kernels": kernel_rooflines(st),
                                   "v_err_vs_fp32": results[st].get("v_err_vs_fp32"),
                                   "tuning": results[st]["tuning"]}
                              for st in storages},
            "in_place": {st: {"glups": r["N"] / (r["ms_per_step"] * 1e-3) / 1e9, "ms_per_step": r["ms_per_step"],
                              "roofline": roofline(st, r), "kernel_ms": r["kernel_ms"], "tuning": r["tuning"],
                              "note": "one population array (AA-pattern streaming); layout alternates per step"}
                         for st, r in inplace.items()},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "serving": serving,
            "channel": channel,
            "slot_box_640": slot,
            "gpu_launches": int(head["launches_per_step"] * args.steps),
            "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    if pg is not None:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
