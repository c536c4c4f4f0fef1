"""Throughput of the CS and FD lattice Boltzmann hot path on GB300.

One step = one pass of the whole path over the roofline workload, advanced
together as one batch: a CS D2Q9 step on an 8192^2 lattice (collide + stream,
one launch), an FD 16-velocity step on a 4096^2 lattice (three SSP-RK3 stage
launches with WENO-5 and BGK), and the fused float64 observables (mass,
momentum, Taylor-Green amplitude) of both lattices. Storage is FP32
deviations; both states are far larger than L2 (2.4 GB and 3.2 GB), so
nothing is flushed between steps.

Metric: MLUPS (million lattice-node updates per second) over the workload,
whole job (all ranks); per-kernel CUDA-event durations give the roofline
fractions of the dominant kernel (the FD stage) against the FP32 peak and
the measured HBM copy bandwidth. The same line carries the end-to-end rate
through the public API (host fields in, observables out), the batched
(256 mixed lattices, FP32 vs FP64 one at a time) and served (Poisson stream)
legs, and the FP64 oracle's rate on every host core (cpu_baseline).

--impl reference times the FP64 C oracle on the host cores instead (the
paper publishes no implementation or timings), on bounded samples, one
oracle process per core. --served-full N runs only the served stream in its
full configuration (lattices 64^2..4096^2, 1k..20k steps; several minutes).
Multi-GPU: replicas only (each rank advances its own copy; no collective on
the data path).
"""
from __future__ import annotations

import argparse
import json
import re
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import lbm_workloads as wl  # noqa: E402

CS_N = 8192
FD_N = 4096
FD_DT = 1e-5
FD_TAU = 5e-4
CS_TAU = 0.8 / math.sqrt(3.0)
U0 = 0.01
FD_CFL = 0.4
METRIC = "MLUPS & % HBM roofline, CS and FD; batched FP32 vs plain FP64; p50/p99"
WORKLOAD = "roofline lattices: CS D2Q9 8192^2 + FD 16-velocity 4096^2, FP32 deviation storage, Taylor-Green"
# algorithmic bytes per lattice update (FP32): CS reads and writes 9 values;
# an FD step reads Q, 2Q, 2Q and writes Q, Q, Q values over its three stages.
CS_BYTES_LU = 18 * 4
FD_BYTES_LU = 8 * 16 * 4
# Algorithmic FP32 flops of one FD lattice update (3 RK stages, 16
# populations), counted from the textbook formulas, every +, -, x, / one flop:
# per population and stage two WENO-5 interfaces (one per axis; an interface
# is shared by the two nodes it separates) of 64 flops each (candidates 15,
# smoothness indicators 30, weights 19) plus 3 for the flux difference, 13 for
# the equilibrium, BGK and stage combination, 3 for the moments.
WENO5_FLOPS = 64
FD_FLOPS_LU = 3 * 16 * (2 * (WENO5_FLOPS + 3) + 13 + 3)
# FP32 peak from unit counts and clock: 152 SMs x 128 FP32 lanes x 2 flops
# (an FMA) x 2.07 GHz.
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
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
            for nm, v in zip(names, parts[5:9]):
                if v.lower() in ("active", "1"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- CPU oracle
def oracle_rates(budget_s: float = 12.0):
    """Seconds per lattice update of the FP64 C oracle (single thread) on this
    host: CS D2Q9 and FD 16-velocity, timed on bounded samples."""
    import oracle
    out = {}
    n = 512
    rho, ux, uy = wl.taylor_green(n, n, U0 * math.sqrt(3))
    f = oracle.equilibrium(3, rho, ux, uy)
    oracle.cs_run(f, CS_TAU, 1)
    steps, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < budget_s * 0.25:
        f = oracle.cs_run(f, CS_TAU, 2)
        steps += 2
    out["cs"] = (time.perf_counter() - t0) / (steps * n * n)
    out["cs_sample"] = f"CS D2Q9 {n}^2 x {steps} steps"
    n = 128
    rho, ux, uy = wl.taylor_green(n, n, U0)
    f = oracle.equilibrium(4, rho, ux, uy)
    steps, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < budget_s * 0.75:
        f = oracle.fd_run(f, 1.0 / n, 2e-4, FD_TAU, 1)
        steps += 1
    out["fd"] = (time.perf_counter() - t0) / (steps * n * n)
    out["fd_sample"] = f"FD 16-velocity {n}^2 x {steps} steps"
    return out


def host_cores() -> int:
    """Cores this process may run on (its CPU set), else the machine's count."""
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def _oracle_worker(budget_s: float):
    return oracle_rates(budget_s)


def oracle_pool(nproc: int):
    """One worker process per host core for the oracle. Spawned, not forked:
    no CUDA state of the parent is inherited. The oracle library is built
    once here first, so the workers only load it."""
    import multiprocessing as mp
    from oracle import build as oracle_build
    oracle_build.build()
    return mp.get_context("spawn").Pool(nproc)


def oracle_rates_all_cores(pool, nproc: int, budget_s: float):
    """The oracle's bounded samples on every host core at once: one
    independent single-thread oracle run per core, all timed over the same
    wall-clock window. Returns the per-process rates."""
    return pool.map(_oracle_worker, [budget_s] * nproc)


def cpu_value(rates):
    cells = CS_N * CS_N + FD_N * FD_N
    per_step = CS_N * CS_N * rates["cs"] + FD_N * FD_N * rates["fd"]
    return cells / per_step / 1e6


# ---------------------------------------------------------------- GPU arm
def build_batch(torch, stream):
    import paper_1904_02471_gb300 as pkg
    specs = [pkg.make_spec("cs", 3, CS_N, CS_N, CS_TAU, 0.0, 0.0, "fp32", storage="inplace"),
             pkg.make_spec("fd", 4, FD_N, FD_N, FD_TAU, FD_DT, 0.0, "fp32")]
    B = pkg.Batch(specs, stream=stream)
    fields = []
    for i, (n, U) in enumerate(((CS_N, U0 * math.sqrt(3)), (FD_N, U0))):
        rho, ux, uy = wl.taylor_green(n, n, U)
        pin = [torch.from_numpy(a).pin_memory().numpy() for a in (rho, ux, uy)]
        fields.append(pin)
        comp, px, py, norm = wl.probe_taylor_green(n, n)
        B.set_probe(i, comp, px, py, norm)
    return B, fields


def run_gpu(args, rank, world):
    import torch
    import paper_1904_02471_gb300 as pkg  # noqa: F401
    from paper_1904_02471_gb300 import build
    build.build()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    rates, rates_all, ncores = None, None, host_cores()
    if rank == 0 and not args.no_cpu_baseline:
        rates = oracle_rates(args.cpu_budget)
        with oracle_pool(ncores) as pool:
            rates_all = oracle_rates_all_cores(pool, ncores, args.cpu_budget)

    stream = torch.cuda.Stream()
    B, fields = build_batch(torch, stream)
    for i in range(2):
        B.init(i, *fields[i])
    tune_report = B.tune(2)
    groups = B.groups()
    cap = args.warmup + args.steps + 8
    for i in range(2):
        B.record(i, 1, cap)
    B.step_profiled(args.warmup)

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    l0 = B.kernel_launches
    w0 = time.perf_counter()
    torch.cuda.nvtx.range_push("bench_timed")  # lets a profiler select the timed region
    ms, total_ms = B.step_profiled(args.steps)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    wall = time.perf_counter() - w0
    launches = B.kernel_launches - l0
    if dist:
        dist.barrier()
    clk = clocks.stop()
    from paper_1904_02471_gb300 import replicas
    t_max = replicas.job_time(dist, total_ms, device="cuda")

    # check the run stayed finite and conserved mass (float64 sums)
    ser = [B.series(i) for i in range(2)]
    finite = all(s["nonfinite"] == 0 for sr in ser for s in sr)
    drift = [abs(sr[-1]["mass"] - sr[0]["mass"]) / sr[0]["mass"] for sr in ser]

    # e2e through the public API: host fields in (pinned), K steps, observables out
    # One untimed pass of the same sequence first (as the device timing has
    # warm-up steps): on this host the first DMA over a large, freshly pinned
    # buffer also pays for its address translations; its time is reported.
    def e2e_pass():
        torch.cuda.synchronize()
        e0 = time.perf_counter()
        for i in range(2):
            B.init(i, *fields[i])   # returns after the state is on the device
        e1 = time.perf_counter()
        B.step(args.steps)
        B.sync()
        e2 = time.perf_counter()
        obs = [B.observables(i) for i in range(2)]
        e3 = time.perf_counter()
        return obs, e3 - e0, {"init_ms": round((e1 - e0) * 1e3, 2), "steps_ms": round((e2 - e1) * 1e3, 2),
                              "observables_ms": round((e3 - e2) * 1e3, 2)}
    _, warm_wall, _ = e2e_pass()
    obs, e_wall, e_parts = e2e_pass()
    e_parts["untimed_warmup_pass_ms"] = round(warm_wall * 1e3, 2)
    assert all(o["nonfinite"] == 0 for o in obs)
    h2d = sum(a.nbytes for fl in fields for a in fl) / args.steps
    d2h = 2 * 48 / args.steps

    peak, peak_kind = peaks()
    gi = {(g["model"], g["q"]): k for k, g in enumerate(groups)}
    gcs, gfd = gi[(0, 3)], gi[(1, 4)]
    K = args.steps
    cs_ms = ms[gcs][0] / K
    fd_stage_ms = [ms[gfd][s] / K for s in range(3)]
    fin_ms = (ms[gcs][3] + ms[gfd][3]) / K
    cells = CS_N * CS_N + FD_N * FD_N
    value = replicas.whole_job_rate(cells * K, world, t_max / 1e3) / 1e6
    cs_gbs = CS_N * CS_N * CS_BYTES_LU / (cs_ms / 1e3) / 1e9
    fd_stage_avg = sum(fd_stage_ms) / 3
    fd_gbs = FD_N * FD_N * FD_BYTES_LU / 3 / (fd_stage_avg / 1e3) / 1e9
    fd_tflops = FD_N * FD_N * FD_FLOPS_LU / 3 / (fd_stage_avg / 1e3) / 1e12
    fd_ty = fd_tile_height(tune_report, gfd)
    traffic = committed_traffic()
    rec = {
        "metric": METRIC,
        "value": round(value, 2),
        "unit": "MLUPS",
        "n_gpus": world,
        "steps": K,
        "warmup": args.warmup,
        "ms_per_step": round(t_max / K, 4),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic (Taylor-Green initial state, seeded generators)",
        "config": {
            "workload": WORKLOAD,
            "cs": {"lattice": [CS_N, CS_N], "tau_lu": CS_TAU, "velocities": 9,
                   "storage": "in place (one buffer, AA access pattern)"},
            "fd": {"lattice": [FD_N, FD_N], "tau_fd": FD_TAU, "dt_fd": FD_DT, "velocities": 16,
                   "scheme": "WENO-5 + SSP-RK3, 3 stage launches"},
            "observables": "fused float64 mass/momentum/amplitude every step",
            "l2": "inputs larger than L2 (2.4 GB + 3.2 GB resident state), no flush",
            "parallelism": f"replicas x{world}",
            "tuning": tune_report.strip(),
        },
        "per_model": {
            "cs": {"mlups": round(CS_N * CS_N / (cs_ms / 1e3) / 1e6, 1), "ms_per_step": round(cs_ms, 4),
                   "gbs": round(cs_gbs, 1), "frac_hbm": round(cs_gbs / peak, 3), "bytes_per_lu": CS_BYTES_LU},
            "fd": {"mlups": round(FD_N * FD_N / (sum(fd_stage_ms) / 1e3) / 1e6, 1),
                   "ms_per_step": round(sum(fd_stage_ms), 4), "stage_ms": [round(x, 4) for x in fd_stage_ms],
                   "gbs": round(fd_gbs, 1), "frac_hbm": round(fd_gbs / peak, 3), "bytes_per_lu": FD_BYTES_LU},
            "finalize_ms_per_step": round(fin_ms, 4),
        },
        "roofline": {"kernel": f"fd_stage_kernel<float,4,{fd_ty}> (FD RK stage, Q=16)", "bound": "alu",
                     "achieved": round(fd_tflops, 2), "peak": round(FP32_PEAK_TFLOPS, 1), "unit": "TFLOP/s",
                     "frac": round(fd_tflops / FP32_PEAK_TFLOPS, 4),
                     "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 flops x 2070 MHz",
                     "traffic": traffic.get("fd_stage") if traffic else None,
                     "algorithmic_flops_per_launch": FD_N * FD_N * FD_FLOPS_LU // 3,
                     "algorithmic_bytes_per_launch": FD_N * FD_N * FD_BYTES_LU // 3,
                     "hbm": {"achieved": round(fd_gbs, 1), "peak": peak, "unit": "GB/s",
                             "frac": round(fd_gbs / peak, 4), "peak_source": peak_kind}},
        "e2e": {"value": round(world * cells * K / e_wall / 1e6, 2), "unit": "MLUPS",
                "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h), "parts": e_parts},
        "gpu_launches": int(launches),
        "clocks": clk,
        "checks": {"finite": finite, "rel_mass_drift": [float(f"{d:.3e}") for d in drift],
                   "host_wall_s": round(wall, 4)},
    }
    if not args.no_extras:
        rec["batched"] = run_batched(torch)
        rec["served"] = run_served(torch)
    if rates is not None:
        rec["cpu_baseline"] = {
            "value": round(sum(cpu_value(r) for r in rates_all), 4), "unit": "MLUPS", "cores": ncores, "kind": "oracle",
            "sample": f"{rates['cs_sample']}; {rates['fd_sample']}; FP64 C oracle, one independent single-thread "
                      f"process per host core ({ncores}) on the same samples at once, rates summed; rates "
                      "extrapolated per node update to the workload mix",
            "single_core_value": round(cpu_value(rates), 4)}
    B.close()
    if dist:
        dist.destroy_process_group()
    return rec


# ---------------------------------------------------------------- batched + served
def _instance_spec(pkg, d, prec):
    """Spec of one batched/served instance: CS D2Q9 with tau_LU = tau*/sqrt 3
    (FP32: in-place storage), or FD 16-velocity with tau_FD from Eq.
    (nu-transfer) and the largest stable time step (CFL and dt <= tau)."""
    n = d["n"]
    tau_lu = d["tau_star"] / math.sqrt(3.0)
    if d["model"] == "cs":
        return pkg.make_spec("cs", 3, n, n, tau_lu, 0.0, 0.0, prec, storage="inplace" if prec == "fp32" else "ab")
    tau_fd = pkg.lbm_tau_fd_from_lu(n, tau_lu)
    return pkg.make_spec("fd", 4, n, n, tau_fd, fd_dt(pkg, 4, n, tau_fd), 0.0, prec)


def fd_dt(pkg, q, n, tau_fd, cfl=FD_CFL):
    """FD time step of the synthetic workloads: dt <= tau (Sec. 4.1) and a
    Courant number max|v| dt/dx of FD_CFL. CFL = 1, the bound Sec. 4.1 states
    for its quasi-1D runs, is not stable for WENO-5 + RK3 advection along
    both axes at once."""
    return min(tau_fd, cfl * pkg.lbm_fd_max_dt(q, 1.0 / n, 1e300))


def _fields(d):
    n = d["n"]
    U = U0 * (math.sqrt(3.0) if d["model"] == "cs" else 1.0)
    return wl.shear_wave(n, n, U) if d.get("init") == "shear" else wl.taylor_green(n, n, U)


def run_batched(torch, steps=192, plain_steps=2):
    """256 independent lattices (sides from {32..512}, tau* in [0.51, 2], half
    CS, half FD 16-velocity): all advanced together in FP32 (one persistent
    launch per group and step, graph replays) against the plain form, each
    lattice alone in FP64, one at a time."""
    import paper_1904_02471_gb300 as pkg
    inst = wl.batched_instances(256, seed=0)
    cells = sum(d["n"] ** 2 for d in inst)
    B = pkg.Batch([_instance_spec(pkg, d, "fp32") for d in inst])
    for i, d in enumerate(inst):
        B.init(i, *_fields(d))
    tune = B.tune(2)
    B.step(32)
    B.sync()
    t0 = time.perf_counter()
    B.step(steps)
    B.sync()
    t_b = time.perf_counter() - t0
    mlups_b = cells * steps / t_b / 1e6
    # accuracy of the FP32 batch against FP64 runs of the same lattices
    probe = [i for i, d in enumerate(inst) if d["n"] <= 64][:4]
    got = {i: B.moments(i) for i in probe}
    done = B.steps_done(probe[0]) if probe else 0
    B.close()
    err = 0.0
    for i in probe:
        d = inst[i]
        with pkg.Lattice(**_lat_kwargs(pkg, d, "fp64")) as L:
            L.init(*_fields(d))
            L.step(done)
            _, u, v = L.moments()
        U = U0 * (math.sqrt(3.0) if d["model"] == "cs" else 1.0)
        err = max(err, float(np.max(np.abs(got[i][1] - u))) / U, float(np.max(np.abs(got[i][2] - v))) / U)
    # plain: FP64, one lattice at a time
    t_plain, work = 0.0, 0
    per_model = {"cs": [0, 0.0], "fd": [0, 0.0]}
    for d in inst:
        with pkg.Lattice(**_lat_kwargs(pkg, d, "fp64")) as L:
            L.init(*_fields(d))
            L.step(1)
            L.sync()
            t0 = time.perf_counter()
            L.step(plain_steps)
            L.sync()
            dt = time.perf_counter() - t0
        t_plain += dt
        work += d["n"] ** 2 * plain_steps
        per_model[d["model"]][0] += d["n"] ** 2 * plain_steps
        per_model[d["model"]][1] += dt
    mlups_p = work / t_plain / 1e6
    return {
        "workload": "256 lattices, sides uniform in {32,64,128,256,512}, tau* U[0.51,2], half CS D2Q9 / half FD "
                    "16-velocity, shear-wave and Taylor-Green initial states (seed 0); FP32 CS in place",
        "cells": cells,
        "fp32_batched": {"mlups": round(mlups_b, 1), "steps": steps, "s": round(t_b, 4), "tuning": tune.strip()},
        "fp64_plain_one_at_a_time": {
            "mlups": round(mlups_p, 2), "steps_each": plain_steps,
            "cs_mlups": round(per_model["cs"][0] / max(per_model["cs"][1], 1e-12) / 1e6, 2),
            "fd_mlups": round(per_model["fd"][0] / max(per_model["fd"][1], 1e-12) / 1e6, 2)},
        "speedup": round(mlups_b / mlups_p, 1),
        "fp32_vs_fp64_max_rel_velocity_error": float(f"{err:.3e}"),
        "accuracy_sample": f"{len(probe)} lattices (side <= 64) after {done} steps",
    }


def _lat_kwargs(pkg, d, prec):
    s = _instance_spec(pkg, d, prec)
    return dict(model="cs" if s.model == 0 else "fd", q=s.q_per_axis, nx=s.nx, ny=s.ny, tau=s.tau, dt=s.dt,
                precision=prec)


def run_served(torch, n_req=100, seed=0, sides=(64, 128, 256, 512, 1024), steps=(1000, 5000), duration_s=30.0,
               rate_per_s=None, budget_gb=64):
    """Served stream: Poisson arrivals of CS / FD Taylor-Green runs (FP32)
    into the continuous-batching server; latency = completion - arrival.
    The arrival rate is n_req / duration_s unless rate_per_s is given."""
    import paper_1904_02471_gb300 as pkg
    from paper_1904_02471_gb300 import lbm
    rate = rate_per_s if rate_per_s else n_req / duration_s
    reqs = wl.served_stream(n_req, seed, rate_per_s=rate, sides=sides, steps=steps)
    work = sum(r["n"] ** 2 * r["steps"] for r in reqs)
    S = lbm.Server(budget_gb << 30, 256, 128)
    t0 = time.perf_counter()
    tickets = []
    for r in reqs:
        delay = r["arrival"] - (time.perf_counter() - t0)
        if delay > 0:
            time.sleep(delay)
        spec = _instance_spec(pkg, {"model": r["model"], "n": r["n"], "tau_star": r["tau_star"]}, "fp32")
        U = U0 * (math.sqrt(3.0) if r["model"] == "cs" else 1.0)
        tickets.append(S.submit(lbm.make_request(spec, r["steps"], "tg", U, obs_every=0)))
    S.drain(7200)
    res = [S.poll(t) for t in tickets]
    S.close()
    lat = sorted(x["t_done"] - x["t_submit"] for x in res)
    makespan = max(x["t_done"] for x in res) - min(x["t_submit"] for x in res)
    ok = sum(1 for x in res if x["status"] == 0)
    span = reqs[-1]["arrival"]
    return {
        "workload": f"{n_req} Poisson arrivals (seed {seed}) over ~{span:.0f} s, CS or FD 16-velocity "
                    f"Taylor-Green, sides {sides[0]}..{sides[-1]} (powers of 2), steps U[{steps[0]},{steps[1]}], FP32 "
                    "(CS in place)",
        "requests": n_req, "completed_ok": ok,
        "aggregate_mlups": round(work / makespan / 1e6, 1),
        "latency_s": {"p50": round(float(np.percentile(lat, 50)), 4), "p99": round(float(np.percentile(lat, 99)), 4),
                      "max": round(lat[-1], 4)},
        "makespan_s": round(makespan, 3),
    }


def lattice_rates(torch, sides, steps=8):
    """Single-lattice FP32 rates (lattice updates per second) of the served
    instance kinds, CS (in place) and FD 16-velocity, per side: a few steps
    of one lattice alone after one untimed step."""
    import paper_1904_02471_gb300 as pkg
    rates = {}
    for model in ("cs", "fd"):
        for n in sides:
            d = {"model": model, "n": n, "tau_star": 0.8}
            s = _instance_spec(pkg, d, "fp32")
            with pkg.Lattice(model, s.q_per_axis, n, n, s.tau, dt=s.dt, precision="fp32",
                             storage="inplace" if model == "cs" else "ab") as L:
                L.init(*_fields(d))
                L.step(1)
                L.sync()
                k = steps if model == "fd" and n > 512 else 64 * steps
                t0 = time.perf_counter()
                L.step(k)
                L.sync()
                rates[(model, n)] = n * n * k / (time.perf_counter() - t0)
    return rates


def run_served_full(torch, n_req, loads, seed=0):
    """The served-stream configuration in full: sides 64^2..4096^2, 1k..20k
    steps. The arrival rate is set to `load` times an estimate of the
    capacity: the mean service time of a request of the stream, each lattice
    run alone at its measured single-lattice rate (an underestimate of the
    server's capacity, which batches small lattices)."""
    sides = (64, 128, 256, 512, 1024, 2048, 4096)
    steps = (1000, 20000)
    rates = lattice_rates(torch, sides)
    probe = wl.served_stream(n_req, seed, rate_per_s=1.0, sides=sides, steps=steps)
    service = sum(r["n"] ** 2 * r["steps"] / rates[(r["model"], r["n"])] for r in probe) / n_req
    out = {"metric": "served stream, full configuration", "unit": "MLUPS", "dtype": "f32",
           "data": "synthetic (Taylor-Green initial states, seeded arrivals)",
           "single_lattice_mlups": {f"{m}{n}": round(v / 1e6, 1) for (m, n), v in rates.items()},
           "mean_service_s_alone": round(service, 3), "runs": []}
    for load in loads:
        rec = run_served(torch, n_req=n_req, seed=seed, sides=sides, steps=steps, rate_per_s=load / service,
                         budget_gb=128)
        rec["load"] = load
        rec["rate_per_s"] = round(load / service, 5)
        out["runs"].append(rec)
    return out


def fd_tile_height(report, gi):
    """Tile height of the FD group's kernel variant, from the tuner's report."""
    m = re.search(rf"\[g{gi} FD q4 fp32 (cached )?tile=(\d+)(x(\d+))?", report)
    if not m:
        return "*"
    if m.group(4):
        return m.group(4)
    return {0: "8", 1: "4", 2: "16", 3: "2"}.get(int(m.group(2)), "*")


def committed_traffic():
    """DRAM bytes per launch from the committed ncu summary, per kernel, for
    the kernels whose sources have not changed since it was taken."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    try:
        from paper_1904_02471_gb300 import build
        with open(p) as fh:
            d = json.load(fh)
        return {k: v["bytes_per_launch"] for k, v in d.get("kernels", {}).items()
                if v.get("source_digest") == build.kernel_digest(k)}
    except Exception:
        return None


# ---------------------------------------------------------------- reference arm
def run_reference(args, rank, world):
    if rank != 0:
        return None
    import oracle  # noqa: F401
    ncores = host_cores()
    vals, per_steps = [], []
    rates = None
    with oracle_pool(ncores) as pool:
        for s in range(args.warmup + args.steps):
            rs = oracle_rates_all_cores(pool, ncores, args.cpu_budget / max(1, args.steps))
            if s >= args.warmup:
                v = sum(cpu_value(r) for r in rs)
                vals.append(v)
                per_steps.append((CS_N * CS_N + FD_N * FD_N) / (v * 1e6))
            rates = rs[0]
    val = statistics.median(vals)
    per_step_s = statistics.median(per_steps)
    sample = (f"{rates['cs_sample']}; {rates['fd_sample']} per step and process; FP64 C oracle, one independent "
              f"single-thread process per host core ({ncores}) at once, rates summed")
    return {
        "impl": "reference", "metric": METRIC, "value": round(val, 4), "unit": "MLUPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(per_step_s * 1e3, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (Taylor-Green initial state)",
        "config": {"workload": WORKLOAD, "reference": "plain FP64 C oracle (no published implementation)"},
        "cpu_baseline": {"value": round(val, 4), "unit": "MLUPS", "cores": ncores, "kind": "oracle", "sample": sample},
        "e2e": {"value": round(val, 4), "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-budget", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the batched and served sections")
    ap.add_argument("--served-full", type=int, default=0, metavar="N_REQ",
                    help="only run the served stream in its full configuration (sides up to 4096^2, up to 20k "
                         "steps) with N_REQ requests, at each --served-load, and print that record")
    ap.add_argument("--served-load", type=float, nargs="+", default=[1.0, 1.5])
    args = ap.parse_args()
    if args.served_full:
        import torch
        torch.cuda.init()
        print(json.dumps(run_served_full(torch, args.served_full, args.served_load)))
        return
    if args.warmup < 3:
        args.warmup = 3
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        rec = run_reference(args, rank, world)
    else:
        rec = run_gpu(args, rank, world)
    if rank == 0 and rec is not None:
        print(json.dumps(rec))


if __name__ == "__main__":
    main()
