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
fractions of the dominant kernel (the FD stage) against the FP32 peak
measured on the same GPU and the measured HBM copy bandwidth. The same line
carries the end-to-end rate through the public API (host fields in,
observables out); the batched leg (256 mixed lattices in FP32 against each
lattice alone in FP64 for the same steps, with the FP32 velocity and
decay-rate errors); the served leg (a Poisson stream of CS / FD runs of
64^2..4096^2 nodes and 1k..20k steps into the continuous-batching server:
p50/p99 latency and slowdown, aggregate rate against the plain FP64 form of
the same request list run one at a time, FP32 errors of every run up to
256^2 against FP64); the IMEX leg (FD 16-velocity 4096^2 with tau below the
Courant-limited step: RK3 at dt = tau against IMEX at the Courant limit); the
fused leg (FD 16-velocity 4096^2, the temporally blocked RK3 step against the
three stage launches);
and the FP64 oracle's rate on every host core (cpu_baseline).

--impl reference times the FP64 C oracle on the host cores instead (the
paper publishes no implementation or timings), on bounded samples, one
oracle process per core. --served-full N runs only the served stream with N
requests at each --served-load. --profile-case cs|fd runs one small lattice
for kernel profiling. Multi-GPU: replicas only (each rank advances its own
copy; no collective on the data path).
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
# Nominal FP32 rate per SM and clock, for context beside the measured peak:
# 128 FP32 lanes x 2 flops (an FMA) per cycle.
FP32_FLOPS_PER_SM_CYCLE = 128 * 2


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
    # FP32 peak of this GPU, measured (packed FP32x2 fused multiply-adds on
    # every SM; the FD stage kernel's WENO-5 arithmetic is packed the same way)
    from paper_1904_02471_gb300 import lbm as _lbm
    fp32_flops, n_sm, _ = _lbm.probe_fp32(True)
    fp32_scalar, _, _ = _lbm.probe_fp32(False)
    fp32_peak = fp32_flops / 1e12
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
                     "achieved": round(fd_tflops, 2), "peak": round(fp32_peak, 2), "unit": "TFLOP/s",
                     "frac": round(fd_tflops / fp32_peak, 4),
                     "peak_source": f"measured on this GPU: independent packed FP32x2 fused multiply-add chains "
                                    f"on all {n_sm} SMs, CUDA events (lbm_probe_fp32); one FMA per instruction: "
                                    f"{fp32_scalar / 1e12:.2f} TFLOP/s; nominal {n_sm} SMs x 256 flops/cycle x "
                                    f"{(clk.get('sm_mhz') or 2070):.0f} MHz = "
                                    f"{n_sm * FP32_FLOPS_PER_SM_CYCLE * (clk.get('sm_mhz') or 2070) / 1e6:.1f}",
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
        rec["imex"] = run_imex(torch)
        rec["fused"] = run_fused(torch)
        rec["served"] = run_served(torch, n_req=args.served_requests, load=args.served_load[0],
                                   chunk=args.served_chunk)
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


def _probe(d, n):
    """Amplitude probe of an instance's initial mode (shear or Taylor-Green)."""
    return wl.probe_shear(n, n) if d.get("init") == "shear" else wl.probe_taylor_green(n, n)


def _decay_rates(s32, s64, skip_frac=0.25, floor=1e-3):
    """Decay rates gamma (A ~ exp(-gamma t)) of an FP32 and an FP64 amplitude
    series of the same run, each by the library's log-linear least squares
    over the same window: t >= skip_frac * t_end, and only while the FP64
    amplitude is above `floor` times its start (past that an FP32 amplitude
    sits at its rounding floor, far below which FP64 keeps decaying).
    Returns (g32, g64, ln(A0/A_end) of FP64 over the window)."""
    import paper_1904_02471_gb300 as pkg
    t = np.array([o["time"] for o in s64])
    a64 = np.array([o["amp"] for o in s64])
    a32 = np.array([o["amp"] for o in s32])[:len(t)]
    keep = np.abs(a64) >= floor * abs(a64[0])
    last = int(np.argmin(keep)) if not keep.all() else len(t)
    last = max(last, 4)
    t, a64, a32 = t[:last], a64[:last], a32[:last]
    skip = skip_frac * t[-1]
    g32, _ = pkg.lbm_fit_decay(t, a32, skip)
    g64, _ = pkg.lbm_fit_decay(t, a64, skip)
    return g32, g64, float(math.log(abs(a64[0]) / abs(a64[-1])))


def _error_summary(vel, rate, lnd, what, resolved=0.05):
    """max relative velocity error and relative decay-rate error over a set of
    lattices (FP32 against FP64 of the same lattice and steps); the decay-rate
    error also over the lattices whose amplitude decayed by at least
    ln(A0/A) = `resolved` in the fit window (smaller decays are resolved by
    FP32 only to its rounding of the amplitude)."""
    rate, lnd = np.array(rate), np.array(lnd)
    res = rate[lnd >= resolved]
    return {
        "max_rel_velocity_error": float(f"{max(vel):.3e}"),
        "rel_decay_rate_error": {"max": float(f"{rate.max():.3e}"), "median": float(f"{np.median(rate):.3e}"),
                                 f"max_where_decay_ln_ge_{resolved}": float(f"{res.max():.3e}") if len(res) else None,
                                 f"lattices_where_decay_ln_ge_{resolved}": int(len(res))},
        "lattices": len(vel),
        "amplitude_decay_ln_range": [float(f"{lnd.min():.3e}"), float(f"{lnd.max():.3e}")],
        "how": what,
    }


def run_batched(torch, steps=192, warm=32, every=16, max_err_side=256):
    """256 independent lattices (sides from {32..512}, tau* in [0.51, 2], half
    CS, half FD 16-velocity): all advanced together in FP32 (one persistent
    launch per group and step, graph replays) against the plain form, each
    lattice alone in FP64, one at a time, for the same steps. Accuracy: every
    lattice of side <= max_err_side, FP32 batched against its FP64 run."""
    import paper_1904_02471_gb300 as pkg
    inst = wl.batched_instances(256, seed=0)
    cells = sum(d["n"] ** 2 for d in inst)
    cap = (warm + steps) // every + 2
    B = pkg.Batch([_instance_spec(pkg, d, "fp32") for d in inst])
    for i, d in enumerate(inst):
        B.init(i, *_fields(d))
        B.set_probe(i, *_probe(d, d["n"]))
    tune = B.tune(2)
    for i in range(len(inst)):
        B.record(i, every, cap)
    B.step(warm)
    B.sync()
    t0 = time.perf_counter()
    B.step(steps)
    B.sync()
    t_b = time.perf_counter() - t0
    mlups_b = cells * steps / t_b / 1e6
    sample = [i for i, d in enumerate(inst) if d["n"] <= max_err_side]
    got = {i: (B.moments(i), B.series(i)) for i in sample}
    B.close()
    # plain: FP64, one lattice at a time, the same warm-up and timed steps
    t_plain, work = 0.0, 0
    per_model = {"cs": [0, 0.0], "fd": [0, 0.0]}
    vel, rate, lnd = [], [], []
    for i, d in enumerate(inst):
        with pkg.Lattice(**_lat_kwargs(pkg, d, "fp64")) as L:
            L.init(*_fields(d))
            L.set_probe(*_probe(d, d["n"]))
            L.record(every, cap)
            L.step(warm)
            L.sync()
            t0 = time.perf_counter()
            L.step(steps)
            L.sync()
            dt = time.perf_counter() - t0
            if i in sample:
                (_, u32, v32), ser32 = got[i]
                _, u64, v64 = L.moments()
                U = U0 * (math.sqrt(3.0) if d["model"] == "cs" else 1.0)
                vel.append(max(float(np.max(np.abs(u32 - u64))), float(np.max(np.abs(v32 - v64)))) / U)
                g32, g64, ln64 = _decay_rates(ser32, L.series())
                rate.append(abs(g32 / g64 - 1.0))
                lnd.append(ln64)
        t_plain += dt
        work += d["n"] ** 2 * steps
        per_model[d["model"]][0] += d["n"] ** 2 * steps
        per_model[d["model"]][1] += dt
    mlups_p = work / t_plain / 1e6
    return {
        "workload": "256 lattices, sides uniform in {32,64,128,256,512}, tau* U[0.51,2], half CS D2Q9 / half FD "
                    "16-velocity, shear-wave and Taylor-Green initial states (seed 0); FP32 CS in place",
        "cells": cells,
        "fp32_batched": {"mlups": round(mlups_b, 1), "steps": steps, "untimed_steps_before": warm,
                         "s": round(t_b, 4), "tuning": tune.strip()},
        "fp64_plain_one_at_a_time": {
            "mlups": round(mlups_p, 2), "steps_each": steps, "untimed_steps_before": warm,
            "cs_mlups": round(per_model["cs"][0] / max(per_model["cs"][1], 1e-12) / 1e6, 2),
            "fd_mlups": round(per_model["fd"][0] / max(per_model["fd"][1], 1e-12) / 1e6, 2)},
        "speedup": round(mlups_b / mlups_p, 1),
        "fp32_vs_fp64": _error_summary(
            vel, rate, lnd, f"every lattice of side <= {max_err_side} ({len(sample)} of 256) after {warm + steps} "
            "steps: max |u32 - u64| / U over nodes and components; decay rate of the projected amplitude "
            f"(recorded every {every} steps, log-linear fit over the last 75% of the run while the FP64 amplitude "
            "is above 1e-3 of its start), |g32/g64 - 1|"),
    }


def _lat_kwargs(pkg, d, prec):
    s = _instance_spec(pkg, d, prec)
    return dict(model="cs" if s.model == 0 else "fd", q=s.q_per_axis, nx=s.nx, ny=s.ny, tau=s.tau, dt=s.dt,
                precision=prec, storage="inplace" if (s.model == 0 and prec == "fp32") else "ab")


SERVED_SIDES = (64, 128, 256, 512, 1024, 2048, 4096)
SERVED_STEPS = (1000, 20000)


def lattice_rates(torch, sides, steps=8, prec="fp32"):
    """Single-lattice rates (lattice updates per second) of the served
    instance kinds, CS and FD 16-velocity, per side: a few steps of one
    lattice alone after one untimed step. FP32: CS in place, as served;
    FP64: the plain form (two-buffer CS), fewer steps for the large FD
    lattices, whose FP64 step takes up to 0.2 s."""
    import paper_1904_02471_gb300 as pkg
    rates = {}
    for model in ("cs", "fd"):
        for n in sides:
            d = {"model": model, "n": n, "tau_star": 0.8}
            s = _instance_spec(pkg, d, prec)
            with pkg.Lattice(model, s.q_per_axis, n, n, s.tau, dt=s.dt, precision=prec,
                             storage="inplace" if (model == "cs" and prec == "fp32") else "ab") as L:
                L.init(*_fields(d))
                L.step(1)
                L.sync()
                k = steps if model == "fd" and n > 512 else 64 * steps
                if prec == "fp64" and model == "fd":
                    k = 2 if n >= 2048 else (steps if n >= 256 else 8 * steps)
                t0 = time.perf_counter()
                L.step(k)
                L.sync()
                rates[(model, n)] = n * n * k / (time.perf_counter() - t0)
    return rates


def alone_seconds(reqs, rates):
    """Each run's time alone: side^2 x steps at its kind's single-lattice rate
    (lattice updates per second, keyed by (model, side))."""
    return [r["n"] ** 2 * r["steps"] / rates[(r["model"], r["n"])] for r in reqs]


def run_served(torch, n_req=48, load=1.0, seed=0, sides=SERVED_SIDES, steps=SERVED_STEPS, budget_gb=128,
               chunk=128, max_err_side=256, rates=None):
    """Served stream: Poisson arrivals of CS / FD 16-velocity Taylor-Green runs
    (FP32, sides log-uniform over powers of two, steps uniform) into the
    continuous-batching server; latency = completion - arrival. The arrival
    rate is `load` times an estimate of the capacity: the mean service time
    of the stream's requests, each lattice run alone at its measured rate (an
    underestimate of the server's capacity, which batches small lattices).
    Accuracy: every run of side <= max_err_side keeps its final fields and
    records its amplitude, and is compared with the same run in FP64."""
    import paper_1904_02471_gb300 as pkg
    from paper_1904_02471_gb300 import lbm
    if rates is None:
        rates = lattice_rates(torch, sides)
    probe = wl.served_stream(n_req, seed, rate_per_s=1.0, sides=sides, steps=steps)
    service = sum(alone_seconds(probe, rates)) / n_req
    rate = load / service
    reqs = wl.served_stream(n_req, seed, rate_per_s=rate, sides=sides, steps=steps)
    work = sum(r["n"] ** 2 * r["steps"] for r in reqs)
    sample = [i for i, r in enumerate(reqs) if r["n"] <= max_err_side]
    obs_every = {i: max(1, reqs[i]["steps"] // 32) for i in sample}
    S = lbm.Server(budget_gb << 30, 256, chunk)
    t0 = time.perf_counter()
    tickets = []
    for i, r in enumerate(reqs):
        delay = r["arrival"] - (time.perf_counter() - t0)
        if delay > 0:
            time.sleep(delay)
        spec = _instance_spec(pkg, {"model": r["model"], "n": r["n"], "tau_star": r["tau_star"]}, "fp32")
        U = U0 * (math.sqrt(3.0) if r["model"] == "cs" else 1.0)
        tickets.append(S.submit(lbm.make_request(spec, r["steps"], "tg", U, obs_every=obs_every.get(i, 0),
                                                 keep_moments=i in sample)))
    S.drain(7200)
    res = [S.poll(t) for t in tickets]
    kept = {i: (S.moments(tickets[i], reqs[i]["n"], reqs[i]["n"]), S.series(tickets[i])) for i in sample
            if res[i]["status"] == 0}
    for t in tickets:
        S.release(t)
    S.close()
    lat = sorted(x["t_done"] - x["t_submit"] for x in res)
    makespan = max(x["t_done"] for x in res) - min(x["t_submit"] for x in res)
    ok = sum(1 for x in res if x["status"] == 0)
    span = reqs[-1]["arrival"]
    # the same runs in FP64 (one batch, each with its own step budget)
    vel, rdec, lnd = [], [], []
    if kept:
        idx = sorted(kept)
        specs = [_instance_spec(pkg, {"model": reqs[i]["model"], "n": reqs[i]["n"],
                                      "tau_star": reqs[i]["tau_star"]}, "fp64") for i in idx]
        B = pkg.Batch(specs)
        for b, i in enumerate(idx):
            n = reqs[i]["n"]
            U = U0 * (math.sqrt(3.0) if reqs[i]["model"] == "cs" else 1.0)
            B.init(b, *wl.taylor_green(n, n, U))
            B.set_probe(b, *wl.probe_taylor_green(n, n))
            B.record(b, obs_every[i], reqs[i]["steps"] // obs_every[i] + 1)
            B.set_budget(b, reqs[i]["steps"])
        B.step(max(reqs[i]["steps"] for i in idx))
        B.sync()
        for b, i in enumerate(idx):
            (_, u32, v32), ser32 = kept[i]
            _, u64, v64 = B.moments(b)
            U = U0 * (math.sqrt(3.0) if reqs[i]["model"] == "cs" else 1.0)
            vel.append(max(float(np.max(np.abs(u32 - u64))), float(np.max(np.abs(v32 - v64)))) / U)
            g32, g64, ln64 = _decay_rates(ser32, B.series(b))
            rdec.append(abs(g32 / g64 - 1.0))
            lnd.append(ln64)
        B.close()
    p50, p99 = float(np.percentile(lat, 50)), float(np.percentile(lat, 99))
    # slowdown: latency over the run's time alone at its measured single-lattice rate
    alone = alone_seconds(reqs, rates)
    late = [x["t_done"] - x["t_submit"] for x in res]
    slow = sorted(l / a for l, a in zip(late, alone))
    worst = max(range(n_req), key=lambda i: late[i])
    out = {
        "workload": f"{n_req} Poisson arrivals (seed {seed}) over ~{span:.0f} s, CS D2Q9 (in place) or FD 16-velocity "
                    f"Taylor-Green, sides {sides[0]}..{sides[-1]} (powers of 2, log-uniform), steps "
                    f"U[{steps[0]},{steps[1]}], tau* U[0.51,2], FP32",
        "requests": n_req, "completed_ok": ok, "load": load, "rate_per_s": round(rate, 5),
        "mean_service_s_alone": round(service, 3), "chunk_steps": chunk,
        "aggregate_mlups": round(work / makespan / 1e6, 1),
        "latency_s": {"p50": round(p50, 4), "p99": round(p99, 4), "max": round(lat[-1], 4),
                      "p99_over_p50": round(p99 / p50, 2)},
        "slowdown": {"p50": round(float(np.percentile(slow, 50)), 2), "p99": round(float(np.percentile(slow, 99)), 2),
                     "max": round(slow[-1], 2), "how": "latency / the run's time alone at its single-lattice rate"},
        "longest_latency_run": {"model": reqs[worst]["model"], "side": reqs[worst]["n"],
                                "steps": reqs[worst]["steps"], "arrival_s": round(reqs[worst]["arrival"], 2),
                                "alone_s": round(alone[worst], 2), "latency_s": round(late[worst], 2)},
        "makespan_s": round(makespan, 3),
        "runs": {"columns": ["model", "side", "steps", "arrival_s", "latency_s"],
                 "rows": [[r["model"], r["n"], r["steps"], round(r["arrival"], 2), round(x["t_done"] - x["t_submit"], 3)]
                          for r, x in zip(reqs, res)]},
    }
    # the plain FP64 form on the same request list: each run alone, one after
    # another, at its measured single-lattice FP64 rate
    r64 = lattice_rates(torch, sides, prec="fp64")
    t64 = sum(alone_seconds(reqs, r64))
    out["fp64_one_at_a_time"] = {
        "mlups": round(work / t64 / 1e6, 2), "s": round(t64, 1),
        "how": "the same request list in FP64, each run alone and one after another: sum of side^2 x steps over "
               "the sum of each run's time at its measured single-lattice FP64 rate (CS two buffers, FD 16-velocity; "
               "a few timed steps per kind and side)",
        "single_lattice_mlups": {f"{m}{n}": round(v / 1e6, 2) for (m, n), v in r64.items()}}
    out["speedup_vs_fp64_one_at_a_time"] = round(out["aggregate_mlups"] / out["fp64_one_at_a_time"]["mlups"], 1)
    if vel:
        out["fp32_vs_fp64"] = _error_summary(
            vel, rdec, lnd, f"every run of side <= {max_err_side} ({len(vel)} of {n_req}), its kept final fields "
            "against the same run in FP64: max |u32 - u64| / U; decay rate of the projected amplitude (recorded "
            "every steps/32 steps, log-linear fit over the last 75% of the run while the FP64 amplitude is above "
            "1e-3 of its start), |g32/g64 - 1|")
    return out


def run_imex(torch, n=FD_N, tau=1e-5, steps=24, warm=3):
    """FD 16-velocity FP32 on an n^2 lattice in the stiff regime (tau = 1e-5
    FD units, below the Courant-limited step 0.4 dx / max|v|): SSP-RK3 at its
    largest admitted step dt = tau against IMEX-SSP2(2,2,2) at the Courant
    limit. Per-stage CUDA-event times; physical time advanced per second of
    device time is the figure that decides between them."""
    import paper_1904_02471_gb300 as pkg
    dt_cfl = FD_CFL * pkg.lbm_fd_max_dt(4, 1.0 / n, 1e300)
    out = {"lattice": [n, n], "velocities": 16, "tau_fd": tau, "precision": "fp32", "steps": steps}
    for scheme, dt in (("rk3", min(tau, dt_cfl)), ("imex", dt_cfl)):
        spec = pkg.make_spec("fd", 4, n, n, tau, dt, 0.0, "fp32", scheme=scheme)
        B = pkg.Batch([spec])
        B.init(0, *wl.taylor_green(n, n, U0))
        B.record(0, steps, 4)
        B.step_profiled(warm)
        ms, total = B.step_profiled(steps)
        ser = B.series(0)
        B.close()
        nst = 2 if scheme == "imex" else 3
        stage = [float(ms[0][k]) / steps for k in range(nst)]
        step_ms = sum(stage)
        bytes_lu = (6 if scheme == "imex" else 8) * 16 * 4
        out[scheme] = {"dt": dt, "dt_over_tau": round(dt / tau, 4), "stages": nst,
                       "stage_ms": [round(x, 4) for x in stage], "ms_per_step": round(step_ms, 4),
                       "mlups": round(n * n / (step_ms / 1e3) / 1e6, 1),
                       "gbs": round(n * n * bytes_lu / (step_ms / 1e3) / 1e9, 1), "bytes_per_lu": bytes_lu,
                       "physical_time_per_s": round(dt / (step_ms / 1e3), 6),
                       "finite": all(x["nonfinite"] == 0 for x in ser)}
    out["imex_over_rk3_physical_time_rate"] = round(out["imex"]["physical_time_per_s"] /
                                                    out["rk3"]["physical_time_per_s"], 3)
    return out


def run_fused(torch, n=FD_N, steps=20, warm=3):
    """FD 16-velocity FP32 on an n^2 Taylor-Green lattice (tau = 5e-4, dt =
    1e-5, the roofline configuration): the temporally blocked SSP-RK3 step
    (one launch per step, 2Q values of device memory per update) against the
    three stage launches (8Q values). CUDA-event times per launch. The fused
    kernel also evaluates stages 1 and 2 on the halo of every tile (6.5
    node-stages per updated node for 32 x 8 tiles against 3), so its
    arithmetic per update is 2.2x larger while its bytes are 4x smaller."""
    import paper_1904_02471_gb300 as pkg
    out = {"lattice": [n, n], "velocities": 16, "tau_fd": FD_TAU, "dt_fd": FD_DT, "precision": "fp32",
           "steps": steps}
    for scheme in ("rk3", "rk3_fused"):
        spec = pkg.make_spec("fd", 4, n, n, FD_TAU, FD_DT, 0.0, "fp32", scheme=scheme)
        B = pkg.Batch([spec])
        B.init(0, *wl.taylor_green(n, n, U0))
        tuning = B.tune(2)
        B.record(0, steps, 4)
        B.step_profiled(warm)
        ms, total = B.step_profiled(steps)
        ser = B.series(0)
        B.close()
        nst = 1 if scheme == "rk3_fused" else 3
        stage = [float(ms[0][k]) / steps for k in range(nst)]
        step_ms = sum(stage)
        bytes_lu = (2 if scheme == "rk3_fused" else 8) * 16 * 4
        out[scheme] = {"launches_per_step": nst, "launch_ms": [round(x, 4) for x in stage],
                       "ms_per_step": round(step_ms, 4), "mlups": round(n * n / (step_ms / 1e3) / 1e6, 1),
                       "gbs": round(n * n * bytes_lu / (step_ms / 1e3) / 1e9, 1), "bytes_per_lu": bytes_lu,
                       "frac_hbm": round(n * n * bytes_lu / (step_ms / 1e3) / 1e9 / peaks()[0], 4),
                       "tuning": tuning.strip(), "finite": all(x["nonfinite"] == 0 for x in ser)}
    out["fused_over_rk3"] = round(out["rk3_fused"]["mlups"] / out["rk3"]["mlups"], 3)
    return out


def run_served_full(torch, n_req, loads, seed=0, chunk=128):
    """The served stream at several loads (one record)."""
    sides = SERVED_SIDES
    rates = lattice_rates(torch, sides)
    out = {"metric": "served stream, full configuration", "unit": "MLUPS", "dtype": "f32",
           "data": "synthetic (Taylor-Green initial states, seeded arrivals)",
           "single_lattice_mlups": {f"{m}{n}": round(v / 1e6, 1) for (m, n), v in rates.items()}, "runs": []}
    for load in loads:
        out["runs"].append(run_served(torch, n_req=n_req, load=load, seed=seed, rates=rates, chunk=chunk))
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
    """The FP64 C oracle on the host cores (the paper publishes no
    implementation or timings). Each timed step is one bounded sample per
    process: CS D2Q9 512^2 and FD 16-velocity 128^2 for a share of the CPU
    budget each, one independent single-thread process per host core, all at
    once. `value` combines the measured per-node-update rates of the two
    models in the proportions of the roofline workload (8192^2 CS nodes and
    4096^2 FD nodes per step); `ms_per_step` is the wall time of one sample
    step of this run."""
    if rank != 0:
        return None
    import oracle  # noqa: F401
    ncores = host_cores()
    vals, walls = [], []
    rates = None
    with oracle_pool(ncores) as pool:
        for s in range(args.warmup + args.steps):
            w0 = time.perf_counter()
            rs = oracle_rates_all_cores(pool, ncores, args.cpu_budget / max(1, args.steps))
            w = time.perf_counter() - w0
            if s >= args.warmup:
                vals.append(sum(cpu_value(r) for r in rs))
                walls.append(w)
            rates = rs[0]
    val = statistics.median(vals)
    sample = (f"per step and process: {rates['cs_sample']}; {rates['fd_sample']}; FP64 C oracle, one independent "
              f"single-thread process per host core ({ncores}) at once, rates summed")
    return {
        "impl": "reference", "metric": METRIC, "value": round(val, 4), "unit": "MLUPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(statistics.median(walls) * 1e3, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (Taylor-Green initial state)",
        "config": {"workload": WORKLOAD, "reference": "plain FP64 C oracle (no published implementation)",
                   "ran": sample,
                   "value_is": "the measured CS and FD per-node-update rates of the samples, combined in the "
                               "workload's proportions (8192^2 CS + 4096^2 FD nodes per step): extrapolated per "
                               "node update, not a run of the full lattices",
                   "ms_per_step_is": "wall time of one timed sample step of this run"},
        "cpu_baseline": {"value": round(val, 4), "unit": "MLUPS", "cores": ncores, "kind": "oracle", "sample": sample},
        "e2e": {"value": round(val, 4), "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def run_profile_case(a):
    """One small single lattice for kernel profiling (e.g. under Nsight
    Compute): a Taylor-Green lattice in FP32 deviation storage whose state is
    larger than the 129 MB L2 (CS 2048^2: 302 MB; FD 16-velocity 1024^2:
    201 MB) but small enough that a multi-pass capture ends in seconds. The
    kernel variant can be pinned with --tile, the grid with --grid (0: one
    block per tile)."""
    import torch
    import paper_1904_02471_gb300 as pkg
    torch.cuda.init()
    if a.profile_case == "cs":
        n = a.n or 2048
        L = pkg.Lattice("cs", 3, n, n, 0.8 / math.sqrt(3), precision=a.precision, storage=a.storage)
        if a.tile >= 0:
            L.config(a.tile, a.grid)
        L.init(*wl.taylor_green(n, n, 0.01 * math.sqrt(3)))
        L.step(a.case_steps or 4)
    else:
        n = a.n or 1024
        # IMEX: dt = 5 tau (a step the RK3 scheme refuses)
        tau = 2e-6 if a.scheme == "imex" else 5e-4
        L = pkg.Lattice("fd", a.q, n, n, tau, dt=1e-5, precision=a.precision, scheme=a.scheme)
        if a.tile >= 0:
            L.config(a.tile, a.grid)
        L.init(*wl.taylor_green(n, n, 0.01))
        L.step(a.case_steps or 2)
    L.sync()
    print(a.profile_case, n, "mass", L.observables()["mass"])
    L.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-budget", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the batched and served sections")
    ap.add_argument("--served-requests", type=int, default=48, help="requests of the served stream")
    ap.add_argument("--served-load", type=float, nargs="+", default=[1.0],
                    help="arrival rate as a multiple of the estimated capacity (the line uses the first)")
    ap.add_argument("--served-chunk", type=int, default=128, help="the server's chunk_steps")
    ap.add_argument("--served-full", type=int, default=0, metavar="N_REQ",
                    help="only run the served stream with N_REQ requests at each --served-load and print that "
                         "record")
    ap.add_argument("--profile-case", choices=["cs", "fd"], default=None,
                    help="only run one small lattice for kernel profiling (see run_profile_case)")
    ap.add_argument("--n", type=int, default=0, help="--profile-case: lattice side")
    ap.add_argument("--case-steps", type=int, default=0, help="--profile-case: steps")
    ap.add_argument("--tile", type=int, default=-1, help="--profile-case: kernel tile variant")
    ap.add_argument("--grid", type=int, default=0, help="--profile-case: grid (0: one block per tile)")
    ap.add_argument("--q", type=int, default=4, help="--profile-case fd: nodes per axis")
    ap.add_argument("--precision", default="fp32", help="--profile-case: fp32 or fp64")
    ap.add_argument("--storage", default="ab", choices=["ab", "inplace"], help="--profile-case cs: storage")
    ap.add_argument("--scheme", default="rk3", choices=["rk3", "imex", "rk3_fused"],
                    help="--profile-case fd: time scheme")
    args = ap.parse_args()
    if args.profile_case:
        run_profile_case(args)
        return
    if args.served_full:
        import torch
        torch.cuda.init()
        print(json.dumps(run_served_full(torch, args.served_full, args.served_load, chunk=args.served_chunk)))
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
