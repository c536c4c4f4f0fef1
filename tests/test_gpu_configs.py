"""The named workloads as parity cases (GPU).

* CS D2Q9 shear wave, 64x4, tau* = 0.8, 2000 steps, FP64: every population
  against the oracle, and the decay against exp(-nu k^2 t), nu = (tau*-1/2)/3.
* FD Taylor-Green, 16 velocities, 256^2, nu_FD = tau_FD = 5e-4, dt = 5e-4,
  5000 steps, FP64 and FP32 deviation storage: the oracle checks sampled
  windows of the FP64 state at the end (one step, exact interior); FP32
  against FP64 by decay rate (1e-4) and velocity; the decay against Eq.
  (taylor); and the CS run with the same physical viscosity through Eq.
  (nu-transfer), tau_LU = N tau_FD + sqrt(3)/6, reaches the same nu_app.
* Shock tube 2048x4 (rho_L = 1.5, rho_R = 0.75, tau* = 0.6): CS FP32 for
  1500 steps against the FP64 oracle's density profile; FD 25 velocities in
  FP64 against the oracle for 100 steps, and FP32 against FP64 at 1500 steps.
"""
import math

import numpy as np
import pytest

import lbm_workloads as wl
import oracle
import paper_1904_02471_gb300 as pkg

pytestmark = pytest.mark.gpu

SQ3 = math.sqrt(3.0)


@pytest.fixture(scope="module", autouse=True)
def gpu():
    import torch
    assert torch.cuda.is_available()
    from paper_1904_02471_gb300 import build
    build.build()
    torch.cuda.init()


def rel_err(a, b):
    return float(np.max(np.abs(a - b) / np.abs(b)))


def test_cs_shear_64x4_2000_steps_fp64():
    c = wl.CS_SHEAR_64x4
    nx, ny = c["nx"], c["ny"]
    rho, ux, uy = wl.shear_wave(nx, ny, c["U"])
    comp, px, py, norm = wl.probe_shear(nx, ny)
    with pkg.Lattice("cs", 3, nx, ny, c["tau"]) as L:
        L.init(rho, ux, uy)
        L.set_probe(comp, px, py, norm)
        L.record(100, 100)
        L.step(c["steps"])
        f = L.populations()
        ser = L.series()
        last = L.observables()
    ref = oracle.cs_run(oracle.equilibrium(3, rho, ux, uy), c["tau"], c["steps"])
    assert rel_err(f, ref) < 1e-12
    t = np.array([s["step"] for s in ser] + [last["step"]], float)
    a = np.array([s["amp"] for s in ser] + [last["amp"]])
    gamma, _ = oracle.fit_decay(t, a, 200)
    k = 2 * math.pi / nx
    nu_star = (0.8 - 0.5) / 3
    assert abs(gamma / k ** 2 / nu_star - 1) < 2e-3
    assert abs(a[-1] / a[0] - math.exp(-nu_star * k * k * c["steps"])) < 2e-3


def _tg_run(prec, steps=5000, every=100):
    c = wl.FD_TG_256
    n = c["nx"]
    comp, px, py, norm = wl.probe_taylor_green(n, n)
    L = pkg.Lattice("fd", 4, n, n, c["tau"], dt=c["dt"], precision=prec)
    L.init(*wl.taylor_green(n, n, c["U"]))
    L.set_probe(comp, px, py, norm)
    L.record(every, steps // every + 1)
    L.step(steps)
    return L, L.series()


def test_fd_taylor_green_256_5000_steps():
    c = wl.FD_TG_256
    n, tau, dt = c["nx"], c["tau"], c["dt"]
    L64, s64 = _tg_run("fp64")
    L32, s32 = _tg_run("fp32")
    # oracle: one step from the final FP64 state on sampled windows
    wins = [(0, 0), (250, 3), (128, 200)]
    before = [L64.populations_region(x0, y0, 24, 24) for x0, y0 in wins]
    L64.step(1)
    after = [L64.populations_region(x0, y0, 24, 24) for x0, y0 in wins]
    for f0, f1 in zip(before, after):
        ref = oracle.fd_run(f0, 1.0 / n, dt, tau, 1)
        assert rel_err(f1[:, 9:15, 9:15], ref[:, 9:15, 9:15]) < 1e-12
    # decay: FP32 against FP64, and FP64 against Eq. (taylor) with nu = tau_FD
    t = np.array([s["time"] for s in s64])
    g64 = oracle.fit_decay(t, np.array([s["amp"] for s in s64]), 0.25)[0]
    g32 = oracle.fit_decay(np.array([s["time"] for s in s32]), np.array([s["amp"] for s in s32]), 0.25)[0]
    assert abs(g32 / g64 - 1) < 1e-4, g32 / g64 - 1
    k = 2 * math.pi
    nu64 = g64 / (2 * k * k)
    assert abs(nu64 / tau - 1) < 1e-2, nu64 / tau - 1
    _, u64, _ = L64.moments()
    L32.step(1)
    _, u32, _ = L32.moments()
    assert np.max(np.abs(u32 - u64)) / c["U"] < 1e-4
    # the CS run with the same physical viscosity (Eq. nu-transfer) and the
    # same physical time (one CS step is dt_LU / N in FD time units)
    tau_lu = pkg.lbm_tau_lu_from_fd(n, tau)
    cs_steps = int(round(5000 * dt * n * SQ3))
    comp, px, py, norm = wl.probe_taylor_green(n, n)
    with pkg.Lattice("cs", 3, n, n, tau_lu) as C:
        C.init(*wl.taylor_green(n, n, c["U"]))  # paper units: cs = 1 in both models
        C.set_probe(comp, px, py, norm)
        C.record(50, cs_steps // 50 + 1)
        C.step(cs_steps)
        sc = C.series()
    t_fd = np.array([s["step"] for s in sc]) * (1 / SQ3) / n
    gcs = oracle.fit_decay(t_fd, np.array([s["amp"] for s in sc]), 0.25)[0]
    nu_cs_fd = gcs / (2 * k * k)
    assert abs(nu_cs_fd / tau - 1) < 1e-2, nu_cs_fd / tau - 1
    L64.close()
    L32.close()


def test_shock_tube_cs_fp32_against_fp64_oracle():
    nx, ny = 2048, 4
    rho, ux, uy = wl.shock_tube(nx, ny, 1.5, 0.75, 1024)
    tau = 0.6 / SQ3
    with pkg.Lattice("cs", 3, nx, ny, tau, precision="fp32") as L:
        L.init(rho, ux, uy)
        L.step(1500)
        r, u, _ = L.moments()
    f = oracle.cs_run(oracle.equilibrium(3, rho, ux, uy), tau, 1500)
    r_ref, u_ref, _ = oracle.macro(3, f)
    # Bound: stored deviations reach |g| <= 0.25 (rho from 0.75 to 1.5 about
    # rho0 = 1), float32 ulp 3e-8; a step rounds each of the 9 values about 4
    # times at half an ulp, and the update is non-expansive (|1 - omega| < 1),
    # so after n steps |d rho| <= n * 9 * 4 * 0.5 * 3e-8 = 8.1e-4 at n = 1500.
    bound = 1500 * 9 * 4 * 0.5 * 3e-8
    assert np.max(np.abs(r - r_ref)) < bound, np.max(np.abs(r - r_ref))
    assert np.max(np.abs(u - u_ref)) < bound, np.max(np.abs(u - u_ref))


def test_shock_tube_fd_q5():
    nx, ny = 2048, 4
    rho, ux, uy = wl.shock_tube(nx, ny, 1.5, 0.75, 1024)
    tau = pkg.lbm_tau_fd_from_lu(nx, 0.6 / SQ3)
    dt = pkg.lbm_fd_max_dt(5, 1.0 / nx, tau)
    with pkg.Lattice("fd", 5, nx, ny, tau, dt=dt) as L64:
        L64.init(rho, ux, uy)
        L64.step(100)
        f = L64.populations()
        ref = oracle.fd_run(oracle.equilibrium(5, rho, ux, uy), 1.0 / nx, dt, tau, 100)
        assert rel_err(f, ref) < 1e-12
        L64.step(1400)
        r64, u64, _ = L64.moments()
    with pkg.Lattice("fd", 5, nx, ny, tau, dt=dt, precision="fp32") as L32:
        L32.init(rho, ux, uy)
        L32.step(1500)
        r32, u32, _ = L32.moments()
    # same bound as the CS shock (one rounding per stored value and stage in
    # increment form, 25 values, 3 stages)
    bound = 1500 * 25 * 3 * 0.5 * 3e-8
    assert np.max(np.abs(r32 - r64)) < bound, np.max(np.abs(r32 - r64))
    assert np.max(np.abs(u32 - u64)) < bound, np.max(np.abs(u32 - u64))
