"""FD lattices with the temporally blocked SSP-RK3 step (LBM_TS_RK3_FUSED).

The three stages of Sec. 2 run in one launch per tile: stage 1 on the tile
plus 6 nodes, stage 2 on the tile plus 3, stage 3 on the tile, with f^(1) and
f^(2) in shared memory, so a step reads and writes each population once
(2Q values per update against 8Q for the three stage launches). The scheme is
the same: FP64 storage must match the oracle's RK3 step to 1e-12 relative in
every population (after 1000 steps on a lattice with interior tiles, staged
without wrap), FP32 deviation storage must agree with the three-launch FP32
kernels to rounding. The state alternates between two buffers, so readout,
checkpoints and observables are checked after odd and even step counts.
"""
import math

import numpy as np
import pytest

import lbm_workloads as wl
import oracle
import paper_1904_02471_gb300 as pkg
from paper_1904_02471_gb300 import lbm

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
VMAX = {3: math.sqrt(3.0), 4: 2.3344142183389773, 5: 2.8569700138728056}


@pytest.fixture(scope="module", autouse=True)
def gpu():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1904_02471_gb300 import build
    build.build()
    torch.cuda.init()


def rel_err(a, b):
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-300)))


def _rough_state(q, nx, ny, seed):
    rho, ux, uy = wl.random_smooth(nx, ny, seed=seed, amp_rho=0.05, amp_u=0.05)
    f0 = oracle.equilibrium(q, rho, ux, uy)
    return f0 * (1 + wl.random_uniform(f0.shape, seed=seed + 1, lo=-0.01, hi=0.01))


def _dt_tau(q, nx, cfl=0.4, ratio=1.0):
    dx = 1.0 / nx
    dt = cfl * dx / VMAX[q]
    return dx, dt, dt * ratio


@pytest.mark.parametrize("q,nx,ny,steps", [
    (4, 76, 33, 1000),   # interior 32 x 8 tiles (halo of 9 inside the lattice), 1000 steps
    (3, 20, 18, 201), (4, 33, 9, 150), (5, 20, 18, 61),
    (5, 96, 40, 40),     # FP64 25-velocity set: 32 x 4 tiles, interior ones too
    (4, 70, 37, 51),     # ragged tiles; rows of an even length (FP64 16-byte chunks from wrapped columns)
    (4, 1, 1, 31), (4, 2, 5, 30), (5, 3, 1, 21), (3, 7, 6, 40),
])
def test_fused_fp64_matches_oracle(q, nx, ny, steps):
    """Every population equals the oracle's SSP-RK3 steps to 1e-12 (rough
    state: the nonlinear WENO weights matter); ragged, degenerate and
    self-overlapping halos (lattices smaller than the 9-node halo)."""
    f0 = _rough_state(q, nx, ny, 300 + q + nx)
    dx, dt, tau = _dt_tau(q, nx, ratio=1.5)
    with pkg.Lattice("fd", q, nx, ny, tau, dt=dt, scheme="rk3_fused") as L:
        L.set_populations(f0)
        L.step(steps)
        f = L.populations()
        assert L.steps_done == steps
    ref = oracle.fd_run(f0, dx, dt, tau, steps)
    assert np.all(np.isfinite(ref))
    assert rel_err(f, ref) < TOL64


def test_fused_fp64_equals_three_launch_rk3_and_records_observables():
    """Taylor-Green with a probe: the fused step and the three stage launches
    give the same populations (to rounding), and the observables recorded
    during fused steps equal the oracle's sums on the oracle's states."""
    n, q = 40, 4
    rho, ux, uy = wl.taylor_green(n, n, 0.01)
    comp, px, py, norm = wl.probe_taylor_green(n, n)
    dx, dt, tau = _dt_tau(q, n)
    out = {}
    for scheme in ("rk3", "rk3_fused"):
        with pkg.Lattice("fd", q, n, n, tau, dt=dt, scheme=scheme) as L:
            L.init(rho, ux, uy)
            L.set_probe(comp, px, py, norm)
            L.record(7, 100)
            L.step(43)
            out[scheme] = (L.populations(), L.series(), L.observables())
    assert rel_err(out["rk3_fused"][0], out["rk3"][0]) < 1e-13
    g = oracle.equilibrium(q, rho, ux, uy)
    ser = out["rk3_fused"][1]
    assert [s["step"] for s in ser] == list(range(0, 43, 7))
    for s in ser:
        ob = oracle.observables(g, comp, px, py, norm)
        assert abs(s["mass"] - ob[0]) < TOL64 * ob[0]
        assert abs(s["amp"] - ob[3]) < 1e-10 * abs(ob[3])
        g = oracle.fd_run(g, dx, dt, tau, 7)
    assert abs(out["rk3_fused"][2]["amp"] - out["rk3"][2]["amp"]) < 1e-12 * abs(out["rk3"][2]["amp"])


@pytest.mark.parametrize("q", [3, 4, 5])
def test_fused_fp32_agrees_with_three_launch_fp32(q):
    """FP32 deviation storage: the fused step and the three stage launches
    compute the same formulas per node and stage; they differ only in the
    order of a few float sums, so after 200 steps of a Taylor-Green flow the
    populations agree to a few float roundings and the velocity to 1e-6 of U."""
    n, U = 96, 0.01
    rho, ux, uy = wl.taylor_green(n, n, U)
    dx, dt, tau = _dt_tau(q, n, cfl=0.3)
    res = {}
    for scheme in ("rk3", "rk3_fused"):
        with pkg.Lattice("fd", q, n, n, tau, dt=dt, precision="fp32", scheme=scheme) as L:
            L.init(rho, ux, uy)
            L.step(200)
            res[scheme] = (L.populations(), L.moments())
    f32, f3 = res["rk3_fused"][0], res["rk3"][0]
    assert np.all(np.isfinite(f32))
    assert rel_err(f32, f3) < 1e-6
    for c in (1, 2):
        assert np.max(np.abs(res["rk3_fused"][1][c] - res["rk3"][1][c])) < 1e-6 * U


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_fused_tile_variants_and_grids_agree(prec):
    """32 x 16, 32 x 8 and 32 x 4 output tiles and a persistent grid compute
    every node from the same inputs in the same order: bit-identical
    populations. 32 x 2 has no fused kernel, and 32 x 16 needs more shared
    memory than the device has for FP64 with 16 velocities: both refused."""
    q, nx, ny = 4, 70, 37
    f0 = _rough_state(q, nx, ny, 330)
    dx, dt, tau = _dt_tau(q, nx)
    res = []
    for tile in range(lbm.lbm_n_tiles("fd")):
        for grid in (0, 3):
            with pkg.Lattice("fd", q, nx, ny, tau, dt=dt, precision=prec, scheme="rk3_fused") as L:
                try:
                    L.config(tile, grid)
                except lbm.LbmError as e:
                    assert e.code == lbm.LBM_EINVAL and (tile == 3 or (tile == 2 and prec == "fp64"))
                    continue
                L.set_populations(f0)
                L.step(9)
                res.append(((tile, grid), L.populations()))
    assert len(res) == (6 if prec == "fp32" else 4)
    for cfg, f in res[1:]:
        assert np.array_equal(f, res[0][1]), cfg
    if prec == "fp64":
        assert rel_err(res[0][1], oracle.fd_run(f0, dx, dt, tau, 9)) < TOL64


def test_fused_checkpoint_after_odd_steps_and_batch_equals_alone():
    """The state alternates between two buffers: a checkpoint taken after an
    odd number of steps and loaded into a fresh lattice continues exactly;
    fused, RK3 and IMEX lattices of one velocity set form three groups of a
    batch (graph-replayed chunks), and every lattice computes there what it
    computes alone."""
    q, n = 4, 48
    rho, ux, uy = wl.taylor_green(n, n, 0.01)
    dx, dt, tau = _dt_tau(q, n, cfl=0.3)
    with pkg.Lattice("fd", q, n, n, tau, dt=dt, precision="fp32", scheme="rk3_fused") as L:
        L.init(rho, ux, uy)
        L.step(37)
        ck = L.save()
        L.step(40)
        cont = L.populations()
    with pkg.Lattice("fd", q, n, n, tau, dt=dt, precision="fp32", scheme="rk3_fused") as L:
        L.load(ck)
        assert L.steps_done == 37
        L.step(40)
        assert np.array_equal(L.populations(), cont)

    specs, inits = [], []
    for i, (m, scheme, ratio) in enumerate([(40, "rk3_fused", 1.0), (56, "rk3", 1.0), (33, "rk3_fused", 2.0),
                                            (64, "imex", 4.0), (100, "rk3_fused", 1.0)]):
        d = 0.3 / (m * VMAX[q])
        tau_i = d * ratio if scheme != "imex" else d / ratio
        specs.append(pkg.make_spec("fd", q, m, m, tau_i, d, 0.0, "fp32", scheme=scheme))
        inits.append(wl.taylor_green(m, m, 0.01))
    B = pkg.Batch(specs)
    for i in range(len(specs)):
        B.init(i, *inits[i])
    assert len(B.groups()) == 3
    B.step(71)
    got = [B.populations(i) for i in range(len(specs))]
    B.close()
    for i, s in enumerate(specs):
        with pkg.Lattice("fd", q, s.nx, s.ny, s.tau, dt=s.dt, precision="fp32", scheme=s.scheme) as L:
            L.init(*inits[i])
            L.step(71)
            assert np.array_equal(L.populations(), got[i]), i


def test_fused_fp32_decay_rate_against_fp64():
    """Taylor-Green decay on 128^2 (the paper's nu_FD = 5e-4 at dt = tau):
    FP32 deviation storage against FP64, both fused, decay rate within 1e-4
    and velocity within 1e-4 of U."""
    n, q, U = 128, 4, 0.01
    tau = dt = 5e-4
    rho, ux, uy = wl.taylor_green(n, n, U)
    comp, px, py, norm = wl.probe_taylor_green(n, n)
    out = {}
    for prec in ("fp64", "fp32"):
        with pkg.Lattice("fd", q, n, n, tau, dt=dt, precision=prec, scheme="rk3_fused") as L:
            L.init(rho, ux, uy)
            L.set_probe(comp, px, py, norm)
            L.record(20, 200)
            L.step(2000)
            out[prec] = (L.series(), L.moments())
    g = {}
    for prec, (ser, _) in out.items():
        t = np.array([s["time"] for s in ser])
        a = np.array([s["amp"] for s in ser])
        g[prec] = oracle.fit_decay(t, a, 0.25)[0]
    assert g["fp64"] > 0 and abs(g["fp32"] / g["fp64"] - 1) < 1e-4, g
    assert np.max(np.abs(out["fp32"][1][1] - out["fp64"][1][1])) < 1e-4 * U
