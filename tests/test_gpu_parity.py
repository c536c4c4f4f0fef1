"""GPU parity: the CUDA library (through the C ABI) against the FP64 oracle.

FP64 storage must match the oracle to 1e-12 relative in every population
after up to 1000 steps (the two differ only in rounding order: FMA, the
division-light WENO weight normalisation, reciprocal-times-multiply).
FP32 deviation storage is judged on velocity and decay rate: max relative
velocity error and relative decay-rate error against the FP64 oracle.
Lattice sizes span several tiles with ragged tails (CS tiles 128x2 / 256x1,
FD tiles 32x8).
"""
import math

import numpy as np
import pytest

import lbm_workloads as wl
import oracle
import paper_1904_02471_gb300 as pkg

pytestmark = pytest.mark.gpu

SQ3 = math.sqrt(3.0)
TOL64 = 1e-12


@pytest.fixture(scope="module", autouse=True)
def gpu():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1904_02471_gb300 import build
    build.build()
    torch.cuda.init()


def rel_err(a, b):
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-300)))


# ---------------------------------------------------------------- CS, FP64
def test_cs_fp64_shear_64x4_1000_steps():
    c = wl.CS_SHEAR_64x4
    rho, ux, uy = wl.shear_wave(c["nx"], c["ny"], c["U"])
    with pkg.Lattice("cs", 3, c["nx"], c["ny"], c["tau"]) as L:
        L.init(rho, ux, uy)
        f0 = L.populations()
        # same f^eq up to the factorisation w(rho + rho(...)) vs w rho (1 + ...)
        assert rel_err(f0, oracle.equilibrium(3, rho, ux, uy)) < 1e-14
        L.step(1000)
        f = L.populations()
    ref = oracle.cs_run(oracle.equilibrium(3, rho, ux, uy), c["tau"], 1000)
    assert rel_err(f, ref) < TOL64


@pytest.mark.parametrize("nx,ny", [(300, 7), (129, 5), (1, 1), (1, 6), (7, 1), (2, 3)])
def test_cs_fp64_random_state_ragged(nx, ny):
    rho, ux, uy = wl.random_smooth(nx, ny, seed=nx * 31 + ny, amp_rho=0.1, amp_u=0.1)
    f0 = oracle.equilibrium(3, rho, ux, uy)
    f0 = f0 * (1 + wl.random_uniform(f0.shape, seed=7, lo=-0.05, hi=0.05))
    tau = 0.41
    with pkg.Lattice("cs", 3, nx, ny, tau) as L:
        L.set_populations(f0)
        assert rel_err(L.populations(), f0) == 0.0
        L.step(200)
        f = L.populations()
    assert rel_err(f, oracle.cs_run(f0, tau, 200)) < TOL64


def test_cs_fp64_moments_and_observables():
    nx, ny = 150, 9
    rho, ux, uy = wl.taylor_green(nx, ny, 0.02 * SQ3)
    comp, px, py, norm = wl.probe_taylor_green(nx, ny)
    with pkg.Lattice("cs", 3, nx, ny, 0.5) as L:
        L.init(rho, ux, uy)
        L.set_probe(comp, px, py, norm)
        L.step(100)
        r, u, v = L.moments()
        o = L.observables()
    f = oracle.cs_run(oracle.equilibrium(3, rho, ux, uy), 0.5, 100)
    r2, u2, v2 = oracle.macro(3, f)
    assert rel_err(r, r2) < TOL64
    assert np.max(np.abs(u - u2)) < TOL64 * 0.02 and np.max(np.abs(v - v2)) < TOL64 * 0.02
    ob = oracle.observables(f, comp, px, py, norm)
    assert o["step"] == 100
    assert abs(o["mass"] - ob[0]) < TOL64 * ob[0]
    assert abs(o["mom_x"] - ob[1]) < TOL64 * ob[0] and abs(o["mom_y"] - ob[2]) < TOL64 * ob[0]
    assert abs(o["amp"] - ob[3]) < TOL64 * abs(ob[3])


# ---------------------------------------------------------------- FD, FP64
def test_fd_fp64_taylor_green_q4_1000_steps():
    n = (40, 36)
    rho, ux, uy = wl.taylor_green(n[0], n[1], 0.01)
    dx, dt, tau = 1.0 / n[0], 1e-3, 2e-3
    with pkg.Lattice("fd", 4, n[0], n[1], tau, dt=dt) as L:
        L.init(rho, ux, uy)
        L.step(1000)
        f = L.populations()
    ref = oracle.fd_run(oracle.equilibrium(4, rho, ux, uy), dx, dt, tau, 1000)
    assert rel_err(f, ref) < TOL64


def _fd_interior_tiles(nx, ny, tx=32, ty=8):
    """Tiles whose staged halo (4 columns, 3 rows) needs no periodic wrap:
    the kernel stages those along its interior path."""
    return [(x0, y0) for x0 in range(0, nx, tx) for y0 in range(0, ny, ty)
            if x0 >= 4 and x0 + tx + 4 <= nx and y0 >= 3 and y0 + ty + 3 <= ny]


@pytest.mark.parametrize("q", [4, 5])
def test_fd_fp64_interior_tiles_1000_steps(q):
    """1000 FD steps on a lattice with interior 32 x 8 tiles (staged without
    wrap) and edge tiles, from a rough state, against the oracle at 1e-12 in
    every population. The oracle runs in a thread beside the GPU run (ctypes
    releases the interpreter lock)."""
    import concurrent.futures as cf
    nx, ny = 72, 44
    assert len(_fd_interior_tiles(nx, ny)) == 4
    rho, ux, uy = wl.random_smooth(nx, ny, seed=50 + q, amp_rho=0.05, amp_u=0.05)
    f0 = oracle.equilibrium(q, rho, ux, uy)
    f0 = f0 * (1 + wl.random_uniform(f0.shape, seed=11 + q, lo=-0.01, hi=0.01))
    dx = 1.0 / nx
    vmax = {4: 2.3344142183389773, 5: 2.8569700138728056}[q]
    dt = 0.4 * dx / vmax
    tau = 1.5 * dt
    with cf.ThreadPoolExecutor(1) as ex:
        fut = ex.submit(oracle.fd_run, f0, dx, dt, tau, 1000)
        with pkg.Lattice("fd", q, nx, ny, tau, dt=dt) as L:
            L.config(0, 0)   # 32 x 8 tiles, one block per tile
            L.set_populations(f0)
            L.step(1000)
            f = L.populations()
        ref = fut.result()
    assert np.all(np.isfinite(ref))
    assert rel_err(f, ref) < TOL64


def test_create_from_viscosity_equals_create_from_tau():
    """lbm_create_nu (Sec. 3): a CS lattice made from nu_FD with N = nx has
    the tau_LU of Eq. (nu-transfer) (to rounding: tau = N nu + dt/2 and
    N tau + sqrt(3)/6 may differ in the last bit), an FD lattice made from
    nu_LU = N nu_FD has tau_FD = nu_FD, and each computes bit-identically
    what the lattice made from its resolved spec computes."""
    n = 40
    nu_fd = 5e-4
    rho, ux, uy = wl.shear_wave(n, 4, 0.01 * SQ3)
    with pkg.Lattice("cs", 3, n, 4, None, nu=nu_fd, nu_model="fd") as A:
        assert abs(A.spec.tau - pkg.lbm_tau_lu_from_fd(n, nu_fd)) < 1e-15
        B = pkg.Lattice("cs", 3, n, 4, A.spec.tau)
        for L in (A, B):
            L.init(rho, ux, uy)
            L.step(25)
        assert np.array_equal(A.populations(), B.populations())
        B.close()
    rho, ux, uy = wl.shear_wave(n, n, 0.01)
    with pkg.Lattice("fd", 4, n, n, None, dt=nu_fd, nu=nu_fd * n, nu_model="cs") as A, \
            pkg.Lattice("fd", 4, n, n, nu_fd, dt=nu_fd) as B:
        assert abs(A.spec.tau - nu_fd) < 1e-18
        for L in (A, B):
            L.init(rho, ux, uy)
            L.step(5)
        assert np.array_equal(A.populations(), B.populations())


@pytest.mark.parametrize("q,nx,ny", [(3, 20, 18), (5, 20, 18), (4, 33, 9), (4, 1, 1), (4, 2, 5), (5, 3, 1)])
def test_fd_fp64_random_state(q, nx, ny):
    rho, ux, uy = wl.random_smooth(nx, ny, seed=q * 100 + nx, amp_rho=0.1, amp_u=0.1)
    f0 = oracle.equilibrium(q, rho, ux, uy)
    f0 = f0 * (1 + wl.random_uniform(f0.shape, seed=9, lo=-0.02, hi=0.02))
    dx = 1.0 / nx
    vmax = {3: SQ3, 4: 2.3344142183389773, 5: 2.8569700138728056}[q]
    dt = 0.4 * dx / vmax
    tau = 2 * dt
    with pkg.Lattice("fd", q, nx, ny, tau, dt=dt) as L:
        L.set_populations(f0)
        L.step(300)
        f = L.populations()
    assert rel_err(f, oracle.fd_run(f0, dx, dt, tau, 300)) < TOL64


def test_fd_fp64_shock_q5():
    """Quasi-1D shock (rho_L = 1.5, rho_R = 0.75, 25 velocities) where the
    nonlinear WENO weights are active; tau from tau* = 0.6 via Eq. (nu-transfer)."""
    nx, ny = 256, 4
    rho, ux, uy = wl.shock_tube(nx, ny, 1.5, 0.75, nx // 2)
    tau = pkg.lbm_tau_fd_from_lu(nx, 0.6 / SQ3)
    dt = pkg.lbm_fd_max_dt(5, 1.0 / nx, tau)
    with pkg.Lattice("fd", 5, nx, ny, tau, dt=dt) as L:
        L.init(rho, ux, uy)
        L.step(400)
        f = L.populations()
    ref = oracle.fd_run(oracle.equilibrium(5, rho, ux, uy), 1.0 / nx, dt, tau, 400)
    assert rel_err(f, ref) < TOL64


def test_fd_weno_eps_is_used():
    nx, ny = 24, 8
    rho, ux, uy = wl.shock_tube(nx, ny, 1.2, 0.8, nx // 2)
    f0 = oracle.equilibrium(4, rho, ux, uy)
    dt, tau = 2e-3, 4e-3
    for eps in (1e-6, 1e-2):
        with pkg.Lattice("fd", 4, nx, ny, tau, dt=dt) as L:
            L.set_weno_eps(eps)
            L.set_populations(f0)
            L.step(30)
            assert rel_err(L.populations(), oracle.fd_run(f0, 1 / nx, dt, tau, 30, eps=eps)) < TOL64


def test_fd_fp64_observables_series():
    n = 32
    rho, ux, uy = wl.taylor_green(n, n, 0.01)
    comp, px, py, norm = wl.probe_taylor_green(n, n)
    dt, tau = 2e-3, 4e-3
    with pkg.Lattice("fd", 4, n, n, tau, dt=dt) as L:
        L.init(rho, ux, uy)
        L.set_probe(comp, px, py, norm)
        L.record(10, 100)
        L.step(55)
        ser = L.series()
    assert [s["step"] for s in ser] == [0, 10, 20, 30, 40, 50]
    f = oracle.equilibrium(4, rho, ux, uy)
    for s in ser:
        ob = oracle.observables(f, comp, px, py, norm)
        assert abs(s["mass"] - ob[0]) < TOL64 * ob[0]
        assert abs(s["amp"] - ob[3]) < TOL64 * abs(ob[3]), (s["step"], s["amp"], ob[3])
        assert abs(s["time"] - s["step"] * dt) < 1e-15
        f = oracle.fd_run(f, 1 / n, dt, tau, 10)


# ---------------------------------------------------------------- engine paths
@pytest.mark.parametrize("model,q", [("cs", 3), ("fd", 4)])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_graph_replay_equals_direct_launches(model, q, prec):
    nx, ny = 70, 33
    rho, ux, uy = wl.random_smooth(nx, ny, seed=3)
    kw = dict(dt=1e-3) if model == "fd" else {}
    tau = 0.45 if model == "cs" else 2e-3
    with pkg.Lattice(model, q, nx, ny, tau, precision=prec, **kw) as A, \
            pkg.Lattice(model, q, nx, ny, tau, precision=prec, **kw) as B:
        A.init(rho, ux, uy)
        B.init(rho, ux, uy)
        A.step(70)          # two captured 32-step chunks + 6 direct steps
        for _ in range(70):
            B.step(1)
        assert A.steps_done == B.steps_done == 70
        assert np.array_equal(A.populations(), B.populations())


@pytest.mark.parametrize("model,q,prec", [("cs", 3, "fp64"), ("cs", 3, "fp32"), ("fd", 5, "fp64"), ("fd", 4, "fp32")])
def test_checkpoint_resume_is_bit_identical(model, q, prec):
    nx, ny = 45, 20
    rho, ux, uy = wl.random_smooth(nx, ny, seed=5)
    kw = dict(dt=1e-3) if model == "fd" else {}
    tau = 0.45 if model == "cs" else 2e-3
    with pkg.Lattice(model, q, nx, ny, tau, precision=prec, **kw) as A:
        A.init(rho, ux, uy)
        A.step(13)
        ck = A.save()
        A.step(21)
        fa = A.populations()
    with pkg.Lattice(model, q, nx, ny, tau, precision=prec, **kw) as B:
        B.load(ck)
        assert B.steps_done == 13
        B.step(21)
        assert np.array_equal(B.populations(), fa)


def test_batch_equals_alone():
    """Every lattice of a mixed batch computes bit-for-bit what it computes alone."""
    specs, inits = [], []
    cfg = [("cs", 3, 130, 17, 0.42, 0.0, "fp64"), ("fd", 4, 40, 33, 2e-3, 1e-3, "fp64"),
           ("cs", 3, 64, 64, 0.9, 0.0, "fp32"), ("fd", 5, 24, 24, 3e-3, 1e-3, "fp32"),
           ("cs", 3, 7, 300, 0.31, 0.0, "fp64"), ("fd", 4, 64, 8, 5e-3, 5e-4, "fp32"),
           ("fd", 4, 17, 19, 2e-3, 1e-3, "fp64"), ("cs", 3, 200, 3, 0.6, 0.0, "fp32")]
    for i, (m, q, nx, ny, tau, dt, prec) in enumerate(cfg):
        specs.append(pkg.make_spec(m, q, nx, ny, tau, dt, 0.0, prec))
        inits.append(wl.random_smooth(nx, ny, seed=40 + i))
    B = pkg.Batch(specs)
    for i, (r, u, v) in enumerate(inits):
        B.init(i, r, u, v)
    B.step(37)
    got = [B.populations(i) for i in range(len(cfg))]
    B.close()
    for i, (m, q, nx, ny, tau, dt, prec) in enumerate(cfg):
        with pkg.Lattice(m, q, nx, ny, tau, dt=dt, precision=prec) as L:
            L.init(*inits[i])
            L.step(37)
            assert np.array_equal(L.populations(), got[i]), i


def test_batch_budgets_and_tune():
    cfg = [("cs", 3, 96, 40, 0.5, 0.0), ("fd", 4, 48, 40, 2e-3, 1e-3), ("cs", 3, 33, 65, 0.7, 0.0)]
    specs = [pkg.make_spec(m, q, nx, ny, tau, dt, 0.0, "fp32") for m, q, nx, ny, tau, dt in cfg]
    B = pkg.Batch(specs)
    inits = [wl.random_smooth(c[2], c[3], seed=60 + i) for i, c in enumerate(cfg)]
    for i, (r, u, v) in enumerate(inits):
        B.init(i, r, u, v)
    B.set_budget(0, 10)
    B.set_budget(2, 45)
    rep = B.tune(2)
    assert "tile=" in rep
    B.step(40)
    B.step(20)
    assert [B.steps_done(i) for i in range(3)] == [10, 60, 45]
    got = [B.populations(i) for i in range(3)]
    B.close()
    for i, (m, q, nx, ny, tau, dt) in enumerate(cfg):
        with pkg.Lattice(m, q, nx, ny, tau, dt=dt, precision="fp32") as L:
            L.init(*inits[i])
            L.step([10, 60, 45][i])
            assert np.array_equal(L.populations(), got[i]), i


# ---------------------------------------------------------------- FP32 deviation accuracy
def _decay_fit(series, t_skip):
    t = np.array([s["time"] for s in series])
    a = np.array([s["amp"] for s in series])
    return oracle.fit_decay(t, a, t_skip)[0]


def test_fp32_cs_shear_decay_rate():
    """64x4 shear wave, 2000 steps: FP32-deviation decay rate within 1e-4 of
    the FP64 oracle's; velocity within 5e-5 of the amplitude."""
    c = wl.CS_SHEAR_64x4
    nx, ny = c["nx"], c["ny"]
    rho, ux, uy = wl.shear_wave(nx, ny, c["U"])
    comp, px, py, norm = wl.probe_shear(nx, ny)
    with pkg.Lattice("cs", 3, nx, ny, c["tau"], precision="fp32") as L:
        L.init(rho, ux, uy)
        L.set_probe(comp, px, py, norm)
        L.record(50, 100)
        L.step(2000)
        ser = L.series()
        _, _, v = L.moments()
    f = oracle.equilibrium(3, rho, ux, uy)
    ts, amps = [], []
    for s in range(0, 2000, 50):
        ts.append(s * oracle.CS_DT)
        amps.append(oracle.observables(f, comp, px, py, norm)[3])
        f = oracle.cs_run(f, c["tau"], 50)
    g_ref = oracle.fit_decay(np.array(ts), np.array(amps), 200 * oracle.CS_DT)[0]
    g = _decay_fit(ser, 200 * oracle.CS_DT)
    assert abs(g / g_ref - 1) < 1e-4, g / g_ref - 1
    _, _, v_ref = oracle.macro(3, f)
    # FP32 deviations of size ~w v U carry ~6e-8 relative rounding per step;
    # over 2000 steps the velocity error stays near 1e-5 of U
    assert np.max(np.abs(v - v_ref)) / c["U"] < 5e-5


def test_fp32_fd_taylor_green_decay_rate():
    n = 64
    rho, ux, uy = wl.taylor_green(n, n, 0.01)
    comp, px, py, norm = wl.probe_taylor_green(n, n)
    dt, tau = 2e-3, 5e-3
    steps, every = 400, 20
    with pkg.Lattice("fd", 4, n, n, tau, dt=dt, precision="fp32") as L:
        L.init(rho, ux, uy)
        L.set_probe(comp, px, py, norm)
        L.record(every, 100)
        L.step(steps)
        ser = L.series()
        _, u, _ = L.moments()
    f = oracle.equilibrium(4, rho, ux, uy)
    ts, amps = [], []
    for s in range(0, steps, every):
        ts.append(s * dt)
        amps.append(oracle.observables(f, comp, px, py, norm)[3])
        f = oracle.fd_run(f, 1 / n, dt, tau, every)
    g_ref = oracle.fit_decay(np.array(ts), np.array(amps), 0.1)[0]
    g = _decay_fit(ser, 0.1)
    assert abs(g / g_ref - 1) < 1e-4, g / g_ref - 1
    _, u_ref, _ = oracle.macro(4, f)
    assert np.max(np.abs(u - u_ref)) / 0.01 < 5e-5


# ---------------------------------------------------------------- every kernel variant
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("nx,ny", [(300, 70), (256, 64), (5, 3), (1, 1)])
def test_cs_every_tile_variant(prec, nx, ny):
    """Each CS kernel variant (plain and warp-specialised bulk-copy) gives
    bit-identical states; FP64 ones also match the oracle."""
    from paper_1904_02471_gb300 import lbm
    rho, ux, uy = wl.random_smooth(nx, ny, seed=nx + ny, amp_rho=0.1, amp_u=0.1)
    f0 = oracle.equilibrium(3, rho, ux, uy)
    tau = 0.47
    res = []
    for tile in range(lbm.lbm_n_tiles("cs")):
        for grid in (0, 1, 7):
            with pkg.Lattice("cs", 3, nx, ny, tau, precision=prec) as L:
                L.config(tile, grid)
                L.set_populations(f0)
                L.step(37)
                L.sync()
                res.append(((tile, grid), L.populations()))
    for cfg, f in res[1:]:
        assert np.array_equal(f, res[0][1]), cfg
    if prec == "fp64":
        assert rel_err(res[0][1], oracle.cs_run(f0, tau, 37)) < TOL64


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("q,nx,ny", [(4, 70, 37), (5, 33, 20), (3, 8, 5)])
def test_fd_every_tile_variant(prec, q, nx, ny):
    from paper_1904_02471_gb300 import lbm
    rho, ux, uy = wl.random_smooth(nx, ny, seed=q + nx, amp_rho=0.1, amp_u=0.1)
    f0 = oracle.equilibrium(q, rho, ux, uy)
    dx = 1.0 / nx
    dt, tau = 0.3 * dx / 3.0, 0.6 * dx / 3.0
    res = []
    for tile in range(lbm.lbm_n_tiles("fd")):
        for grid in (0, 3):
            with pkg.Lattice("fd", q, nx, ny, tau, dt=dt, precision=prec) as L:
                try:
                    L.config(tile, grid)
                except lbm.LbmError as e:  # variant too large for this set and precision
                    assert e.code == lbm.LBM_EINVAL and "shared memory" in str(e)
                    continue
                L.set_populations(f0)
                L.step(12)
                res.append(((tile, grid), L.populations()))
    for cfg, f in res[1:]:
        assert np.array_equal(f, res[0][1]), cfg
    if prec == "fp64":
        assert rel_err(res[0][1], oracle.fd_run(f0, dx, dt, tau, 12)) < TOL64


@pytest.mark.parametrize("model,q", [("cs", 3), ("fd", 4)])
@pytest.mark.parametrize("bad", ["rho_zero", "rho_negative", "ux_nan", "uy_inf", "rho_nan"])
def test_init_rejects_bad_fields_on_the_device(model, q, bad):
    """Input checks run in the initialisation kernel: one bad node anywhere
    gives LBM_EINVAL, and the lattice can be initialised again afterwards."""
    from paper_1904_02471_gb300 import lbm
    nx, ny = 37, 11
    rho, ux, uy = wl.random_smooth(nx, ny, seed=71)
    name, kind = bad.split("_")
    args = {"rho": rho, "ux": ux, "uy": uy}
    field = args[name].copy()
    field[7, 29] = {"zero": 0.0, "negative": -0.5, "nan": np.nan, "inf": np.inf}[kind]
    args[name] = field
    kw = dict(dt=1e-3) if model == "fd" else {}
    tau = 0.6 if model == "cs" else 2e-3
    with pkg.Lattice(model, q, nx, ny, tau, **kw) as L:
        with pytest.raises(lbm.LbmError) as err:
            L.init(args["rho"], args["ux"], args["uy"])
        assert err.value.code == lbm.LBM_EINVAL
        L.init(rho, ux, uy)
        L.step(3)
        f = L.populations()
    f0 = oracle.equilibrium(q, rho, ux, uy)
    ref = oracle.cs_run(f0, tau, 3) if model == "cs" else oracle.fd_run(f0, 1.0 / nx, 1e-3, tau, 3)
    assert rel_err(f, ref) < TOL64


def test_set_populations_rejects_non_finite_values():
    from paper_1904_02471_gb300 import lbm
    nx, ny = 20, 13
    rho, ux, uy = wl.random_smooth(nx, ny, seed=72)
    f0 = oracle.equilibrium(3, rho, ux, uy)
    bad = f0.copy()
    bad[4, 12, 19] = np.nan
    with pkg.Lattice("cs", 3, nx, ny, 0.6, storage="inplace") as L:
        with pytest.raises(lbm.LbmError) as err:
            L.set_populations(bad)
        assert err.value.code == lbm.LBM_EINVAL
        L.set_populations(f0)
        L.step(2)
        assert rel_err(L.populations(), oracle.cs_run(f0, 0.6, 2)) < TOL64
