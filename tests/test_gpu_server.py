"""The continuous-batching run server (lbm_server_*) on the GPU.

Each run gives the same result alone and in a mix of concurrent runs;
rounds share device time, so a cheap run is not held to the pace of an
expensive one; admission follows the memory budget and the slot count; runs
that arrive while others are on the GPU start before those finish;
cancellation; and the fitted apparent viscosity of a shear wave matches
Eq. (nulu).
"""
import math
import time

import pytest

import paper_1904_02471_gb300 as pkg
from paper_1904_02471_gb300 import lbm

pytestmark = pytest.mark.gpu

SQ3 = math.sqrt(3.0)
GB = 1 << 30


@pytest.fixture(scope="module", autouse=True)
def gpu():
    import torch
    assert torch.cuda.is_available()
    from paper_1904_02471_gb300 import build
    build.build()
    torch.cuda.init()


def _cs(n, tau, prec="fp32"):
    return pkg.make_spec("cs", 3, n, n, tau, 0.0, 0.0, prec)


def _fd(n, q, prec="fp32", tau_star=0.9, scheme="rk3"):
    # dt <= tau and a Courant number of 0.4 (CFL = 1 is unstable for
    # WENO-5 + RK3 advection along both axes)
    tau = pkg.lbm_tau_fd_from_lu(n, tau_star / SQ3)
    dt = min(tau, 0.4 * pkg.lbm_fd_max_dt(q, 1.0 / n, 1e300))
    return pkg.make_spec("fd", q, n, n, tau, dt, 0.0, prec, scheme=scheme)


MIX = [
    (lambda: _cs(64, 0.5), 300, "tg", 0.01 * SQ3),
    (lambda: _fd(48, 4), 200, "tg", 0.01),
    (lambda: _cs(96, 0.7, "fp64"), 450, "shear", 0.01 * SQ3),
    (lambda: _fd(32, 5, "fp64"), 120, "tg", 0.01),
    (lambda: _cs(40, 1.0), 600, "shear", 0.02 * SQ3),
    (lambda: _fd(40, 4), 260, "shock", 0.0),
    (lambda: _cs(128, 0.35), 100, "shock", 0.0),
    (lambda: _fd(56, 4, "fp32", 1.4), 330, "tg", 0.01),
    (lambda: _fd(44, 4, "fp32", 1.1, "rk3_fused"), 170, "tg", 0.01),   # temporally blocked step
    (lambda: _fd(36, 3, "fp64", 0.8, "rk3_fused"), 90, "shear", 0.01),
]


def _req(i):
    spec_fn, steps, init, U = MIX[i]
    return lbm.make_request(spec_fn(), steps, init, U, obs_every=10, rho_l=1.2, rho_r=0.8, tag=i)


def _run(reqs, budget=8 * GB, slots=64, chunk=64):
    with lbm.Server(budget, slots, chunk) as S:
        tickets = [S.submit(r) for r in reqs]
        S.drain(300)
        return [(S.poll(t), S.series(t)) for t in tickets]


def test_mix_equals_alone():
    """Every run's final observables and series are the same whether it runs
    alone or together with the others (4 slots, so some wait in the queue)."""
    mixed = _run([_req(i) for i in range(len(MIX))], slots=4, chunk=48)
    for i in range(len(MIX)):
        (res_m, ser_m), = [mixed[i]]
        (res_a, ser_a), = _run([_req(i)], chunk=48)
        assert res_m["status"] == lbm.LBM_OK and res_a["status"] == lbm.LBM_OK, (i, res_m["status"])
        assert res_m["user_tag"] == i and res_m["steps"] == MIX[i][1]
        for key in ("mass", "mom_x", "mom_y", "amp"):
            a, b = res_m["last"][key], res_a["last"][key]
            assert abs(a - b) <= 1e-12 * max(1.0, abs(res_a["last"]["mass"]) if key != "amp" else abs(b)), (i, key, a, b)
        assert len(ser_m) == len(ser_a) == MIX[i][1] // 10
        for sm, sa in zip(ser_m, ser_a):
            assert sm["step"] == sa["step"]
            assert abs(sm["amp"] - sa["amp"]) <= 1e-12 * abs(sa["amp"]) + 1e-300


def test_admission_follows_budget_and_slots():
    spec = _cs(1024, 0.6)
    one = 2 * 9 * 1056 * 1024 * 4  # about one lattice's state
    with lbm.Server(int(1.5 * one) + (1 << 20), 8, 32) as S:
        t1 = S.submit(lbm.make_request(spec, 400, "tg", 0.01))
        t2 = S.submit(lbm.make_request(spec, 100, "tg", 0.01))
        S.drain(300)
        r1, r2 = S.poll(t1), S.poll(t2)
    assert r1["status"] == r2["status"] == lbm.LBM_OK
    assert r2["t_admit"] >= r1["t_done"] - 1e-3, (r1, r2)  # second waited for memory
    with lbm.Server(1 << 20, 8, 32) as S:
        with pytest.raises(lbm.LbmError) as ei:
            S.submit(lbm.make_request(spec, 10, "tg", 0.01))
        assert ei.value.code == lbm.LBM_ENOMEM


def test_late_arrivals_overlap():
    """A run submitted while a long run is on the GPU starts (and ends) before it."""
    with lbm.Server(8 * GB, 8, 32) as S:
        t_long = S.submit(lbm.make_request(_cs(512, 0.6), 4000, "tg", 0.01))
        time.sleep(0.05)
        t_short = S.submit(lbm.make_request(_fd(64, 4), 50, "tg", 0.01))
        S.drain(300)
        rl, rs = S.poll(t_long), S.poll(t_short)
    assert rl["status"] == rs["status"] == lbm.LBM_OK
    assert rs["t_admit"] < rl["t_done"] and rs["t_done"] < rl["t_done"]


def test_cancel():
    with lbm.Server(8 * GB, 1, 32) as S:
        t1 = S.submit(lbm.make_request(_cs(256, 0.6), 200000, "tg", 0.01))
        t2 = S.submit(lbm.make_request(_cs(256, 0.6), 10, "tg", 0.01))
        time.sleep(0.2)
        S.cancel(t2)  # still queued (one slot)
        S.cancel(t1)  # running
        S.drain(120)
        assert S.poll(t2)["status"] == lbm.LBM_ECANCELLED
        r1 = S.poll(t1)
        assert r1["status"] == lbm.LBM_ECANCELLED and r1["steps"] < 200000
        with pytest.raises(lbm.LbmError):
            S.poll(12345)


def test_unstable_run_is_reported_non_finite():
    """A run that blows up (FD at CFL = 1 along both axes) finishes with
    LBM_ENONFINITE instead of a silent NaN result; the others are unaffected."""
    n, q = 56, 4
    tau = pkg.lbm_tau_fd_from_lu(n, 1.4 / SQ3)
    bad = pkg.make_spec("fd", q, n, n, tau, pkg.lbm_fd_max_dt(q, 1.0 / n, tau), 0.0, "fp32")
    res = _run([lbm.make_request(bad, 330, "tg", 0.01), _req(0)])
    assert res[0][0]["status"] == lbm.LBM_ENONFINITE
    assert res[1][0]["status"] == lbm.LBM_OK


def test_shear_wave_viscosity_fit():
    """nu_fit of a CS shear wave is nu_LU = tau_LU - dt/2 (Eq. nulu) to within
    the discretisation error of a 64-node wave."""
    tau = 0.8 / SQ3
    spec = pkg.make_spec("cs", 3, 64, 4, tau, 0.0, 0.0, "fp64")
    with lbm.Server(GB, 4, 100) as S:
        t = S.submit(lbm.make_request(spec, 2000, "shear", 0.01 * SQ3, obs_every=50))
        S.drain(120)
        r = S.poll(t)
    nu = pkg.lbm_nu(lbm.LBM_CS, tau, 1 / SQ3)
    assert r["status"] == lbm.LBM_OK
    assert abs(r["nu_fit"] / nu - 1) < 2e-3, r["nu_fit"] / nu


def test_cheap_run_is_not_held_to_the_pace_of_an_expensive_one():
    """Rounds share device time, not steps: a cheap run (CS 64^2) with more
    steps than an expensive one (FD 16-velocity 1024^2), submitted after it,
    finishes first. With rounds of equal steps it would finish last."""
    with lbm.Server(8 * GB, 8, 32) as S:
        t_long = S.submit(lbm.make_request(_fd(1024, 4), 300, "tg", 0.01))
        t_short = S.submit(lbm.make_request(_cs(64, 0.6), 1000, "tg", 0.01 * SQ3))
        S.drain(300)
        rl, rs = S.poll(t_long), S.poll(t_short)
    assert rl["status"] == rs["status"] == lbm.LBM_OK
    assert rl["steps"] == 300 and rs["steps"] == 1000
    assert rs["t_done"] < rl["t_done"], (rs["t_done"], rl["t_done"])


def test_kept_moments_and_release():
    """A run submitted with keep_moments returns its final rho, u fields, the
    same as the lattice computes alone; releasing a finished ticket frees its
    result, series and fields (later calls: LBM_ENOTFOUND) and drops it from
    the finished count, while a running ticket cannot be released."""
    import numpy as np
    import lbm_workloads as wl
    spec = _cs(64, 0.5)
    U = 0.01 * SQ3
    with lbm.Server(8 * GB, 8, 32) as S:
        t_keep = S.submit(lbm.make_request(spec, 300, "tg", U, obs_every=10, keep_moments=True))
        t_plain = S.submit(lbm.make_request(spec, 300, "tg", U, obs_every=10))
        t_long = S.submit(lbm.make_request(_cs(512, 0.6), 200000, "tg", 0.01))
        while S.poll(t_keep) is None or S.poll(t_plain) is None:
            time.sleep(0.01)
        with pytest.raises(lbm.LbmError) as ei:
            S.release(t_long)               # still running
        assert ei.value.code == lbm.LBM_ENOTREADY
        rho, ux, uy = S.moments(t_keep, 64, 64)
        with pytest.raises(lbm.LbmError) as ei:
            S.moments(t_plain, 64, 64)       # not kept
        assert ei.value.code == lbm.LBM_ENOTFOUND
        assert len(S.series(t_keep)) == 30
        before = S.stats()["finished"]
        S.release(t_keep)
        assert S.stats()["finished"] == before - 1
        for call in (lambda: S.poll(t_keep), lambda: S.series(t_keep), lambda: S.moments(t_keep, 64, 64),
                     lambda: S.release(t_keep)):
            with pytest.raises(lbm.LbmError) as ei:
                call()
            assert ei.value.code == lbm.LBM_ENOTFOUND
        S.cancel(t_long)
        S.drain(120)                         # released tickets do not hold the drain
        S.release(t_plain)
        S.release(t_long)
        assert S.stats()["finished"] == 0
    with pkg.Lattice("cs", 3, 64, 64, 0.5, precision="fp32", storage="ab") as L:
        L.init(*wl.taylor_green(64, 64, U))
        L.step(300)
        r2, u2, v2 = L.moments()
    # the server forms the initial fields itself (libm sin/cos; the test uses
    # numpy's), so the two FP32 runs may differ by a float rounding
    assert np.max(np.abs(rho - r2)) < 1e-6
    assert np.max(np.abs(ux - u2)) < 1e-5 * U and np.max(np.abs(uy - v2)) < 1e-5 * U
