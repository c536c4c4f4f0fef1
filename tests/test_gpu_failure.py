"""Failure detection on the GPU without a GPU fault.

The CS bulk-copy kernel (the default CS kernel) is the library's only kernel
with device-side waits, and every wait is bounded (2 s of device time and an
iteration cap). The test injection lbm_inject_wait_timeout makes the first
block's producer skip one row's copies, so that row's consumers wait on an
mbarrier that nothing completes (the "flag that nothing sets"), and limits
every wait to 1 ms. The wait runs out, the launch sets its error word and
finishes after the copies in flight have landed; the host reports
LBM_ETIMEOUT. With the injection off, the same context computes again what
the oracle computes: the CUDA context stays usable.
"""
import math
import time

import numpy as np
import pytest

import lbm_workloads as wl
import oracle
import paper_1904_02471_gb300 as pkg
from paper_1904_02471_gb300 import lbm

pytestmark = pytest.mark.gpu

SQ3 = math.sqrt(3.0)
TAU = 0.8 / SQ3
INJECT_US = 1000


@pytest.fixture(scope="module", autouse=True)
def gpu():
    import torch
    assert torch.cuda.is_available()
    from paper_1904_02471_gb300 import build
    build.build()
    torch.cuda.init()


def rel_err(a, b):
    return float(np.max(np.abs(a - b) / np.abs(b)))


def test_lattice_wait_runs_out_and_context_recovers():
    n = 64
    rho, ux, uy = wl.taylor_green(n, n, 0.01 * SQ3)
    with pkg.Lattice("cs", 3, n, n, TAU) as L:
        L.init(rho, ux, uy)
        L.inject_wait_timeout(INJECT_US)
        t0 = time.perf_counter()
        with pytest.raises(lbm.LbmError) as err:
            L.step(1)
            L.sync()
        assert err.value.code == lbm.LBM_ETIMEOUT
        assert time.perf_counter() - t0 < 30.0
        L.inject_wait_timeout(0)
        L.init(rho, ux, uy)
        L.step(7)
        L.sync()
        f = L.populations()
    ref = oracle.cs_run(oracle.equilibrium(3, rho, ux, uy), TAU, 7)
    assert rel_err(f, ref) < 1e-12


def test_batch_reports_timeout_then_steps_normally():
    n = 96
    specs = [pkg.make_spec("cs", 3, n, n, TAU, 0.0, 0.0, "fp32"),
             pkg.make_spec("cs", 3, 48, 40, TAU, 0.0, 0.0, "fp32")]
    B = pkg.Batch(specs)
    try:
        for i, s in enumerate(specs):
            B.init(i, *wl.taylor_green(s.nx, s.ny, 0.01 * SQ3))
        B.inject_wait_timeout(INJECT_US)
        with pytest.raises(lbm.LbmError) as err:
            B.step(2)
            B.sync()
        assert err.value.code == lbm.LBM_ETIMEOUT
        B.inject_wait_timeout(0)
        for i, s in enumerate(specs):
            B.init(i, *wl.taylor_green(s.nx, s.ny, 0.01 * SQ3))
        B.step(3)
        B.sync()
        for i, s in enumerate(specs):
            r, u, v = B.moments(i)
            r0, u0, v0 = wl.taylor_green(s.nx, s.ny, 0.01 * SQ3)
            f = oracle.cs_run(oracle.equilibrium(3, r0, u0, v0), TAU, 3)
            rr, uu, vv = oracle.macro(3, f)
            # float32 deviations: a few roundings of values <= 1e-2 per step
            assert np.max(np.abs(u - uu)) < 1e-6 and np.max(np.abs(r - rr)) < 1e-6
    finally:
        B.close()


def test_server_run_fails_with_timeout_and_next_run_succeeds():
    req = lambda tag: lbm.make_request(pkg.make_spec("cs", 3, 64, 64, TAU, 0.0, 0.0, "fp32"), 200, "tg",
                                       0.01 * SQ3, obs_every=10, tag=tag)
    with lbm.Server(1 << 30, 4, 50) as S:
        S.inject_wait_timeout(INJECT_US)
        bad = S.submit(req(1))
        S.drain(120)
        assert S.poll(bad)["status"] == lbm.LBM_ETIMEOUT
        S.inject_wait_timeout(0)
        good = S.submit(req(2))
        S.drain(120)
        res = S.poll(good)
        assert res["status"] == lbm.LBM_OK and res["steps"] == 200
        assert res["last"]["nonfinite"] == 0
