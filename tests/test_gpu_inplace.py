"""In-place CS storage (one buffer, AA access pattern) on the GPU.

An in-place lattice performs the same collision on the same values as a
two-buffer lattice, only stored elsewhere, so every readout must agree bit
for bit after any number of steps (even and odd phases), for every CS kernel
variant and grid, in both precisions; FP64 also matches the oracle. State
writes, checkpoints and batches mixing both storages are covered, and the
server admits an in-place run with half the memory.
"""
import math

import numpy as np
import pytest

import lbm_workloads as wl
import oracle
import paper_1904_02471_gb300 as pkg
from paper_1904_02471_gb300 import lbm

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


def _run(storage, prec, nx, ny, tau, f0, steps, tile=None, grid=0):
    with pkg.Lattice("cs", 3, nx, ny, tau, precision=prec, storage=storage) as L:
        if tile is not None:
            L.config(tile, grid)
        L.set_populations(f0)
        out = []
        done = 0
        for n in steps:
            L.step(n - done)
            done = n
            r, u, v = L.moments()
            out.append((L.populations(), r, u, v, L.observables()["mass"]))
        return out


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("nx,ny", [(37, 23), (64, 4), (300, 70), (5, 1)])
def test_inplace_equals_two_buffers_every_variant(prec, nx, ny):
    rho, ux, uy = wl.random_smooth(nx, ny, seed=nx * ny, amp_rho=0.1, amp_u=0.1)
    f0 = oracle.equilibrium(3, rho, ux, uy)
    tau = 0.47
    steps = [1, 2, 5, 40]
    ref = _run("ab", prec, nx, ny, tau, f0, steps)
    for tile in range(lbm.lbm_n_tiles("cs")):
        for grid in (0, 3):
            got = _run("inplace", prec, nx, ny, tau, f0, steps, tile, grid)
            for (fa, ra, ua, va, ma), (fb, rb, ub, vb, mb), n in zip(ref, got, steps):
                assert np.array_equal(fa, fb), (tile, grid, n)
                assert np.array_equal(ra, rb) and np.array_equal(ua, ub) and np.array_equal(va, vb), (tile, grid, n)
                assert ma == mb, (tile, grid, n)
    if prec == "fp64":
        assert rel_err(ref[-1][0], oracle.cs_run(f0, tau, steps[-1])) < 1e-12


@pytest.mark.parametrize("phase_steps", [3, 4])
def test_inplace_checkpoint_and_state_write_at_either_phase(phase_steps):
    nx, ny, tau = 45, 20, 0.45
    rho, ux, uy = wl.random_smooth(nx, ny, seed=7)
    with pkg.Lattice("cs", 3, nx, ny, tau, storage="inplace") as A:
        A.init(rho, ux, uy)
        A.step(phase_steps)
        assert A.device_view().cs_pull_phase == (2 if phase_steps % 2 else 0)
        ck = A.save()
        f_mid = A.populations()
        A.step(9)
        fa = A.populations()
    with pkg.Lattice("cs", 3, nx, ny, tau, storage="inplace") as B:
        B.load(ck)
        B.step(9)
        assert np.array_equal(B.populations(), fa)
    # writing a state at the odd phase, then stepping, equals the oracle
    with pkg.Lattice("cs", 3, nx, ny, tau, storage="inplace") as C:
        C.init(rho, ux, uy)
        C.step(1)
        C.set_populations(f_mid)
        C.step(9)
        assert rel_err(C.populations(), oracle.cs_run(f_mid, tau, 9)) < 1e-12


def test_batch_mixing_storages_equals_alone():
    cfg = [("cs", 96, 40, 0.5, "fp32", "inplace"), ("cs", 33, 65, 0.7, "fp32", "ab"),
           ("cs", 130, 17, 0.42, "fp64", "inplace"), ("fd", 40, 33, 2e-3, "fp64", "ab"),
           ("cs", 64, 64, 0.9, "fp32", "inplace")]
    specs = []
    for m, nx, ny, tau, prec, st in cfg:
        q = 3 if m == "cs" else 4
        dt = 1e-3 if m == "fd" else 0.0
        specs.append(pkg.make_spec(m, q, nx, ny, tau, dt, 0.0, prec, storage=st))
    inits = [wl.random_smooth(c[1], c[2], seed=80 + i) for i, c in enumerate(cfg)]
    B = pkg.Batch(specs)
    try:
        for i, (r, u, v) in enumerate(inits):
            B.init(i, r, u, v)
        B.set_budget(4, 7)    # leaves the others one phase apart
        B.step(11)
        B.sync()
        got = [B.populations(i) for i in range(len(cfg))]
    finally:
        B.close()
    for i, (m, nx, ny, tau, prec, st) in enumerate(cfg):
        q = 3 if m == "cs" else 4
        kw = dict(dt=1e-3) if m == "fd" else {}
        with pkg.Lattice(m, q, nx, ny, tau, precision=prec, storage=st, **kw) as L:
            L.init(*inits[i])
            L.step(7 if i == 4 else 11)
            assert np.array_equal(L.populations(), got[i]), i


def test_server_admits_inplace_run_with_half_the_memory():
    """A budget between the one-buffer and the two-buffer footprint of a
    512^2 FP32 CS run: the two-buffer request can never fit (rejected at
    submit), the in-place one runs."""
    n = 512
    pitch = (n + 8 + 31) // 32 * 32
    buffer_bytes = (9 * pitch * n + 1024) * 4
    budget = int(1.5 * buffer_bytes)
    spec_ab = pkg.make_spec("cs", 3, n, n, 0.8 / SQ3, 0.0, 0.0, "fp32")
    spec_in = pkg.make_spec("cs", 3, n, n, 0.8 / SQ3, 0.0, 0.0, "fp32", storage="inplace")
    with lbm.Server(budget, 2, 500) as S:
        with pytest.raises(lbm.LbmError) as err:
            S.submit(lbm.make_request(spec_ab, 1000, "tg", 0.01 * SQ3, obs_every=100, tag=1))
        assert err.value.code == lbm.LBM_ENOMEM
        t = S.submit(lbm.make_request(spec_in, 1001, "tg", 0.01 * SQ3, obs_every=100, tag=2))
        S.drain(120)
        res = S.poll(t)
        assert res["status"] == lbm.LBM_OK and res["steps"] == 1001 and res["last"]["nonfinite"] == 0
    # and it computes what the two-buffer lattice computes
    rho, ux, uy = wl.taylor_green(n, n, 0.01 * SQ3)
    outs = []
    for st in ("ab", "inplace"):
        with pkg.Lattice("cs", 3, n, n, 0.8 / SQ3, precision="fp32", storage=st) as L:
            L.init(rho, ux, uy)
            L.step(1001)
            outs.append(L.observables())
    assert outs[0]["mass"] == outs[1]["mass"] and outs[0]["mom_x"] == outs[1]["mom_x"]
