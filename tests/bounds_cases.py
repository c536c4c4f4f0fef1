"""Cases run against the bounds-checked build of the library (the library
selected by LBM_LIBRARY): every CS and FD kernel variant (FD: also the
temporally blocked step), both CS storages,
both precisions, ragged and degenerate sizes, batches with step budgets,
region readouts that wrap, checkpoints. A kernel that reaches outside a state
buffer makes the step fail with LBM_ECUDA; FP64 results are also checked
against the oracle. Run by tests/test_gpu_bounds.py in a child process.
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import lbm_workloads as wl  # noqa: E402
import oracle  # noqa: E402
import paper_1904_02471_gb300 as pkg  # noqa: E402
from paper_1904_02471_gb300 import lbm  # noqa: E402


def rel_err(a, b):
    return float(np.max(np.abs(a - b) / np.abs(b)))


def cs_cases():
    n = 0
    for nx, ny in [(1, 1), (5, 1), (1, 6), (7, 3), (33, 65), (260, 40)]:
        rho, ux, uy = wl.random_smooth(nx, ny, seed=nx + 7 * ny, amp_rho=0.1, amp_u=0.1)
        f0 = oracle.equilibrium(3, rho, ux, uy)
        ref = oracle.cs_run(f0, 0.47, 5)
        for prec in ("fp64", "fp32"):
            for storage in ("ab", "inplace"):
                for tile in range(lbm.lbm_n_tiles("cs")):
                    for grid in (0, 5):
                        with pkg.Lattice("cs", 3, nx, ny, 0.47, precision=prec, storage=storage) as L:
                            L.config(tile, grid)
                            L.set_populations(f0)
                            L.step(5)
                            L.sync()
                            f = L.populations()
                            L.moments()
                            L.observables()
                            L.populations_region(nx - 1, ny - 1, min(3, nx), min(2, ny))
                            if prec == "fp64":
                                assert rel_err(f, ref) < 1e-12, (nx, ny, storage, tile, grid)
                            n += 1
    return n


def fd_cases():
    n = 0
    for q in (3, 4, 5):
        for nx, ny in [(6, 6), (7, 9), (40, 17), (70, 33)]:
            rho, ux, uy = wl.random_smooth(nx, ny, seed=q + nx + ny, amp_rho=0.05, amp_u=0.05)
            f0 = oracle.equilibrium(q, rho, ux, uy)
            dt = 0.4 * pkg.lbm_fd_max_dt(q, 1.0 / nx, 1e300)
            tau = 2 * dt
            ref = oracle.fd_run(f0, 1.0 / nx, dt, tau, 2)
            for prec in ("fp64", "fp32"):
                for tile in range(lbm.lbm_n_tiles("fd")):
                    with pkg.Lattice("fd", q, nx, ny, tau, dt=dt, precision=prec) as L:
                        try:
                            L.config(tile, 3)
                        except lbm.LbmError as e:  # variant too large for this set and precision
                            assert e.code == lbm.LBM_EINVAL
                            continue
                        L.set_populations(f0)
                        L.step(2)
                        L.sync()
                        f = L.populations()
                        L.observables()
                        L.populations_region(nx - 2, 0, min(5, nx), min(3, ny))
                        if prec == "fp64":
                            assert rel_err(f, ref) < 1e-12, (q, nx, ny, tile)
                        n += 1
    return n


def fused_cases():
    """Temporally blocked FD steps: halos of 9 nodes that wrap (also several
    times around lattices smaller than the halo), interior tiles staged
    without wrap, an odd step count (the state ends in the second buffer)."""
    n = 0
    for q in (3, 4, 5):
        for nx, ny in [(1, 1), (6, 6), (7, 9), (40, 17), (70, 33), (96, 40)]:
            rho, ux, uy = wl.random_smooth(nx, ny, seed=q + 3 * nx + ny, amp_rho=0.05, amp_u=0.05)
            f0 = oracle.equilibrium(q, rho, ux, uy)
            dt = 0.4 * pkg.lbm_fd_max_dt(q, 1.0 / nx, 1e300)
            tau = 2 * dt
            ref = oracle.fd_run(f0, 1.0 / nx, dt, tau, 3)
            for prec in ("fp64", "fp32"):
                for tile in range(lbm.lbm_n_tiles("fd")):
                    with pkg.Lattice("fd", q, nx, ny, tau, dt=dt, precision=prec, scheme="rk3_fused") as L:
                        try:
                            L.config(tile, 3)
                        except lbm.LbmError as e:  # no fused kernel for this tile, or too large
                            assert e.code == lbm.LBM_EINVAL
                            continue
                        L.set_populations(f0)
                        L.step(3)
                        L.sync()
                        f = L.populations()
                        L.observables()
                        L.populations_region(max(nx - 2, 0), 0, min(5, nx), min(3, ny))
                        if prec == "fp64":
                            assert rel_err(f, ref) < 1e-12, (q, nx, ny, tile)
                        n += 1
    return n


def batch_case():
    cfg = [("cs", 3, 130, 17, 0.42, 0.0, "fp64", "inplace"), ("fd", 4, 40, 33, 2e-3, 1e-3, "fp32", "ab"),
           ("cs", 3, 7, 300, 0.31, 0.0, "fp32", "ab"), ("fd", 5, 24, 24, 3e-3, 1e-3, "fp64", "ab"),
           ("cs", 3, 200, 3, 0.6, 0.0, "fp32", "inplace"), ("fd", 3, 6, 6, 5e-3, 1e-3, "fp32", "ab")]
    specs = [pkg.make_spec(m, q, nx, ny, tau, dt, 0.0, prec, storage=st) for m, q, nx, ny, tau, dt, prec, st in cfg]
    B = pkg.Batch(specs)
    try:
        for i, c in enumerate(cfg):
            B.init(i, *wl.random_smooth(c[2], c[3], seed=90 + i))
        B.set_budget(1, 3)
        B.set_budget(4, 4)
        B.tune(1)
        B.step(7)
        B.sync()
        for i in range(len(cfg)):
            B.populations(i)
            B.observables(i)
    finally:
        B.close()


def checkpoint_case():
    with pkg.Lattice("cs", 3, 45, 20, 0.45, storage="inplace") as A:
        A.init(*wl.random_smooth(45, 20, seed=3))
        A.step(3)
        ck = A.save()
    with pkg.Lattice("cs", 3, 45, 20, 0.45, storage="inplace") as B:
        B.load(ck)
        B.step(4)
        B.sync()


def main():
    assert os.environ.get("LBM_LIBRARY"), "run with LBM_LIBRARY set to the bounds-checked build"
    import torch
    torch.cuda.init()
    n_cs = cs_cases()
    n_fd = fd_cases()
    n_ff = fused_cases()
    batch_case()
    checkpoint_case()
    print(f"bounds-checked runs ok: {n_cs} CS, {n_fd} FD, {n_ff} fused FD, batch, checkpoint")


if __name__ == "__main__":
    main()
