"""Apparent viscosity of CS and FD runs of the same physical system (the set-up
of Tables 1-2 of the paper, Sec. 4.2-4.3).

For N = 20..60 nodes per wavelength and nu_FD = tau_FD = 5e-4 (FD units: unit
domain, T = m = 1):
  * FD: dx = 1/N, dt = 5e-4, nu_app from a log-linear fit of the projected
    amplitude against Eq. (shear_sol) (shear wave, k = (2 pi, 0)) or Eq.
    (taylor) (Taylor-Green, k = (2 pi, 2 pi));
  * CS: D2Q9 with tau_LU = N tau_FD + sqrt(3)/6 (Eq. nu-transfer), times
    converted by t_FD = t_LU / N, so nu_app is in FD units too.
The relative error |nu_app / nu_0 - 1| and its order of convergence in N are
reported. Runs are on the GPU through the library (FP64 storage).

    python -m paper_1904_02471_gb300.viscosity_tables [--q 4] [--t-end 1.0] [--json out.json]
"""
from __future__ import annotations

import argparse
import json
import math

import numpy as np

SQ3 = math.sqrt(3.0)


def _fields(kind, n, U):
    import lbm_workloads as wl
    if kind == "shear":
        return wl.shear_wave(n, n, U), wl.probe_shear(n, n)
    return wl.taylor_green(n, n, U), wl.probe_taylor_green(n, n)


def nu_app(model, kind, n, q=4, nu0=5e-4, dt_fd=5e-4, t_end=1.0, U=0.01, samples=50, precision="fp64"):
    """Apparent viscosity (FD units) of one run."""
    import paper_1904_02471_gb300 as pkg
    (rho, ux, uy), (comp, px, py, norm) = _fields(kind, n, U)
    if model == "fd":
        L = pkg.Lattice("fd", q, n, n, nu0, dt=dt_fd, precision=precision)
        steps = int(round(t_end / dt_fd))
        t_unit = dt_fd                       # FD time per step
    else:
        L = pkg.Lattice("cs", 3, n, n, pkg.lbm_tau_lu_from_fd(n, nu0), precision=precision)
        steps = int(round(t_end * n * SQ3))  # t_FD = steps * dt_LU / N
        t_unit = 1.0 / (SQ3 * n)
    every = max(1, steps // samples)
    with L:
        L.init(rho, ux, uy)
        L.set_probe(comp, px, py, norm)
        L.record(every, steps // every + 2)
        L.step(steps)
        ser = L.series()
    t = np.array([s["step"] for s in ser], float) * t_unit
    a = np.array([s["amp"] for s in ser])
    gamma, _ = pkg.lbm_fit_decay(t, a, 0.1 * t_end)
    k2 = (2 * math.pi) ** 2 * (1 if kind == "shear" else 2)
    return gamma / k2


def table(kind, ns=(20, 30, 40, 50, 60), q=4, nu0=5e-4, t_end=1.0):
    rows = []
    for n in ns:
        cs = nu_app("cs", kind, n, nu0=nu0, t_end=t_end)
        fd = nu_app("fd", kind, n, q=q, nu0=nu0, t_end=t_end)
        rows.append({"N": n, "tau_lu": (n * nu0 + SQ3 / 6), "cs_nu_app": cs, "cs_rel_err": abs(cs / nu0 - 1),
                     "fd_nu_app": fd, "fd_rel_err": abs(fd / nu0 - 1)})
    return rows


def order(rows, key):
    """Least-squares slope of log(err) against log(N) (convergence order)."""
    n = np.log([r["N"] for r in rows])
    e = np.log([max(r[key], 1e-300) for r in rows])
    return -np.polyfit(n, e, 1)[0]


def main():
    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("--q", type=int, default=4)
    ap.add_argument("--t-end", type=float, default=1.0)
    ap.add_argument("--json", default="")
    a = ap.parse_args()
    torch.cuda.init()
    out = {}
    for kind in ("shear", "tg"):
        rows = table(kind, q=a.q, t_end=a.t_end)
        out[kind] = {"rows": rows, "cs_order": order(rows, "cs_rel_err"), "fd_order": order(rows, "fd_rel_err")}
        print(f"{kind}: N  tau_LU  CS nu_app  rel.err   FD nu_app  rel.err")
        for r in rows:
            print(f"  {r['N']:3d} {r['tau_lu']:.4f} {r['cs_nu_app']:.7f} {r['cs_rel_err']:.2e} "
                  f"{r['fd_nu_app']:.7f} {r['fd_rel_err']:.2e}")
        print(f"  order: CS {out[kind]['cs_order']:.2f}, FD {out[kind]['fd_order']:.2f}")
    if a.json:
        with open(a.json, "w") as fh:
            json.dump(out, fh, indent=1)


if __name__ == "__main__":
    main()
