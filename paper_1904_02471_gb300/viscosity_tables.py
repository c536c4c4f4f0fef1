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
reported. Runs are on the GPU through the library (FP64 storage). The FD
columns are computed for the 3-node set (whose largest speed sqrt(3) the
paper's CFL argument of Sec. 4.1 implies) and the 4-node set, and for a sweep
of the WENO-5 regulariser eps (the paper does not print it; 1e-6 is the
library's default, 1e30 gives the linear weights). With --paper the printed
Table 1-2 columns are added to the output as context.

    python -m paper_1904_02471_gb300.viscosity_tables [--q 3 4] [--eps 1e-6 ...] [--t-end 1.0]
        [--json out.json] [--paper tests/golden/paper_values.json]
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


def run_series(model, kind, n, q=4, nu0=5e-4, dt_fd=5e-4, t_end=1.0, U=0.01, samples=50, precision="fp64",
               eps=None):
    """Recorded amplitude of one run: (t in FD units, A, every, steps)."""
    import paper_1904_02471_gb300 as pkg
    (rho, ux, uy), (comp, px, py, norm) = _fields(kind, n, U)
    if model == "fd":
        L = pkg.Lattice("fd", q, n, n, nu0, dt=dt_fd, precision=precision)
        if eps is not None:
            L.set_weno_eps(eps)
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
    return t, a, every, steps


def fit_nu(kind, t, a, t_end):
    """nu_app of a recorded amplitude: log-linear fit over t >= t_end / 10,
    gamma / (m k^2), m = 1 shear (Eq. shear_sol), 2 Taylor-Green (Eq. taylor)."""
    import paper_1904_02471_gb300 as pkg
    gamma, _ = pkg.lbm_fit_decay(t, a, 0.1 * t_end)
    k2 = (2 * math.pi) ** 2 * (1 if kind == "shear" else 2)
    return gamma / k2


def nu_app(model, kind, n, q=4, nu0=5e-4, dt_fd=5e-4, t_end=1.0, U=0.01, samples=50, precision="fp64", eps=None):
    """Apparent viscosity (FD units) of one run."""
    t, a, _, _ = run_series(model, kind, n, q, nu0, dt_fd, t_end, U, samples, precision, eps)
    return fit_nu(kind, t, a, t_end)


def table(kind, ns=(20, 30, 40, 50, 60), qs=(4,), epss=(None,), nu0=5e-4, t_end=1.0):
    """One row per N: CS, and FD for each velocity set q and WENO eps
    (key fd_q{q}_eps{eps}; eps None is the library default)."""
    rows = []
    for n in ns:
        cs = nu_app("cs", kind, n, nu0=nu0, t_end=t_end)
        r = {"N": n, "tau_lu": (n * nu0 + SQ3 / 6), "cs_nu_app": cs, "cs_rel_err": abs(cs / nu0 - 1)}
        for q in qs:
            for eps in epss:
                fd = nu_app("fd", kind, n, q=q, nu0=nu0, t_end=t_end, eps=eps)
                tag = f"fd_q{q}" + ("" if eps is None else f"_eps{eps:g}")
                r[tag + "_nu_app"] = fd
                r[tag + "_rel_err"] = abs(fd / nu0 - 1)
        rows.append(r)
    return rows


def order(rows, key):
    """Least-squares slope of log(err) against log(N) (convergence order)."""
    n = np.log([r["N"] for r in rows])
    e = np.log([max(r[key], 1e-300) for r in rows])
    return -np.polyfit(n, e, 1)[0]


def main():
    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("--q", type=int, nargs="+", default=[3, 4])
    ap.add_argument("--eps", type=float, nargs="+", default=[1e-6, 1e-8, 1e-10, 1e-12, 1e30])
    ap.add_argument("--t-end", type=float, default=1.0)
    ap.add_argument("--json", default="")
    ap.add_argument("--paper", default="", help="JSON with the printed Table 1-2 columns (context)")
    a = ap.parse_args()
    torch.cuda.init()
    epss = [None if e == 1e-6 else e for e in a.eps]
    out = {"about": "apparent viscosity nu_app (FD units) of shear waves (Table 1 set-up) and Taylor-Green "
                    "vortices (Table 2 set-up), nu_0 = tau_FD = 5e-4, FD dt = 5e-4, t_end = %g, FP64; FD keys "
                    "fd_q{nodes per axis}[_eps{WENO eps}] (no eps: 1e-6)" % a.t_end}
    for kind in ("shear", "tg"):
        rows = table(kind, qs=a.q, epss=epss, t_end=a.t_end)
        keys = [k[:-len("_rel_err")] for k in rows[0] if k.endswith("_rel_err")]
        out[kind] = {"rows": rows, "order": {k: order(rows, k + "_rel_err") for k in keys}}
        print(f"{kind}: N  tau_LU  " + "  ".join(keys))
        for r in rows:
            print(f"  {r['N']:3d} {r['tau_lu']:.4f} " + " ".join(f"{r[k + '_rel_err']:.2e}" for k in keys))
        print("  order: " + ", ".join(f"{k} {v:.2f}" for k, v in out[kind]["order"].items()))
    if a.paper:
        with open(a.paper) as fh:
            out["paper_printed"] = json.load(fh)["nu_app_tables"]
    if a.json:
        with open(a.json, "w") as fh:
            json.dump(out, fh, indent=1)


if __name__ == "__main__":
    main()
