"""Small single-lattice cases for kernel profiling (e.g. under Nsight Compute).

    python -m paper_1904_02471_gb300.profile_cases cs  [--n 2048] [--steps 4] [--tile 5] [--grid G] [--storage inplace]
    python -m paper_1904_02471_gb300.profile_cases fd  [--n 1024] [--steps 2] [--tile 0] [--q 4] [--grid G]

Each case is a Taylor-Green lattice in FP32 deviation storage whose state is
larger than the 129 MB L2 (CS 2048^2: 302 MB; FD 16-velocity 1024^2: 201 MB),
so DRAM counters mean what they say, yet small enough that a multi-pass
capture ends in seconds. The kernel variant can be pinned with --tile, the
grid with --grid (0: the default, one block per tile; the benchmark's
tuner picks one block per tile for the FD stage).
"""
from __future__ import annotations

import argparse
import math


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("model", choices=["cs", "fd"])
    ap.add_argument("--n", type=int, default=0)
    ap.add_argument("--steps", type=int, default=0)
    ap.add_argument("--tile", type=int, default=-1)
    ap.add_argument("--q", type=int, default=4)
    ap.add_argument("--precision", default="fp32")
    ap.add_argument("--grid", type=int, default=0)
    ap.add_argument("--storage", default="ab", choices=["ab", "inplace"])
    a = ap.parse_args()

    import torch

    import lbm_workloads as wl
    import paper_1904_02471_gb300 as pkg
    torch.cuda.init()
    if a.model == "cs":
        n = a.n or 2048
        L = pkg.Lattice("cs", 3, n, n, 0.8 / math.sqrt(3), precision=a.precision, storage=a.storage)
        if a.tile >= 0:
            L.config(a.tile, a.grid)
        L.init(*wl.taylor_green(n, n, 0.01 * math.sqrt(3)))
        L.step(a.steps or 4)
    else:
        n = a.n or 1024
        L = pkg.Lattice("fd", a.q, n, n, 5e-4, dt=1e-5, precision=a.precision)
        if a.tile >= 0:
            L.config(a.tile, a.grid)
        L.init(*wl.taylor_green(n, n, 0.01))
        L.step(a.steps or 2)
    L.sync()
    print(a.model, n, "mass", L.observables()["mass"])


if __name__ == "__main__":
    main()
