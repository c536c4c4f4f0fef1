"""The paper's own experiments, run through the library on the GPU (FP64).

* Sec. 4.1 shock tube: rho_L = 1.1, rho_R = 0.9, N = 2048, tau_FD in
  {1e-4, 1e-3} (tau_LU from Eq. nu-transfer), profiles at t_FD = 0.1128:
  400 CS steps; FD with the 3-root set and the paper's time steps
  dt = 1/(N sqrt 3) (tau_FD = 1e-3, 400 steps) or 1/(3 N sqrt 3)
  (tau_FD = 1e-4, 1200 steps). Both are compared with the inviscid similarity
  solution (oracle) and with each other, and the plateau density with the
  printed rho_c ~ 0.995.
* Sec. 4.2-4.3 (Tables 1-2 set-up): apparent viscosity of CS and FD runs of
  the same system for N = 20..60; FD converges at about fifth order, CS stays
  within its second-order error.
"""
import math

import numpy as np
import pytest

import lbm_workloads as wl
import oracle
import paper_1904_02471_gb300 as pkg
from paper_1904_02471_gb300 import viscosity_tables as vt

pytestmark = pytest.mark.gpu

SQ3 = math.sqrt(3.0)
N = 2048
X0 = 1024


@pytest.fixture(scope="module", autouse=True)
def gpu():
    import torch
    assert torch.cuda.is_available()
    from paper_1904_02471_gb300 import build
    build.build()
    torch.cuda.init()


def _shock(model, tau_fd):
    rho, ux, uy = wl.shock_tube(N, 1, 1.1, 0.9, X0)
    if model == "cs":
        L = pkg.Lattice("cs", 3, N, 1, pkg.lbm_tau_lu_from_fd(N, tau_fd))
        steps = 400
        t_fd = steps / (N * SQ3)
    else:
        dt = 1.0 / (N * SQ3) if tau_fd >= 1e-3 else 1.0 / (3 * N * SQ3)
        L = pkg.Lattice("fd", 3, N, 1, tau_fd, dt=dt)
        steps = 400 if tau_fd >= 1e-3 else 1200
        t_fd = steps * dt
    with L:
        L.init(rho, ux, uy)
        L.step(steps)
        r, u, _ = L.moments()
    return r[0], u[0], t_fd


@pytest.mark.parametrize("tau_fd", [1e-4, 1e-3])
def test_shock_tube_against_similarity_solution(tau_fd):
    x = np.arange(N, dtype=float)
    win = np.abs(x - X0) < 400          # the waves from the periodic image stay outside
    res = {}
    for model in ("cs", "fd"):
        r, u, t = _shock(model, tau_fd)
        assert abs(t - 0.1128) < 2e-4
        xi = (x[win] - (X0 + 0.5)) / (t * N)  # FD units: x_FD = x / N
        r_ex, u_ex = oracle.shock_profile(xi, 1.1, 0.9)
        l1r, l1u = np.mean(np.abs(r[win] - r_ex)), np.mean(np.abs(u[win] - u_ex))
        # viscous smearing of the inviscid solution over a window of 800 nodes
        assert l1r < 1e-2 and l1u < 1e-2, (model, tau_fd, l1r, l1u)
        s = oracle.shock_solution(1.1, 0.9)
        plateau = (xi > s["xi_c"] + 0.15) & (xi < s["xi_s"] - 0.15)
        assert abs(np.mean(r[win][plateau]) - 0.995) < 2e-3, (model, np.mean(r[win][plateau]))
        res[model] = r
    # the two models simulate the same physical system (Sec. 3 mapping)
    assert np.mean(np.abs(res["cs"][win] - res["fd"][win])) < 5e-3


def test_viscosity_tables_orders():
    ns = (20, 30, 40, 50, 60)
    for kind in ("shear", "tg"):
        rows = vt.table(kind, ns=ns, q=4, t_end=5.0)
        fd_order = vt.order(rows, "fd_rel_err")
        assert fd_order > 4.0, (kind, fd_order, rows)
        assert rows[-1]["fd_rel_err"] < 1e-4, rows[-1]
        for r in rows:
            assert r["cs_rel_err"] < 5e-2, r
