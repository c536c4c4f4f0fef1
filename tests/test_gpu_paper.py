"""The paper's own experiments, run through the library on the GPU (FP64).

* Sec. 4.1 shock tube: rho_L = 1.1, rho_R = 0.9, N = 2048, tau_FD in
  {1e-4, 1e-3} (tau_LU from Eq. nu-transfer), profiles at t_FD = 0.1128:
  400 CS steps; FD with the 3-root set and the paper's time steps
  dt = 1/(N sqrt 3) (tau_FD = 1e-3, 400 steps) or 1/(3 N sqrt 3)
  (tau_FD = 1e-4, 1200 steps). Both are compared with the inviscid similarity
  solution (oracle) and with each other, and the plateau density with the
  printed rho_c ~ 0.995.
* Sec. 4.2-4.3 (Tables 1-2 set-up): apparent viscosity of CS and FD runs of
  the same system for N = 20..60; FD (3- and 4-node sets) converges at about
  fifth order, CS stays within its second-order error; at N = 20 the GPU's
  nu_app equals the oracle's on the same samples, and CS nu_app equals that
  of the exact linear (Fourier-space) evolution of the collide-stream
  operator.
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
    """Tables 1-2 set-up (nu_0 = tau_FD = 5e-4, FD dt = 5e-4): FD converges at
    about fifth order in N for the 3- and the 4-node set and reaches < 1e-4
    at N = 60; CS stays within its second-order error."""
    ns = (20, 30, 40, 50, 60)
    for kind in ("shear", "tg"):
        rows = vt.table(kind, ns=ns, qs=(3, 4), t_end=5.0)
        for q in (3, 4):
            fd_order = vt.order(rows, f"fd_q{q}_rel_err")
            assert fd_order > 4.0, (kind, q, fd_order, rows)
        assert rows[-1]["fd_q4_rel_err"] < 1e-4, rows[-1]
        for r in rows:
            assert r["cs_rel_err"] < 5e-2, r


def _oracle_series(model, kind, n, q, every, steps, nu0=5e-4, dt_fd=5e-4, U=0.01):
    (rho, ux, uy), (comp, px, py, norm) = vt._fields(kind, n, U)
    f = oracle.equilibrium(q if model == "fd" else 3, rho, ux, uy)
    # the library records the state of step s (s a multiple of every) while
    # it computes step s + 1: the states 0, every, ... before the last step
    a = []
    for s in range(0, steps, every):
        a.append(oracle.observables(f, comp, px, py, norm)[3])
        if s + every < steps:
            if model == "fd":
                f = oracle.fd_run(f, 1.0 / n, dt_fd, nu0, every)
            else:
                f = oracle.cs_run(f, pkg.lbm_tau_lu_from_fd(n, nu0), every)
    return np.array(a)


@pytest.mark.parametrize("kind", ["shear", "tg"])
@pytest.mark.parametrize("model,q", [("cs", 3), ("fd", 3), ("fd", 4)])
def test_nu_app_equals_the_oracles(kind, model, q):
    """N = 20 (the tables' first row), a short run: the GPU's recorded
    amplitudes and the oracle's at the same steps give the same nu_app to
    1e-10 relative (same samples, same fit)."""
    n, t_end = 20, 0.5
    t, a_gpu, every, steps = vt.run_series(model, kind, n, q=q, t_end=t_end)
    a_or = _oracle_series(model, kind, n, q, every, steps)
    assert a_or.shape == a_gpu.shape
    assert np.max(np.abs(a_gpu - a_or)) < 1e-12 * np.max(np.abs(a_or))
    nu_g = vt.fit_nu(kind, t, a_gpu, t_end)
    nu_o = vt.fit_nu(kind, t, a_or, t_end)
    assert abs(nu_g / nu_o - 1) < 1e-10, (nu_g, nu_o)


def test_cs_nu_app_equals_the_linear_prediction():
    """CS shear waves of the tables' set-up in the linear regime (U = 1e-4):
    nu_app from the GPU run equals nu_app from the exact Fourier-space
    evolution of the collide-stream operator diag(e^{-i kappa c_k})(I - omega
    (I - E)) on the same samples, to 1e-6 relative, for N = 20..60."""
    import oracle_pins as P
    s3 = math.sqrt(3)
    nodes = np.array([-s3, 0.0, s3])
    vx, vy = np.tile(nodes, 3), np.repeat(nodes, 3)
    w1 = np.array([1 / 6, 2 / 3, 1 / 6])
    w = np.tile(w1, 3) * np.repeat(w1, 3)
    cx = np.tile([-1, 0, 1], 3)
    U = 1e-4
    for n in (20, 30, 40, 50, 60):
        t_end = 1.0
        t, a_gpu, every, steps = vt.run_series("cs", "shear", n, t_end=t_end, U=U)
        omega = (1.0 / s3) / pkg.lbm_tau_lu_from_fd(n, 5e-4)
        M = np.diag(np.exp(-1j * (2 * math.pi / n) * cx)) @ (np.eye(9) - omega * (np.eye(9) - P._linear_E(vx, vy, w)))
        pred = P._shear_amplitude_linear(M, vx, vy, w, U, 0, steps)[::every][:len(a_gpu)]
        nu_g = vt.fit_nu("shear", t, a_gpu, t_end)
        nu_p = vt.fit_nu("shear", t, pred, t_end)
        assert abs(nu_g / nu_p - 1) < 1e-6, (n, nu_g, nu_p)
