"""The oracle's FD path against the FDLB columns printed in Tables 1-2.

Sec. 4.2 (shear waves, Table 1) and Sec. 4.3 (Taylor-Green vortices,
Table 2) print the relative error of the apparent viscosity of FD runs at
nu_0 = tau_FD = 5e-4, dt = 5e-4, N = 20..60 nodes per wavelength. The paper
states neither the velocity set of these runs nor the WENO-5 regulariser
epsilon; the reading that reproduces every printed FD error is the 3-node
(D2Q9) product set, the one whose largest speed sqrt(3) the CFL argument of
Sec. 4.1 uses, with epsilon = 1e-10. At N = 20 and 30 the printed errors come
from the nonlinear WENO weights (the linear weights give errors 5-10 times
smaller), so matching them pins the whole FD pipeline: equilibrium,
smoothness indicators and weights, SSP-RK3, BGK, the projected amplitude and
the decay fit. The same runs with the common epsilon = 1e-6, or with the
4-node set, miss the printed values by far more than their rounding.
"""
import json
import math
import os

import numpy as np
import pytest

import lbm_workloads as wl
import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")
NU0, DT, T_END, U = 5e-4, 5e-4, 1.0, 0.01


def _printed(kind):
    with open(GOLD) as fh:
        t = json.load(fh)["nu_app_tables"]
    cols = t["columns"]
    return {r[0]: r[cols.index("fd_rel_err")] for r in t[kind]}


def _rel_err(kind, n, q, eps, samples=50):
    """|nu_app / nu_0 - 1| of one FD run of the oracle: amplitude recorded
    `samples` times over t_end = 1, log-linear fit over t >= t_end / 10,
    nu_app = gamma / (m k^2), m = 1 (shear, Eq. shear_sol), 2 (Taylor-Green,
    Eq. taylor), k = 2 pi."""
    if kind == "shear":
        (rho, ux, uy), (comp, px, py, norm) = wl.shear_wave(n, n, U), wl.probe_shear(n, n)
    else:
        (rho, ux, uy), (comp, px, py, norm) = wl.taylor_green(n, n, U), wl.probe_taylor_green(n, n)
    f = oracle.equilibrium(q, rho, ux, uy)
    steps = int(round(T_END / DT))
    every = steps // samples
    t, a = [], []
    for s in range(0, steps, every):
        t.append(s * DT)
        a.append(oracle.observables(f, comp, px, py, norm)[3])
        f = oracle.fd_run(f, 1.0 / n, DT, NU0, every, eps=eps)
    gamma, _ = oracle.fit_decay(np.array(t), np.array(a), 0.1 * T_END)
    m = 1 if kind == "shear" else 2
    return abs(gamma / (m * (2 * math.pi) ** 2) / NU0 - 1)


@pytest.mark.parametrize("kind", ["shear", "tg"])
@pytest.mark.parametrize("n", [20, 30])
def test_fd_errors_equal_the_printed_columns(kind, n):
    """3-node set, epsilon = 1e-10: the printed error to within 1e-3
    absolute and 2% relative (the printed values have four decimals; the
    paper's fit window is not stated)."""
    got, want = _rel_err(kind, n, 3, 1e-10), _printed(kind)[n]
    assert abs(got - want) < 1e-3 and abs(got / want - 1) < 0.02, (kind, n, got, want)


@pytest.mark.parametrize("q,eps", [(3, 1e-6), (4, 1e-10)])
def test_other_readings_miss_the_printed_columns(q, eps):
    """The reading is decided by the printed values: the default epsilon of
    WENO-5 (1e-6) or the 4-node set miss the Table 1 N = 20 error by more than
    20%."""
    got, want = _rel_err("shear", 20, q, eps), _printed("shear")[20]
    assert abs(got / want - 1) > 0.2, (q, eps, got, want)
