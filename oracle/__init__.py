"""FP64 CPU oracle for the CS and FD isothermal lattice Boltzmann updates.

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package. The CUDA library shares no code with it.

The heavy loops live in ``lbm_oracle.c`` (plain C, FP64, no FMA contraction);
this module marshals numpy arrays into it and adds the host-side pieces of the
paper that are closed forms:

* unit conversion between the FD and CS ("LU") conventions, Sec. 3,
  Eq. (nu-transfer): tau_LU = N tau_FD + sqrt(3)/6;
* viscosities, Eq. (nulu) nu_LU = tau_LU - dt/2 and Eq. (nu_fd) nu_FD = tau_FD;
* the isothermal Riemann solution of Sec. 4.1 (zeta root, rarefaction fan,
  plateau, shock speed);
* the log-linear decay fit used to extract nu_app (Sec. 4.2, 4.3).

Array layout: f[k, y, x] (numpy C order), k = ix + n*iy over the ascending 1D
Gauss-Hermite nodes.

Pins: ``tests/test_oracle_*.py``. Nothing here is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

from . import build as _build

_LIBS: dict[int, ctypes.CDLL] = {}

_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)


def _lib(mutant: int = 0) -> ctypes.CDLL:
    if mutant not in _LIBS:
        path = _build.build(mutant)
        lib = ctypes.CDLL(path)
        i, d, i64 = ctypes.c_int, ctypes.c_double, ctypes.c_int64
        lib.or_hermite_rule.argtypes = [i, _D, _D]
        lib.or_velocity_set.argtypes = [i, _D, _D, _D]
        lib.or_feq_cell.argtypes = [i, _D, _D, _D, d, d, d, _D]
        lib.or_macro.argtypes = [i, i, i, _D, _D, _D, _D, _D, _D]
        lib.or_equilibrium.argtypes = [i, i, i, _D, _D, _D, _D, _D, _D, _D]
        lib.or_cs_step.argtypes = [i, i, i, _D, _D, _D, _I, _I, d, _D, _D]
        lib.or_cs_run.argtypes = [i, i, i, _D, _D, _D, _I, _I, d, i64, _D, _D]
        lib.or_lattice_vectors.argtypes = [i, _D, _D, d, d, _I, _I]
        lib.or_weno5_face.argtypes = [_D, d, _D]
        lib.or_weno5_face.restype = d
        lib.or_fd_rhs.argtypes = [i, i, i, _D, _D, _D, d, d, d, _D, _D]
        lib.or_fd_step.argtypes = [i, i, i, _D, _D, _D, d, d, d, d, _D, _D]
        lib.or_fd_run.argtypes = [i, i, i, _D, _D, _D, d, d, d, d, i64, _D, _D]
        lib.or_fd_imex_step.argtypes = [i, i, i, _D, _D, _D, d, d, d, d, _D, _D, _D]
        lib.or_fd_imex_run.argtypes = [i, i, i, _D, _D, _D, d, d, d, d, i64, _D, _D]
        lib.or_observables.argtypes = [i, i, i, _D, _D, _D, i, _D, _D, d, _D]
        _LIBS[mutant] = lib
    return _LIBS[mutant]


def _p(a: np.ndarray):
    assert a.flags.c_contiguous
    if a.dtype == np.float64:
        return a.ctypes.data_as(_D)
    if a.dtype == np.int32:
        return a.ctypes.data_as(_I)
    raise TypeError(a.dtype)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


# --------------------------------------------------------------------------
# Velocity sets (Sec. 1-2) and pointwise physics (Eqs. herfeq, f_moments_discrete)
# --------------------------------------------------------------------------

def hermite_rule(n: int, mutant: int = 0):
    """1D Gauss-Hermite rule (probabilists', weights summing to 1), ascending."""
    x = np.zeros(n)
    w = np.zeros(n)
    if _lib(mutant).or_hermite_rule(n, _p(x), _p(w)) != 0:
        raise ValueError(f"no rule for n={n}")
    return x, w


def velocity_set(n: int, mutant: int = 0):
    """Product set {v_k, w_k}, K = n^2, k = ix + n*iy. Returns (vx, vy, w)."""
    K = n * n
    vx, vy, w = np.zeros(K), np.zeros(K), np.zeros(K)
    if _lib(mutant).or_velocity_set(n, _p(vx), _p(vy), _p(w)) != 0:
        raise ValueError(f"no velocity set for n={n}")
    return vx, vy, w


def feq_cell(n: int, rho: float, ux: float, uy: float, mutant: int = 0) -> np.ndarray:
    vx, vy, w = velocity_set(n, mutant)
    out = np.zeros(n * n)
    _lib(mutant).or_feq_cell(n * n, _p(vx), _p(vy), _p(w), rho, ux, uy, _p(out))
    return out


def equilibrium(n: int, rho, ux, uy, mutant: int = 0) -> np.ndarray:
    """f = f^eq(rho, u) on a lattice; rho, ux, uy are [ny, nx]."""
    rho, ux, uy = _f64(rho), _f64(ux), _f64(uy)
    ny, nx = rho.shape
    vx, vy, w = velocity_set(n, mutant)
    f = np.zeros((n * n, ny, nx))
    _lib(mutant).or_equilibrium(nx, ny, n * n, _p(vx), _p(vy), _p(w), _p(rho), _p(ux), _p(uy), _p(f))
    return f


def macro(n: int, f, mutant: int = 0):
    """(rho, ux, uy) of a lattice f[k, y, x]."""
    f = _f64(f)
    K, ny, nx = f.shape
    vx, vy, _ = velocity_set(n, mutant)
    rho, ux, uy = np.zeros((ny, nx)), np.zeros((ny, nx)), np.zeros((ny, nx))
    _lib(mutant).or_macro(nx, ny, K, _p(vx), _p(vy), _p(f), _p(rho), _p(ux), _p(uy))
    return rho, ux, uy


# --------------------------------------------------------------------------
# CS model (Sec. 2, Eq. sc_evolution); D2Q9: dx = 1, dt = 1/sqrt(3)
# --------------------------------------------------------------------------

CS_DT = 1.0 / math.sqrt(3.0)


def lattice_vectors(n: int, dt: float = CS_DT, dx: float = 1.0, mutant: int = 0):
    vx, vy, _ = velocity_set(n, mutant)
    cx = np.zeros(n * n, dtype=np.int32)
    cy = np.zeros(n * n, dtype=np.int32)
    if _lib(mutant).or_lattice_vectors(n * n, _p(vx), _p(vy), dt, dx, _p(cx), _p(cy)) != 0:
        raise ValueError("velocity set is off-lattice for this dt/dx")
    return cx, cy


def cs_run(f, tau_lu: float, steps: int, dt: float = CS_DT, mutant: int = 0) -> np.ndarray:
    """`steps` CS updates of the pre-collision state f[k, y, x] (D2Q9)."""
    f = _f64(f).copy()
    K, ny, nx = f.shape
    n = int(round(math.sqrt(K)))
    vx, vy, w = velocity_set(n, mutant)
    cx, cy = lattice_vectors(n, dt, 1.0, mutant)
    tmp = np.empty_like(f)
    omega = dt / tau_lu
    _lib(mutant).or_cs_run(nx, ny, K, _p(vx), _p(vy), _p(w), _p(cx), _p(cy), omega, int(steps), _p(f), _p(tmp))
    return f


def cs_run_omega(f, omega: float, steps: int, mutant: int = 0) -> np.ndarray:
    """CS updates with the relaxation factor omega = dt/tau given directly."""
    f = _f64(f).copy()
    K, ny, nx = f.shape
    n = int(round(math.sqrt(K)))
    vx, vy, w = velocity_set(n, mutant)
    cx, cy = lattice_vectors(n, CS_DT, 1.0, mutant)
    tmp = np.empty_like(f)
    _lib(mutant).or_cs_run(nx, ny, K, _p(vx), _p(vy), _p(w), _p(cx), _p(cy), omega, int(steps), _p(f), _p(tmp))
    return f


# --------------------------------------------------------------------------
# FD model (Sec. 2): WENO-5 advection + SSP-RK3, BGK inside every stage
# --------------------------------------------------------------------------

WENO_EPS = 1e-6


def weno5_face(s, eps: float = WENO_EPS, mutant: int = 0):
    """Interface value from (f_{i-2}..f_{i+2}); returns (value, detail[9])."""
    s = _f64(s)
    d = np.zeros(9)
    v = _lib(mutant).or_weno5_face(_p(s), eps, _p(d))
    return v, d


def fd_rhs(f, dx: float, tau: float, eps: float = WENO_EPS, mutant: int = 0) -> np.ndarray:
    f = _f64(f)
    K, ny, nx = f.shape
    n = int(round(math.sqrt(K)))
    vx, vy, w = velocity_set(n, mutant)
    L = np.zeros_like(f)
    _lib(mutant).or_fd_rhs(nx, ny, K, _p(vx), _p(vy), _p(w), dx, tau, eps, _p(f), _p(L))
    return L


def fd_run(f, dx: float, dt: float, tau: float, steps: int, eps: float = WENO_EPS,
           mutant: int = 0) -> np.ndarray:
    """`steps` SSP-RK3 steps of f[k, y, x]."""
    f = _f64(f).copy()
    K, ny, nx = f.shape
    n = int(round(math.sqrt(K)))
    vx, vy, w = velocity_set(n, mutant)
    work = np.empty((3,) + f.shape)
    _lib(mutant).or_fd_run(nx, ny, K, _p(vx), _p(vy), _p(w), dx, dt, tau, eps, int(steps), _p(f), _p(work))
    return f


def fd_imex_run(f, dx: float, dt: float, tau: float, steps: int, eps: float = WENO_EPS,
                mutant: int = 0) -> np.ndarray:
    """`steps` IMEX-SSP2(2,2,2) steps of f[k, y, x] (explicit WENO-5 advection,
    implicit BGK; lifts dt < tau, Sec. 4.1)."""
    f = _f64(f).copy()
    K, ny, nx = f.shape
    n = int(round(math.sqrt(K)))
    vx, vy, w = velocity_set(n, mutant)
    work = np.empty((7,) + f.shape)
    _lib(mutant).or_fd_imex_run(nx, ny, K, _p(vx), _p(vy), _p(w), dx, dt, tau, eps, int(steps), _p(f), _p(work))
    return f


def fd_imex_stages(f, dx: float, dt: float, tau: float, eps: float = WENO_EPS, mutant: int = 0):
    """One IMEX step: returns (f^{n+1}, [Y_1, Y_2]) with the stage values."""
    f = _f64(f).copy()
    K, ny, nx = f.shape
    n = int(round(math.sqrt(K)))
    vx, vy, w = velocity_set(n, mutant)
    work = np.empty((7,) + f.shape)
    ys = np.empty((2,) + f.shape)
    _lib(mutant).or_fd_imex_step(nx, ny, K, _p(vx), _p(vy), _p(w), dx, dt, tau, eps, _p(f), _p(work), _p(ys))
    return f, [ys[0], ys[1]]


# --------------------------------------------------------------------------
# Diagnostics
# --------------------------------------------------------------------------

def observables(f, comp: int, px, py, norm: float, mutant: int = 0) -> np.ndarray:
    """[sum rho, sum rho ux, sum rho uy, A], A = norm * sum u_comp px[x] py[y]."""
    f = _f64(f)
    K, ny, nx = f.shape
    n = int(round(math.sqrt(K)))
    vx, vy, _ = velocity_set(n, mutant)
    out = np.zeros(4)
    _lib(mutant).or_observables(nx, ny, K, _p(vx), _p(vy), _p(f), comp, _p(_f64(px)), _p(_f64(py)), norm, _p(out))
    return out


def fit_decay(t, a, t_skip: float = 0.0):
    """Least-squares fit ln A = ln A0 - gamma t over t >= t_skip; returns (gamma, A0)."""
    t = np.asarray(t, dtype=np.float64)
    a = np.asarray(a, dtype=np.float64)
    m = t >= t_skip
    slope, icpt = np.polyfit(t[m], np.log(np.abs(a[m])), 1)
    return -slope, math.exp(icpt)


# --------------------------------------------------------------------------
# Units (Sec. 3) and viscosities (Eqs. nulu, nu_fd, nu-transfer)
# --------------------------------------------------------------------------

def nu_lu(tau_lu: float, dt_lu: float = CS_DT) -> float:
    """Eq. (nulu): nu_LU = tau_LU - dt_LU/2."""
    return tau_lu - dt_lu / 2.0


def nu_fd(tau_fd: float, T: float = 1.0, m: float = 1.0) -> float:
    """Eq. (nu_fd): nu_FD = tau_FD T / m."""
    return tau_fd * T / m


def tau_lu_from_fd(n_lu: int, tau_fd: float) -> float:
    """Eq. (nu-transfer): tau_LU = N_LU tau_FD + sqrt(3)/6."""
    return n_lu * tau_fd + math.sqrt(3.0) / 6.0


def tau_fd_from_lu(n_lu: int, tau_lu: float) -> float:
    return (tau_lu - math.sqrt(3.0) / 6.0) / n_lu


def dt_fd_of_cs_step(n_lu: int) -> float:
    """One CS step, dt_LU = 1/sqrt(3), in FD time units: t_ref;LU = t_ref;FD / N."""
    return CS_DT / n_lu


# --------------------------------------------------------------------------
# Isothermal Riemann problem (Sec. 4.1)
# --------------------------------------------------------------------------

def shock_zeta(rho_l: float, rho_r: float) -> float:
    """Smallest root zeta > 0 of g(z) = 2 + z^2 - (rL/rR) e^{-z} - (rR/rL) e^{z} = 0.

    g(0+) < 0 for rho_l != rho_r; the physical root is the first crossing to
    g > 0, bracketed by a geometric scan and refined by bisection."""
    def g(z):
        return 2.0 + z * z - (rho_l / rho_r) * math.exp(-z) - (rho_r / rho_l) * math.exp(z)
    if not rho_l > rho_r:
        raise ValueError("need rho_l > rho_r")
    lo, hi = 1e-14, 1e-6
    while g(hi) <= 0.0:
        lo, hi = hi, hi * 1.25
        if hi > 50.0:
            raise ValueError("no root found")
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if g(mid) > 0.0:
            hi = mid
        else:
            lo = mid
    return 0.5 * (lo + hi)


def shock_solution(rho_l: float, rho_r: float, cs: float = 1.0):
    """(zeta, xi_r, xi_c, u_c, rho_c, xi_s) of the isothermal Riemann problem.

    Rarefaction head xi_r = -cs; plateau u_c = zeta cs, rho_c = rho_L e^{-zeta};
    tail xi_c = cs (zeta - 1); shock speed xi_s = zeta cs / (1 - (rR/rL) e^{zeta}).
    """
    z = shock_zeta(rho_l, rho_r)
    return {
        "zeta": z,
        "xi_r": -cs,
        "xi_c": cs * (z - 1.0),
        "u_c": z * cs,
        "rho_c": rho_l * math.exp(-z),
        "xi_s": z * cs / (1.0 - (rho_r / rho_l) * math.exp(z)),
    }


def shock_profile(xi, rho_l: float, rho_r: float, cs: float = 1.0):
    """Density and velocity at similarity variable xi = (x - x0)/t.

    In the fan u* = xi + cs and rho* = rho_L exp(-u*/cs) (the isothermal
    Riemann invariant; the first form printed in Eq. (shock_rhostar) has a sign
    slip, the second form is used)."""
    s = shock_solution(rho_l, rho_r, cs)
    xi = np.asarray(xi, dtype=np.float64)
    rho = np.where(xi < s["xi_r"], rho_l, 0.0)
    u = np.zeros_like(xi)
    fan = (xi >= s["xi_r"]) & (xi < s["xi_c"])
    u = np.where(fan, xi + cs, u)
    rho = np.where(fan, rho_l * np.exp(-(xi + cs) / cs), rho)
    plat = (xi >= s["xi_c"]) & (xi < s["xi_s"])
    u = np.where(plat, s["u_c"], u)
    rho = np.where(plat, s["rho_c"], rho)
    right = xi >= s["xi_s"]
    rho = np.where(right, rho_r, rho)
    return rho, u
