"""Seeded synthetic inputs for the CS and FD lattice Boltzmann runs.

This module holds initial fields and workload lists only: no moments, no
equilibria, no updates. Both the oracle side and the CUDA side of the tests
(and bench.py) take their inputs from here, so the two never share any of the
method's arithmetic.

Conventions: fields are numpy float64 arrays of shape [ny, nx] (x fastest);
node coordinates are x_i = i * dx with dx = 1 (CS, lattice units) or dx = 1/N
(FD, unit domain), so that CS and FD nodes coincide one by one.

Initial conditions follow the paper's experiments:
* shear wave, Sec. 4.2: rho = rho0, u_x = 0, u_y = U sin(k x), k = 2 pi / L;
* Taylor-Green vortex, Sec. 4.3, Eq. (tg): u_x = U sin(kx) cos(ky),
  u_y = -U cos(kx) sin(ky); the paper does not give rho, so it is taken from
  the steady pressure balance p = p0 + rho0 U^2/4 (cos 2kx + cos 2ky) with
  p = rho cs^2 (isothermal, cs = 1 in the paper's units);
* shock tube, Sec. 4.1: rho = rho_L for x_i <= x0, rho_R otherwise, u = 0.
"""
from __future__ import annotations

import math

import numpy as np


def _grid(nx: int, ny: int):
    x = np.arange(nx, dtype=np.float64)[None, :].repeat(ny, 0)
    y = np.arange(ny, dtype=np.float64)[:, None].repeat(nx, 1)
    return x, y


def shear_wave(nx: int, ny: int, U: float, rho0: float = 1.0):
    """u_y = U sin(2 pi x / nx): one wavelength across the lattice."""
    x, _ = _grid(nx, ny)
    rho = np.full((ny, nx), rho0)
    ux = np.zeros((ny, nx))
    uy = U * np.sin(2.0 * math.pi * x / nx)
    return rho, ux, uy


def taylor_green(nx: int, ny: int, U: float, rho0: float = 1.0, cs2: float = 1.0):
    """Taylor-Green vortex with one wavelength across each axis (square cells)."""
    x, y = _grid(nx, ny)
    kx = 2.0 * math.pi * x / nx
    ky = 2.0 * math.pi * y / ny
    ux = U * np.sin(kx) * np.cos(ky)
    uy = -U * np.cos(kx) * np.sin(ky)
    rho = rho0 * (1.0 + U * U / (4.0 * cs2) * (np.cos(2.0 * kx) + np.cos(2.0 * ky)))
    return rho, ux, uy


def shock_tube(nx: int, ny: int, rho_l: float, rho_r: float, x0: int):
    """Density step at node x0 (rho_L where x_i <= x0), fluid at rest."""
    x, _ = _grid(nx, ny)
    rho = np.where(x <= x0, rho_l, rho_r).astype(np.float64)
    return rho, np.zeros((ny, nx)), np.zeros((ny, nx))


def random_smooth(nx: int, ny: int, seed: int, amp_rho: float = 0.05, amp_u: float = 0.05,
                  modes: int = 3, rho0: float = 1.0):
    """Smooth random periodic fields: a few low Fourier modes with seeded phases."""
    rng = np.random.default_rng(seed)
    x, y = _grid(nx, ny)
    out = []
    for amp in (amp_rho, amp_u, amp_u):
        fld = np.zeros((ny, nx))
        for _ in range(modes):
            mx, my = rng.integers(0, 3, size=2)
            ph = rng.uniform(0, 2 * math.pi)
            a = rng.uniform(-1, 1)
            fld += a * np.sin(2 * math.pi * (mx * x / nx + my * y / ny) + ph)
        out.append(amp * fld / modes)
    rho = rho0 + out[0]
    return rho, out[1], out[2]


def random_uniform(shape, seed: int, lo: float, hi: float) -> np.ndarray:
    """Seeded uniform random array (used to perturb arbitrary states)."""
    return np.random.default_rng(seed).uniform(lo, hi, size=shape)


def probe_shear(nx: int, ny: int):
    """Projection onto the shear mode: A = (2/(nx ny)) sum u_y sin(kx)."""
    px = np.sin(2.0 * math.pi * np.arange(nx) / nx)
    py = np.ones(ny)
    return 1, px, py, 2.0 / (nx * ny)


def probe_taylor_green(nx: int, ny: int):
    """Projection onto the TG mode: A = (4/(nx ny)) sum u_x sin(kx) cos(ky)."""
    px = np.sin(2.0 * math.pi * np.arange(nx) / nx)
    py = np.cos(2.0 * math.pi * np.arange(ny) / ny)
    return 0, px, py, 4.0 / (nx * ny)


# --------------------------------------------------------------------------
# Named workloads, stated in the paper's units (T = m = 1, cs = 1).
# A tau given "in lattice units" (dt = 1, cs^2 = 1/3) is tau_LU * sqrt(3);
# a lattice-unit velocity is the paper-unit velocity / sqrt(3).
# --------------------------------------------------------------------------

SQRT3 = math.sqrt(3.0)

# CS D2Q9 shear-wave damping on a periodic 64x4 lattice, tau* = 0.8 (lattice
# units), u_y = 0.01 sin(2 pi x/64) (lattice units), 2000 steps.
CS_SHEAR_64x4 = dict(model="cs", q=3, nx=64, ny=4, tau=0.8 / SQRT3, U=0.01 * SQRT3, steps=2000,
                     init="shear")

# FD Taylor-Green, 16-velocity Gauss-Hermite set (4 roots per axis), periodic
# 256x256 unit domain, U = 0.01, nu_FD = tau_FD = 5e-4, dt_FD = 5e-4, 5000 steps.
FD_TG_256 = dict(model="fd", q=4, nx=256, ny=256, tau=5e-4, dt=5e-4, U=0.01, steps=5000, init="tg")

# Single large lattices for the bandwidth roofline: CS D2Q9 8192^2 and FD
# 16-velocity 4096^2, FP32 deviation storage, Taylor-Green initial state.
CS_ROOFLINE = dict(model="cs", q=3, nx=8192, ny=8192, tau=0.8 / SQRT3, U=0.01 * SQRT3, init="tg")
FD_ROOFLINE = dict(model="fd", q=4, nx=4096, ny=4096, tau=5e-4, dt=1e-5, U=0.01, init="tg")


def batched_instances(n: int = 256, seed: int = 0, sizes=(32, 64, 128, 256, 512)):
    """The batched workload: n independent square lattices.

    Side uniform over `sizes`, tau* uniform in [0.51, 2.0] (lattice units),
    even entries CS D2Q9, odd entries FD 16-velocity; CS runs alternate shear
    wave / Taylor-Green initial states, FD runs are Taylor-Green.
    Returns dicts with model, q, n, tau_star, init.
    """
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        side = int(rng.choice(sizes))
        tau_star = float(rng.uniform(0.51, 2.0))
        if i % 2 == 0:
            out.append(dict(model="cs", q=3, n=side, tau_star=tau_star,
                            init="shear" if (i // 2) % 2 == 0 else "tg"))
        else:
            out.append(dict(model="fd", q=4, n=side, tau_star=tau_star, init="tg"))
    return out


def served_stream(n: int, seed: int, rate_per_s: float, sides=(64, 128, 256, 512, 1024, 2048, 4096),
                  steps=(1000, 20000)):
    """Poisson arrivals of Taylor-Green runs: (arrival_s, model, side, steps, tau_star).

    Side log-uniform over powers of two, steps uniform in [steps[0], steps[1]],
    CS or FD with probability 1/2, tau* uniform in [0.51, 2.0].
    """
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for _ in range(n):
        t += float(rng.exponential(1.0 / rate_per_s))
        out.append(dict(arrival=t, model="cs" if rng.random() < 0.5 else "fd",
                        n=int(rng.choice(sides)), steps=int(rng.integers(steps[0], steps[1] + 1)),
                        tau_star=float(rng.uniform(0.51, 2.0))))
    return out
