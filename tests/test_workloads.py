"""The seeded synthetic inputs (lbm_workloads): the paper's initial
conditions and the batched and served workload lists, on the CPU.

They hold no arithmetic of the method; these tests pin the recipe they
state: field formulas, probe normalisation (a projection of the initial
field returns its amplitude), the distributions of the batched and served
workloads, and that a served stream's arrival rate only rescales its
arrival times (the full served-stream benchmark relies on that).
"""
import math

import numpy as np

import lbm_workloads as wl


def test_initial_fields():
    nx, ny, U = 24, 16, 0.03
    rho, ux, uy = wl.shear_wave(nx, ny, U)
    x = np.arange(nx)
    assert np.all(rho == 1.0) and np.all(ux == 0.0)
    assert np.allclose(uy, U * np.sin(2 * math.pi * x / nx)[None, :], rtol=0, atol=1e-15)

    rho, ux, uy = wl.taylor_green(nx, ny, U)
    kx = 2 * math.pi * np.arange(nx)[None, :] / nx
    ky = 2 * math.pi * np.arange(ny)[:, None] / ny
    assert np.allclose(ux, U * np.sin(kx) * np.cos(ky), atol=1e-15)
    assert np.allclose(uy, -U * np.cos(kx) * np.sin(ky), atol=1e-15)
    # steady pressure balance with cs = 1: p = rho, grad p = -rho0 (u . grad) u
    assert np.allclose(rho, 1 + U * U / 4 * (np.cos(2 * kx) + np.cos(2 * ky)), atol=1e-15)
    # on a square lattice (square cells, one wavelength per axis) the velocity
    # field is divergence free: spectral derivative of its single Fourier modes
    n = 20
    _, ux, uy = wl.taylor_green(n, n, U)
    k = 2j * math.pi * np.fft.fftfreq(n)
    div = np.fft.ifft2(k[None, :] * np.fft.fft2(ux) + k[:, None] * np.fft.fft2(uy)).real
    assert np.max(np.abs(div)) < 1e-14
    # and the density is the steady pressure balance grad p = -rho0 (u . grad) u,
    # p = cs^2 rho with cs = 1 (paper units)
    rho, ux, uy = wl.taylor_green(n, n, U)

    def d(f, axis):
        kk = k[None, :] if axis == 1 else k[:, None]
        return np.fft.ifft2(kk * np.fft.fft2(f)).real

    for p_grad, u_comp in ((d(rho, 1), ux), (d(rho, 0), uy)):
        conv = ux * d(u_comp, 1) + uy * d(u_comp, 0)
        assert np.max(np.abs(p_grad + conv)) < 1e-15

    rho, ux, uy = wl.shock_tube(16, 4, 1.5, 0.75, 7)
    assert np.all(rho[:, :8] == 1.5) and np.all(rho[:, 8:] == 0.75)   # rho_L where x_i <= x0
    assert not ux.any() and not uy.any()


def test_probes_return_the_initial_amplitude():
    nx, ny, U = 32, 12, 0.02
    for fields, probe, comp_field in ((wl.shear_wave, wl.probe_shear, 2), (wl.taylor_green, wl.probe_taylor_green, 1)):
        f = fields(nx, ny, U)
        comp, px, py, norm = probe(nx, ny)
        u = f[1 + comp]
        assert 1 + comp == comp_field
        assert abs(norm * np.sum(u * px[None, :] * py[:, None]) - U) < 1e-15


def test_batched_workload_recipe():
    a = wl.batched_instances(256, seed=0)
    assert a == wl.batched_instances(256, seed=0)                    # seeded
    assert len(a) == 256
    assert [d["model"] for d in a] == ["cs", "fd"] * 128
    assert all(d["n"] in (32, 64, 128, 256, 512) for d in a)
    assert all(0.51 <= d["tau_star"] <= 2.0 for d in a)
    cs = [d for d in a if d["model"] == "cs"]
    assert [d["init"] for d in cs] == ["shear", "tg"] * 64
    assert all(d["init"] == "tg" and d["q"] == 4 for d in a if d["model"] == "fd")
    sides = {s: sum(d["n"] == s for d in a) for s in (32, 64, 128, 256, 512)}
    assert min(sides.values()) >= 30                                # every side drawn often


def test_served_stream_recipe():
    s = wl.served_stream(400, seed=0, rate_per_s=2.0)
    t = np.array([r["arrival"] for r in s])
    assert np.all(np.diff(t) > 0)
    assert abs(np.mean(np.diff(t)) - 0.5) < 0.1                     # Poisson, mean gap 1/rate
    assert all(r["n"] in (64, 128, 256, 512, 1024, 2048, 4096) for r in s)
    assert all(1000 <= r["steps"] <= 20000 for r in s)
    frac_cs = np.mean([r["model"] == "cs" for r in s])
    assert 0.4 < frac_cs < 0.6
    # the rate only rescales the arrival times: same runs, in the same order
    s2 = wl.served_stream(400, seed=0, rate_per_s=0.5)
    for r, r2 in zip(s, s2):
        assert (r["model"], r["n"], r["steps"], r["tau_star"]) == (r2["model"], r2["n"], r2["steps"], r2["tau_star"])
        assert abs(r2["arrival"] - 4 * r["arrival"]) < 1e-9 * max(1.0, r2["arrival"])
