"""Pins for the FP64 oracle: each check ties one part of the oracle to something
other than the oracle itself (a library routine, a closed form, an invariant,
a number printed in the paper, or an independent Fourier-space analysis).

Every check takes ``mutant``: 0 checks the oracle as built; m > 0 runs the same
check against a build of the oracle with a planted mistake (see OR_MUTANT in
oracle/lbm_oracle.c). tests/test_oracle_pins.py runs them all on the real
oracle, tests/test_oracle_mutants.py shows each planted mistake is caught.
"""
from __future__ import annotations

import json
import math
import os

import numpy as np

import oracle
import lbm_workloads as wl

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as fh:
        return json.load(fh)


def _double_factorial(m):
    r = 1
    while m > 1:
        r *= m
        m -= 2
    return r


def _gauss_moment(a):
    """E[v^a] for v ~ N(0, 1): 0 for odd a, (a-1)!! for even a."""
    return 0.0 if a % 2 else float(_double_factorial(a - 1))


# --------------------------------------------------------------------------
# Velocity sets (Sec. 1-2)
# --------------------------------------------------------------------------

def check_rule_vs_numpy(mutant=0):
    """1D rule equals numpy's Gauss-HermiteE rule (weights normalised to 1)."""
    from numpy.polynomial.hermite_e import hermegauss
    for n in range(2, 9):
        x, w = oracle.hermite_rule(n, mutant)
        xr, wr = hermegauss(n)
        wr = wr / wr.sum()
        assert np.allclose(x, xr, rtol=0, atol=1e-13), (n, x, xr)
        assert np.allclose(w, wr, rtol=1e-13, atol=0), (n, w, wr)


def check_rule_closed_forms(mutant=0):
    """Closed-form nodes and weights for 3, 4 and 5 nodes."""
    s3, s6, s10 = math.sqrt(3), math.sqrt(6), math.sqrt(10)
    cases = {
        3: ([-s3, 0.0, s3], [1 / 6, 2 / 3, 1 / 6]),
        4: ([-math.sqrt(3 + s6), -math.sqrt(3 - s6), math.sqrt(3 - s6), math.sqrt(3 + s6)],
            [(3 - s6) / 12, (3 + s6) / 12, (3 + s6) / 12, (3 - s6) / 12]),
        5: ([-math.sqrt(5 + s10), -math.sqrt(5 - s10), 0.0, math.sqrt(5 - s10), math.sqrt(5 + s10)],
            [(7 - 2 * s10) / 60, (7 + 2 * s10) / 60, 8 / 15, (7 + 2 * s10) / 60, (7 - 2 * s10) / 60]),
    }
    for n, (xe, we) in cases.items():
        x, w = oracle.hermite_rule(n, mutant)
        assert np.allclose(x, xe, rtol=0, atol=1e-14), (n, x)
        assert np.allclose(w, we, rtol=1e-14, atol=0), (n, w)


def check_set_moments(mutant=0):
    """sum_k w_k vx^a vy^b = E[v^a] E[v^b] for all a, b <= 2n-1 (product Gauss rule)."""
    for n in (3, 4, 5):
        vx, vy, w = oracle.velocity_set(n, mutant)
        for a in range(2 * n):
            for b in range(2 * n):
                terms = w * vx ** a * vy ** b
                got = float(np.sum(terms))
                exp = _gauss_moment(a) * _gauss_moment(b)
                scale = max(1.0, float(np.sum(np.abs(terms))))
                assert abs(got - exp) <= 1e-14 * scale, (n, a, b, got, exp)


def check_set_ordering(mutant=0):
    """Population order k = ix + n*iy over ascending nodes (the documented layout)."""
    s3 = math.sqrt(3)
    nodes = [-s3, 0.0, s3]
    vx, vy, w = oracle.velocity_set(3, mutant)
    for k in range(9):
        assert abs(vx[k] - nodes[k % 3]) < 1e-14 and abs(vy[k] - nodes[k // 3]) < 1e-14, (k, vx[k], vy[k])


# --------------------------------------------------------------------------
# Equilibrium and moments (Eqs. herfeq, f_moments_discrete)
# --------------------------------------------------------------------------

def check_feq_moments(mutant=0):
    """Hermite moments of f^eq: rho, rho u, rho(delta + uu), and the third and
    fourth moments of a second-order expansion (isothermal, cs^2 = T/m = 1)."""
    rng = np.random.default_rng(7)
    for n in (3, 4, 5):
        vx, vy, _ = oracle.velocity_set(n, mutant)
        for _ in range(5):
            rho = rng.uniform(0.5, 1.5)
            u = rng.uniform(-0.3, 0.3, size=2)
            f = oracle.feq_cell(n, rho, u[0], u[1], mutant)
            v = np.stack([vx, vy])
            tol = 1e-13
            assert abs(f.sum() - rho) < tol
            assert np.allclose(v @ f, rho * u, atol=tol)
            P = np.einsum("ak,bk,k->ab", v, v, f)
            assert np.allclose(P, rho * (np.eye(2) + np.outer(u, u)), atol=tol)
            # third moment: rho (u_a d_bc + u_b d_ac + u_c d_ab)
            Q3 = np.einsum("ak,bk,ck,k->abc", v, v, v, f)
            d = np.eye(2)
            E3 = rho * (np.einsum("a,bc->abc", u, d) + np.einsum("b,ac->abc", u, d) + np.einsum("c,ab->abc", u, d))
            assert np.allclose(Q3, E3, atol=tol)
            if n >= 4:
                m4 = float(np.sum(f * vx ** 4))
                assert abs(m4 - rho * (3.0 + 6.0 * u[0] ** 2)) < tol


def check_macro_of_equilibrium(mutant=0):
    rho, ux, uy = wl.random_smooth(7, 5, seed=3, amp_rho=0.2, amp_u=0.2)
    for n in (3, 4, 5):
        f = oracle.equilibrium(n, rho, ux, uy, mutant)
        r2, ux2, uy2 = oracle.macro(n, f, mutant)
        assert np.allclose(r2, rho, atol=1e-14) and np.allclose(ux2, ux, atol=1e-14)
        assert np.allclose(uy2, uy, atol=1e-14)


# --------------------------------------------------------------------------
# CS update (Eq. sc_evolution)
# --------------------------------------------------------------------------

def check_cs_fixed_point(mutant=0):
    """A uniform equilibrium is a fixed point of collide + stream."""
    rho = np.full((5, 6), 1.1)
    ux = np.full((5, 6), 0.05)
    uy = np.full((5, 6), -0.03)
    f0 = oracle.equilibrium(3, rho, ux, uy, mutant)
    f = oracle.cs_run(f0, 0.7, 20, mutant=mutant)
    assert np.max(np.abs(f - f0)) < 1e-14


def check_cs_streaming_direction(mutant=0):
    """With omega = 0 a value in population k moves from x to x + c_k, where
    c_k = (ix - 1, iy - 1) for the D2Q9 nodes (-sqrt3, 0, sqrt3)."""
    nx, ny = 7, 5
    for k in range(9):
        f = np.ones((9, ny, nx))
        f[k, 2, 3] = 2.0
        g = oracle.cs_run_omega(f, 0.0, 1, mutant)
        cx, cy = k % 3 - 1, k // 3 - 1
        exp = np.ones_like(f)
        exp[k, (2 + cy) % ny, (3 + cx) % nx] = 2.0
        assert np.array_equal(g, exp), k


def check_cs_periodic_return(mutant=0):
    """Pure streaming (omega = 0) on an 8x6 lattice returns exactly after 24 steps."""
    f = wl.random_uniform((9, 6, 8), seed=5, lo=0.0, hi=1.0)
    g = oracle.cs_run_omega(f, 0.0, 24, mutant)
    assert np.array_equal(f, g)
    h = oracle.cs_run_omega(f, 0.0, 1, mutant)
    assert not np.array_equal(f, h)


def check_cs_omega_one(mutant=0):
    """omega = 1: f_k(x + c_k, t + 1) = f^eq_k(x, t)."""
    rho, ux, uy = wl.random_smooth(6, 5, seed=11, amp_rho=0.1, amp_u=0.1)
    feq = oracle.equilibrium(3, rho, ux, uy, mutant)
    f0 = feq + wl.random_uniform(feq.shape, seed=12, lo=-0.01, hi=0.01)
    r0, u0x, u0y = oracle.macro(3, f0, mutant)
    feq0 = oracle.equilibrium(3, r0, u0x, u0y, mutant)
    f1 = oracle.cs_run_omega(f0, 1.0, 1, mutant)
    for k in range(9):
        cx, cy = k % 3 - 1, k // 3 - 1
        exp = np.roll(np.roll(feq0[k], cy, axis=0), cx, axis=1)
        assert np.allclose(f1[k], exp, atol=1e-15), k


def check_cs_conservation(mutant=0):
    """Total mass and momentum are invariants of the CS update."""
    rho, ux, uy = wl.random_smooth(16, 12, seed=21, amp_rho=0.1, amp_u=0.1)
    f = oracle.equilibrium(3, rho, ux, uy, mutant)
    f = f + wl.random_uniform(f.shape, seed=22, lo=-1e-3, hi=1e-3)
    px, py = np.ones(16), np.ones(12)
    o0 = oracle.observables(f, 0, px, py, 1.0, mutant)
    g = oracle.cs_run(f, 0.61, 100, mutant=mutant)
    o1 = oracle.observables(g, 0, px, py, 1.0, mutant)
    assert abs(o1[0] - o0[0]) < 1e-13 * abs(o0[0])
    assert abs(o1[1] - o0[1]) < 1e-13 * abs(o0[0]) and abs(o1[2] - o0[2]) < 1e-13 * abs(o0[0])


def _linear_E(vx, vy, w):
    """Linearised equilibrium about rho = 1, u = 0: d feq_k = w_k (d rho + v_k . d j)."""
    return w[:, None] * (1.0 + np.outer(vx, vx) + np.outer(vy, vy))


def _shear_amplitude_linear(step_matrix, vx, vy, w, U, axis, steps):
    """Exact linear evolution of the e^{i kappa x} component of a shear wave.

    axis 0: u_y = U sin(kappa x); axis 1: u_x = U sin(kappa y). The initial
    equilibrium's kappa component is w_k v_k,c U / (2i) (c the velocity
    component carrying the wave); A(t) = -2 Im(sum_k v_k,c c_k(t))."""
    vc = vy if axis == 0 else vx
    c = (w * vc * U / 2j).astype(complex)
    out = []
    for _ in range(steps + 1):
        out.append(-2.0 * np.imag(np.sum(vc * c)))
        c = step_matrix @ c
    return np.array(out)


def _cs_exact_rational(f, omega, steps):
    """Brute-force D2Q9 collide + stream in exact rational arithmetic, lattice
    units (c in {-1, 0, 1}, w = (2/3, 1/6, 1/6) per axis, cs^2 = 1/3):
    f_k(x + c_k, t + 1) = f_k - omega (f_k - w_k rho (1 + 3 c.u + 9/2 (c.u)^2 - 3/2 u^2)).
    Written out here, independently of the oracle."""
    from fractions import Fraction as Fr
    K, ny, nx = len(f), len(f[0]), len(f[0][0])
    w1 = {-1: Fr(1, 6), 0: Fr(2, 3), 1: Fr(1, 6)}
    cs = [(k % 3 - 1, k // 3 - 1) for k in range(9)]
    for _ in range(steps):
        new = [[[None] * nx for _ in range(ny)] for _ in range(K)]
        for y in range(ny):
            for x in range(nx):
                fk = [f[k][y][x] for k in range(9)]
                rho = sum(fk)
                ux = sum(fk[k] * cs[k][0] for k in range(9)) / rho
                uy = sum(fk[k] * cs[k][1] for k in range(9)) / rho
                usq = ux * ux + uy * uy
                for k, (cx, cy) in enumerate(cs):
                    cu = cx * ux + cy * uy
                    feq = w1[cx] * w1[cy] * rho * (1 + 3 * cu + Fr(9, 2) * cu * cu - Fr(3, 2) * usq)
                    new[k][(y + cy) % ny][(x + cx) % nx] = fk[k] - omega * (fk[k] - feq)
        f = new
    return f


def check_cs_exact_rational(mutant=0):
    """In lattice units with a rational omega the CS update is a rational map;
    the oracle (paper units: v = sqrt3 c, u = sqrt3 u_lattice, the same
    populations) agrees with the exact result to rounding after 3 steps on a
    7x5 lattice, and the exact result conserves mass exactly."""
    from fractions import Fraction as Fr
    nx, ny, omega = 7, 5, Fr(3, 4)
    rho = [[1 + Fr((3 * x + 5 * y) % 7 - 3, 50) for x in range(nx)] for y in range(ny)]
    ul = [[Fr((x + 2 * y) % 5 - 2, 100) for x in range(nx)] for y in range(ny)]
    vl = [[Fr((3 * x + y) % 5 - 2, 100) for x in range(nx)] for y in range(ny)]
    w1 = {-1: Fr(1, 6), 0: Fr(2, 3), 1: Fr(1, 6)}
    f0 = []
    for k in range(9):
        cx, cy = k % 3 - 1, k // 3 - 1
        plane = []
        for y in range(ny):
            row = []
            for x in range(nx):
                cu = cx * ul[y][x] + cy * vl[y][x]
                usq = ul[y][x] ** 2 + vl[y][x] ** 2
                row.append(w1[cx] * w1[cy] * rho[y][x] * (1 + 3 * cu + Fr(9, 2) * cu * cu - Fr(3, 2) * usq))
            plane.append(row)
        f0.append(plane)
    fe = _cs_exact_rational(f0, omega, 3)
    assert sum(v for p in fe for r in p for v in r) == sum(v for p in f0 for r in p for v in r)
    sq3 = math.sqrt(3.0)
    r = np.array([[float(v) for v in row] for row in rho])
    u = sq3 * np.array([[float(v) for v in row] for row in ul])
    v = sq3 * np.array([[float(q) for q in row] for row in vl])
    fo = oracle.cs_run_omega(oracle.equilibrium(3, r, u, v, mutant), float(omega), 3, mutant)
    exact = np.array([[[float(q) for q in row] for row in p] for p in fe])
    assert np.max(np.abs(fo - exact)) < 2e-15 * np.max(np.abs(exact)), np.max(np.abs(fo - exact))


def check_cs_linear_modes(mutant=0):
    """Shear-wave amplitude A(t) of the oracle equals the exact linear prediction
    from the Fourier-space collide-stream matrix diag(e^{-i kappa.c_k})(I - omega(I - E))
    to 1e-7 relative over 120 steps (U = 1e-4: nonlinear terms enter at O(U^2)
    relative, since the quadratic terms do not project onto the kappa mode)."""
    s3 = math.sqrt(3)
    nodes = np.array([-s3, 0.0, s3])
    vx = np.tile(nodes, 3)
    vy = np.repeat(nodes, 3)
    w1 = np.array([1 / 6, 2 / 3, 1 / 6])
    w = np.tile(w1, 3) * np.repeat(w1, 3)
    cxv = np.tile([-1, 0, 1], 3)
    cyv = np.repeat([-1, 0, 1], 3)
    U = 1e-4
    for axis, (nx, ny) in ((0, (24, 3)), (1, (3, 20))):
        tau_lu = 0.37
        omega = (1.0 / s3) / tau_lu
        kappa = 2 * math.pi / (nx if axis == 0 else ny)
        kc = cxv if axis == 0 else cyv
        M = np.diag(np.exp(-1j * kappa * kc)) @ (np.eye(9) - omega * (np.eye(9) - _linear_E(vx, vy, w)))
        steps = 120
        pred = _shear_amplitude_linear(M, vx, vy, w, U, axis, steps)
        if axis == 0:
            rho, ux, uy = wl.shear_wave(nx, ny, U)
            comp, px, py, norm = wl.probe_shear(nx, ny)
        else:
            rho, uy, ux = (a.T.copy() for a in wl.shear_wave(ny, nx, U))
            comp, px, py, norm = 0, np.ones(nx), np.sin(2 * math.pi * np.arange(ny) / ny), 2.0 / (nx * ny)
        f = oracle.equilibrium(3, rho, ux, uy, mutant)
        got = []
        for t in range(steps + 1):
            got.append(oracle.observables(f, comp, px, py, norm, mutant)[3])
            f = oracle.cs_run(f, tau_lu, 1, mutant=mutant)
        got = np.array(got)
        rel = np.max(np.abs(got - pred)) / U
        assert rel < 1e-7, (axis, rel)


def check_cs_decay_closed_form(mutant=0):
    """64x4 shear wave, tau* = 0.8 (lattice units), 2000 steps: nu_app from a
    log-linear fit matches nu* = (tau* - 1/2)/3, i.e. Eq. (nulu)
    nu_LU = tau_LU - dt/2 = sqrt(3) nu*, within the O(k^2) discretisation error."""
    c = wl.CS_SHEAR_64x4
    nx, ny = c["nx"], c["ny"]
    rho, ux, uy = wl.shear_wave(nx, ny, c["U"])
    comp, px, py, norm = wl.probe_shear(nx, ny)
    f = oracle.equilibrium(3, rho, ux, uy, mutant)
    ts, amps = [], []
    every = 100
    for s in range(0, c["steps"] + 1, every):
        ts.append(s)
        amps.append(oracle.observables(f, comp, px, py, norm, mutant)[3])
        if s < c["steps"]:
            f = oracle.cs_run(f, c["tau"], every, mutant=mutant)
    gamma, _ = oracle.fit_decay(np.array(ts, float), np.array(amps), t_skip=200)
    k = 2 * math.pi / nx
    nu_app = gamma / k ** 2  # lattice units per step
    nu_star = (0.8 - 0.5) / 3.0
    assert abs(nu_app / nu_star - 1.0) < 2e-3, nu_app / nu_star - 1.0
    # A(2000)/A(0) against exp(-nu* k^2 t) = 0.1455
    assert abs(amps[-1] / amps[0] - math.exp(-nu_star * k * k * c["steps"])) < 2e-3


# --------------------------------------------------------------------------
# WENO-5 (Jiang & Shu), the FD advection of Sec. 2
# --------------------------------------------------------------------------

def _cell_averages(coef, centers):
    """Cell averages over [j - 1/2, j + 1/2] of the polynomial sum coef[p] x^p."""
    P = np.polynomial.Polynomial(coef).integ()
    return np.array([P(j + 0.5) - P(j - 0.5) for j in centers])


def check_weno_quadratic_exact(mutant=0):
    """Every candidate is exact for quadratics, so the face value equals h(1/2)
    for cell averages of any quadratic h, whatever the weights."""
    rng = np.random.default_rng(31)
    for _ in range(20):
        coef = rng.uniform(-1, 1, size=3) * np.array([1.0, 0.3, 0.1])
        s = _cell_averages(coef, [-2, -1, 0, 1, 2])
        v, d = oracle.weno5_face(s, 1e-6, mutant)
        h = np.polynomial.Polynomial(coef)(0.5)
        assert abs(v - h) < 1e-13, (v, h)
        assert np.allclose(d[0:3], h, atol=1e-13)


def check_weno_beta(mutant=0):
    """Smoothness indicators equal the Jiang-Shu integral
    beta_r = int_{cell i} (p_r')^2 + (p_r'')^2 dx (dx = 1), p_r the quadratic with
    the cell averages of stencil r, for cell averages of random cubics."""
    rng = np.random.default_rng(33)
    for _ in range(20):
        coef = rng.uniform(-1, 1, size=4) * np.array([1.0, 0.5, 0.2, 0.1])
        s = _cell_averages(coef, [-2, -1, 0, 1, 2])
        _, d = oracle.weno5_face(s, 1e-6, mutant)
        for r in range(3):
            cells = [-2 + r, -1 + r, r]
            A = np.array([[(((j + 0.5) ** (p + 1)) - ((j - 0.5) ** (p + 1))) / (p + 1) for p in range(3)]
                          for j in cells])
            pc = np.linalg.solve(A, s[r:r + 3])
            p = np.polynomial.Polynomial(pc)
            integrand = p.deriv() ** 2 + p.deriv(2) ** 2
            I = integrand.integ()
            beta = I(0.5) - I(-0.5)
            assert abs(d[3 + r] - beta) < 1e-12 * max(1.0, beta), (r, d[3 + r], beta)


def check_weno_linear_weights(mutant=0):
    """With eps >> beta (1e30) the weights are the linear ones, which make the 5-point
    reconstruction exact for quartics: face value = h(1/2)."""
    rng = np.random.default_rng(35)
    for _ in range(20):
        coef = rng.uniform(-1, 1, size=5) * np.array([1.0, 0.5, 0.2, 0.1, 0.05])
        s = _cell_averages(coef, [-2, -1, 0, 1, 2])
        v, d = oracle.weno5_face(s, 1e30, mutant)
        assert np.allclose(d[6:9], [0.1, 0.6, 0.3], rtol=1e-12, atol=0)
        h = np.polynomial.Polynomial(coef)(0.5)
        assert abs(v - h) < 1e-13, (v, h)


def check_weno_eno(mutant=0):
    """Across a jump the weight moves to the smooth stencil (ENO property)."""
    v, d = oracle.weno5_face([0.0, 0.0, 0.0, 1.0, 1.0], 1e-6, mutant)
    assert d[6] > 1 - 1e-9 and abs(v) < 1e-9
    v, d = oracle.weno5_face([0.0, 0.0, 1.0, 1.0, 1.0], 1e-6, mutant)
    assert d[8] > 1 - 1e-9 and abs(v - 1.0) < 1e-9


def _d5(f, axis, positive):
    """Fifth-order upwind-biased first derivative (h = 1), textbook 6-point form."""
    def sh(m):  # f_{j+m}
        return np.roll(f, -m, axis=axis)
    if positive:
        return (-2 * sh(-3) + 15 * sh(-2) - 60 * sh(-1) + 20 * sh(0) + 30 * sh(1) - 3 * sh(2)) / 60.0
    return (2 * sh(3) - 15 * sh(2) + 60 * sh(1) - 20 * sh(0) - 30 * sh(-1) + 3 * sh(-2)) / 60.0


def check_fd_linear_advection(mutant=0):
    """With linear weights (eps huge) and no collision (tau huge), the FD right-hand
    side is -v_x D5_x f - v_y D5_y f, D5 upwinded by the sign of each component."""
    for n in (4, 5):
        K = n * n
        vx, vy, _ = oracle.velocity_set(n, mutant)
        f = wl.random_uniform((K, 10, 12), seed=40 + n, lo=0.0, hi=1.0)
        dx = 0.125
        L = oracle.fd_rhs(f, dx, 1e300, 1e30, mutant)
        s3, s6, s10 = math.sqrt(3), math.sqrt(6), math.sqrt(10)
        nodes = {4: [-math.sqrt(3 + s6), -math.sqrt(3 - s6), math.sqrt(3 - s6), math.sqrt(3 + s6)],
                 5: [-math.sqrt(5 + s10), -math.sqrt(5 - s10), 0.0, math.sqrt(5 - s10), math.sqrt(5 + s10)]}[n]
        for k in range(K):
            ax, ay = nodes[k % n], nodes[k // n]
            exp = np.zeros((10, 12))
            if ax != 0.0:
                exp -= ax * _d5(f[k], 1, ax > 0) / dx
            if ay != 0.0:
                exp -= ay * _d5(f[k], 0, ay > 0) / dx
            assert np.allclose(L[k], exp, rtol=0, atol=1e-11 * max(1.0, np.abs(exp).max())), (n, k)


def check_fd_rk3_relaxation(mutant=0):
    """Spatially uniform state: f - f^eq is multiplied per step by the SSP-RK3
    stability polynomial R(z) = 1 + z + z^2/2 + z^3/6, z = -dt/tau."""
    for n in (4, 5):
        K = n * n
        feq = oracle.feq_cell(n, 1.05, 0.02, -0.03, mutant)
        pert = wl.random_uniform(K, seed=50 + n, lo=-1e-3, hi=1e-3)
        f0 = np.repeat(np.repeat((feq + pert)[:, None, None], 4, 1), 5, 2).copy()
        r, ux, uy = oracle.macro(n, f0, mutant)
        fe = oracle.equilibrium(n, r, ux, uy, mutant)
        dt, tau = 3e-4, 5e-4
        f1 = oracle.fd_run(f0, 0.1, dt, tau, 1, 1e-6, mutant)
        z = -dt / tau
        R = 1 + z + z * z / 2 + z ** 3 / 6
        assert np.allclose(f1 - fe, R * (f0 - fe), rtol=0, atol=1e-15), n


def check_fd_conservation(mutant=0):
    """Conservative flux form + mass/momentum-conserving BGK: totals are invariant."""
    for n in (4, 5):
        rho, ux, uy = wl.random_smooth(16, 12, seed=60 + n, amp_rho=0.1, amp_u=0.1)
        f = oracle.equilibrium(n, rho, ux, uy, mutant)
        f = f + wl.random_uniform(f.shape, seed=70 + n, lo=-1e-4, hi=1e-4)
        px, py = np.ones(16), np.ones(12)
        o0 = oracle.observables(f, 0, px, py, 1.0, mutant)
        g = oracle.fd_run(f, 1 / 16, 5e-3, 1e-2, 30, 1e-6, mutant)
        o1 = oracle.observables(g, 0, px, py, 1.0, mutant)
        assert abs(o1[0] - o0[0]) < 1e-13 * abs(o0[0])
        assert abs(o1[1] - o0[1]) < 1e-13 * abs(o0[0]) and abs(o1[2] - o0[2]) < 1e-13 * abs(o0[0])


def check_fd_fixed_point(mutant=0):
    for n in (4, 5):
        rho = np.full((6, 7), 0.9)
        f0 = oracle.equilibrium(n, rho, np.full((6, 7), -0.04), np.full((6, 7), 0.07), mutant)
        f = oracle.fd_run(f0, 1 / 7, 1e-2, 2e-2, 10, 1e-6, mutant)
        assert np.max(np.abs(f - f0)) < 1e-14


def check_fd_linear_modes(mutant=0):
    """FD shear-wave amplitude equals the exact linear prediction from the
    Fourier-space operator: symbol of D5 for each upwind direction, linearised
    BGK, and the RK3 polynomial G = I + dtL + (dtL)^2/2 + (dtL)^3/6 (eps huge so
    the WENO weights are the linear ones), for the 3-, 4- and 5-node sets."""
    U = 1e-4
    for n in (3, 4, 5):
        K = n * n
        s3, s6, s10 = math.sqrt(3), math.sqrt(6), math.sqrt(10)
        nodes = {3: [-s3, 0.0, s3],
                 4: [-math.sqrt(3 + s6), -math.sqrt(3 - s6), math.sqrt(3 - s6), math.sqrt(3 + s6)],
                 5: [-math.sqrt(5 + s10), -math.sqrt(5 - s10), 0.0, math.sqrt(5 - s10), math.sqrt(5 + s10)]}[n]
        w1 = {3: [1 / 6, 2 / 3, 1 / 6],
              4: [(3 - s6) / 12, (3 + s6) / 12, (3 + s6) / 12, (3 - s6) / 12],
              5: [(7 - 2 * s10) / 60, (7 + 2 * s10) / 60, 8 / 15, (7 + 2 * s10) / 60, (7 - 2 * s10) / 60]}[n]
        vx = np.tile(nodes, n)
        vy = np.repeat(nodes, n)
        w = np.tile(w1, n) * np.repeat(w1, n)
        nx, ny = 16, 2
        dx = 1.0 / nx
        dt, tau = 2e-3, 4e-3
        th = 2 * math.pi / nx
        m = np.arange(-3, 4)
        ap = np.array([-2, 15, -60, 20, 30, -3, 0]) / 60.0      # coefficients of f_{j+m}, v > 0
        an = -ap[::-1]                                           # v < 0
        sym_p = np.sum(ap * np.exp(1j * th * m)) / dx
        sym_n = np.sum(an * np.exp(1j * th * m)) / dx
        adv = np.array([vx[k] * (sym_p if vx[k] > 0 else sym_n) if vx[k] != 0 else 0.0 for k in range(K)])
        Lh = -np.diag(adv) - (np.eye(K) - _linear_E(vx, vy, w)) / tau
        A = dt * Lh
        G = np.eye(K) + A + A @ A / 2 + A @ A @ A / 6
        steps = 60
        pred = _shear_amplitude_linear(G, vx, vy, w, U, 0, steps)
        rho, ux, uy = wl.shear_wave(nx, ny, U)
        comp, px, py, norm = wl.probe_shear(nx, ny)
        f = oracle.equilibrium(n, rho, ux, uy, mutant)
        got = []
        for _ in range(steps + 1):
            got.append(oracle.observables(f, comp, px, py, norm, mutant)[3])
            f = oracle.fd_run(f, dx, dt, tau, 1, 1e30, mutant)
        rel = np.max(np.abs(np.array(got) - pred)) / U
        assert rel < 1e-7, (n, rel)


def _fd_mp_ops(nodes, weights, nx, ny, dx, tau, eps, mp):
    """The FD right-hand side in mpmath, written out from the definitions:
    Jiang-Shu WENO-5 interface values upwinded by the sign of each velocity
    component (v = 0: no advection) in conservative flux differences (A), and
    BGK with the moments of the state it acts on (C). Periodic."""
    n = len(nodes)
    K = n * n
    v = [(nodes[k % n], nodes[k // n]) for k in range(K)]
    w = [weights[k % n] * weights[k // n] for k in range(K)]

    def face(a, b, c, d, e):   # value at i+1/2 from f_{i-2..i+2}, upwind side left
        q = [(2 * a - 7 * b + 11 * c) / 6, (-b + 5 * c + 2 * d) / 6, (2 * c + 5 * d - e) / 6]
        beta = [mp.mpf(13) / 12 * (a - 2 * b + c) ** 2 + (a - 4 * b + 3 * c) ** 2 / 4,
                mp.mpf(13) / 12 * (b - 2 * c + d) ** 2 + (b - d) ** 2 / 4,
                mp.mpf(13) / 12 * (c - 2 * d + e) ** 2 + (3 * c - 4 * d + e) ** 2 / 4]
        alpha = [dr / (eps + bt) ** 2 for dr, bt in zip((mp.mpf(1) / 10, mp.mpf(6) / 10, mp.mpf(3) / 10), beta)]
        return sum(al * qq for al, qq in zip(alpha, q)) / sum(alpha)

    def line_flux_diff(g, vel):   # (F_{i+1/2} - F_{i-1/2}) along a periodic line
        m = len(g)
        F = []
        for i in range(m):   # F[i] = value at face i - 1/2
            if vel > 0:
                F.append(face(*[g[(i - 3 + s) % m] for s in range(5)]))
            else:
                F.append(face(*[g[(i + 2 - s) % m] for s in range(5)]))
        return [F[(i + 1) % m] - F[i] for i in range(m)]

    def A(g):
        out = [[[mp.mpf(0)] * nx for _ in range(ny)] for _ in range(K)]
        for k in range(K):
            if v[k][0] != 0:
                for y in range(ny):
                    d = line_flux_diff(g[k][y], v[k][0])
                    for x in range(nx):
                        out[k][y][x] -= v[k][0] * d[x] / dx
            if v[k][1] != 0:
                for x in range(nx):
                    d = line_flux_diff([g[k][y][x] for y in range(ny)], v[k][1])
                    for y in range(ny):
                        out[k][y][x] -= v[k][1] * d[y] / dx
        return out

    def feq(g):
        out = [[[mp.mpf(0)] * nx for _ in range(ny)] for _ in range(K)]
        for y in range(ny):
            for x in range(nx):
                rho = sum(g[k][y][x] for k in range(K))
                ux = sum(g[k][y][x] * v[k][0] for k in range(K)) / rho
                uy = sum(g[k][y][x] * v[k][1] for k in range(K)) / rho
                usq = ux * ux + uy * uy
                for k in range(K):
                    xi = v[k][0] * ux + v[k][1] * uy
                    out[k][y][x] = w[k] * rho * (1 + xi + xi * xi / 2 - usq / 2)
        return out

    def C(g):
        e = feq(g)
        return [[[-(g[k][y][x] - e[k][y][x]) / tau for x in range(nx)] for y in range(ny)] for k in range(K)]

    def axpy(a, x, b, y):
        return [[[a * x[k][j][i] + b * y[k][j][i] for i in range(nx)] for j in range(ny)] for k in range(K)]

    return A, C, feq, axpy


def _fd_mp_run(f, nodes, weights, dx, dt, tau, eps, steps, mp):
    """Brute-force FD update in mpmath (_fd_mp_ops), SSP-RK3 in Shu-Osher form."""
    K, ny, nx = len(f), len(f[0]), len(f[0][0])
    A, C, _, axpy = _fd_mp_ops(nodes, weights, nx, ny, dx, tau, eps, mp)

    def L(g):
        return axpy(1, A(g), 1, C(g))

    for _ in range(steps):
        f1 = axpy(1, f, dt, L(f))
        f2 = axpy(mp.mpf(3) / 4, f, mp.mpf(1) / 4, axpy(1, f1, dt, L(f1)))
        f = axpy(mp.mpf(1) / 3, f, mp.mpf(2) / 3, axpy(1, f2, dt, L(f2)))
    return f


def check_fd_high_precision(mutant=0):
    """The oracle's FD step against a 30-digit mpmath brute force written from
    the definitions: 16 velocities with the closed-form Gauss-Hermite nodes
    +-sqrt(3 -+ sqrt 6), weights (3 +- sqrt 6)/12 (2 steps), and 25 velocities
    with nodes 0, +-sqrt(5 -+ sqrt 10), weights 8/15, (7 +- 2 sqrt 10)/60 (one
    step; its zero components do not advect); 6x6 lattice, a rough state so
    that the nonlinear WENO weights are far from linear."""
    import mpmath as mp
    mp.mp.dps = 30
    s6, s10 = mp.sqrt(6), mp.sqrt(10)
    sets = {4: ([-mp.sqrt(3 + s6), -mp.sqrt(3 - s6), mp.sqrt(3 - s6), mp.sqrt(3 + s6)],
                [(3 - s6) / 12, (3 + s6) / 12, (3 + s6) / 12, (3 - s6) / 12], 2),
            5: ([-mp.sqrt(5 + s10), -mp.sqrt(5 - s10), mp.mpf(0), mp.sqrt(5 - s10), mp.sqrt(5 + s10)],
                [(7 - 2 * s10) / 60, (7 + 2 * s10) / 60, mp.mpf(8) / 15, (7 + 2 * s10) / 60, (7 - 2 * s10) / 60], 1)}
    nx = ny = 6
    for n, (nodes, weights, steps) in sets.items():
        K = n * n
        rho, ux, uy = wl.random_smooth(nx, ny, seed=31, amp_rho=0.2, amp_u=0.1)
        f0 = oracle.equilibrium(n, rho, ux, uy, mutant)
        f0 = f0 * (1 + wl.random_uniform(f0.shape, seed=32, lo=-0.2, hi=0.2))
        dx, dt, tau, eps = 1.0 / nx, 0.02, 0.05, 1e-6
        fm = [[[mp.mpf(float(f0[k, y, x])) for x in range(nx)] for y in range(ny)] for k in range(K)]
        fm = _fd_mp_run(fm, nodes, weights, mp.mpf(dx), mp.mpf(dt), mp.mpf(tau), mp.mpf(eps), steps, mp)
        exact = np.array([[[float(fm[k][y][x]) for x in range(nx)] for y in range(ny)] for k in range(K)])
        fo = oracle.fd_run(f0, dx, dt, tau, steps, eps=eps, mutant=mutant)
        err = np.max(np.abs(fo - exact)) / np.max(np.abs(exact))
        assert err < 1e-13, (n, err)


# ---------------------------------------------------------------- FD, IMEX
# IMEX-SSP2(2,2,2) (Pareschi and Russo 2005): explicit and implicit tableaux.
IMEX_G = 1.0 - 1.0 / math.sqrt(2.0)
IMEX_AE = np.array([[0.0, 0.0], [1.0, 0.0]])
IMEX_AI = np.array([[IMEX_G, 0.0], [1.0 - 2.0 * IMEX_G, IMEX_G]])
IMEX_BE = np.array([0.5, 0.5])
IMEX_BI = np.array([0.5, 0.5])


def _imex_linear_step_matrix(Ah, Ch, dt):
    """One IMEX Runge-Kutta step of the linear system y' = Ah y + Ch y (Ah
    explicit, Ch implicit), built from the tableaux by generic linear solves:
    (I - dt a_ii Ch) Y_i = y + dt sum_{j<i} (a~_ij Ah + a_ij Ch) Y_j,
    y' = y + dt sum_i (b~_i Ah + b_i Ch) Y_i. Returns the matrix y -> y'."""
    K = Ah.shape[0]
    I = np.eye(K, dtype=complex)
    Ys = []
    for i in range(2):
        rhs = I.copy()
        for j in range(i):
            rhs = rhs + dt * (IMEX_AE[i, j] * Ah + IMEX_AI[i, j] * Ch) @ Ys[j]
        Ys.append(np.linalg.solve(I - dt * IMEX_AI[i, i] * Ch, rhs))
    G = I.copy()
    for i in range(2):
        G = G + dt * (IMEX_BE[i] * Ah + IMEX_BI[i] * Ch) @ Ys[i]
    return G


def check_imex_relaxation(mutant=0):
    """Spatially uniform state (no advection): f - f^eq is multiplied per step
    by the implicit tableau's stability function R(z) = 1 + z b^T (I - z A)^-1 1,
    z = -dt/tau (second order: R = e^z + O(z^3); L-stable: R(-inf) = 0), for
    non-stiff and stiff dt/tau. The scheme's update f + dt sum b_i C(Y_i)
    evaluates C(Y) = -(Y - f^eq)/tau by cancellation, so its rounding grows
    with dt/tau: the tolerance does too."""
    one = np.ones(2)
    for n in (4, 5):
        K = n * n
        feq = oracle.feq_cell(n, 1.05, 0.02, -0.03, mutant)
        pert = wl.random_uniform(K, seed=150 + n, lo=-1e-3, hi=1e-3)
        f0 = np.repeat(np.repeat((feq + pert)[:, None, None], 4, 1), 5, 2).copy()
        r, ux, uy = oracle.macro(n, f0, mutant)
        fe = oracle.equilibrium(n, r, ux, uy, mutant)
        for ratio in (0.5, 5.0, 50.0):
            tau = 1e-3
            dt = ratio * tau
            z = -ratio
            R = 1 + z * IMEX_BI @ np.linalg.solve(np.eye(2) - z * IMEX_AI, one)
            f1 = oracle.fd_imex_run(f0, 0.1, dt, tau, 1, 1e-6, mutant)
            assert np.allclose(f1 - fe, R * (f0 - fe), rtol=0, atol=1e-15 * (1 + ratio)), (n, ratio)
    # the tableau itself: second order in z, L-stable
    for z in (-1e-3, -2e-3):
        R = 1 + z * IMEX_BI @ np.linalg.solve(np.eye(2) - z * IMEX_AI, one)
        assert abs(R - math.exp(z)) < 0.1 * abs(z) ** 3
    assert abs(1 - IMEX_BI @ np.linalg.solve(IMEX_AI, one)) < 1e-15


def check_imex_stiff_limit(mutant=0):
    """tau -> 0: the first stage relaxes to the equilibrium of f^n in one
    stage, every stage keeps the moments of its explicit part (the collision
    conserves rho and rho u), and the step stays finite."""
    n = 4
    rho, ux, uy = wl.random_smooth(8, 6, seed=160, amp_rho=0.1, amp_u=0.1)
    f0 = oracle.equilibrium(n, rho, ux, uy, mutant)
    f0 = f0 * (1 + wl.random_uniform(f0.shape, seed=161, lo=-0.05, hi=0.05))
    r, u, v = oracle.macro(n, f0, mutant)
    fe = oracle.equilibrium(n, r, u, v, mutant)
    dt = 1e-2
    f1, (y1, y2) = oracle.fd_imex_stages(f0, 1 / 8, dt, 1e-14 * dt, 1e-6, mutant)
    assert np.max(np.abs(y1 - fe)) < 1e-12 * np.max(np.abs(fe))
    assert np.all(np.isfinite(f1))
    # moments of Y_1 = moments of f^n (Z_1 = f^n)
    m0 = oracle.macro(n, f0, mutant)
    m1 = oracle.macro(n, y1, mutant)
    for a, b in zip(m0, m1):
        assert np.max(np.abs(a - b)) < 1e-12


def check_imex_linear_modes(mutant=0):
    """IMEX shear-wave amplitude equals the exact linear prediction: the
    symbol of the linear-weight WENO-5 (D5) for each upwind direction as the
    explicit operator, the linearised BGK as the implicit one, and the step
    matrix built from the two tableaux by generic linear solves
    (_imex_linear_step_matrix), for the 3-, 4- and 5-node sets, at dt/tau = 0.5
    and at dt/tau = 5 (stiff for the explicit scheme)."""
    U = 1e-4
    for n in (3, 4, 5):
        K = n * n
        vx, vy, w = oracle.velocity_set(n)
        nx, ny = 16, 2
        dx = 1.0 / nx
        th = 2 * math.pi / nx
        m = np.arange(-3, 4)
        ap = np.array([-2, 15, -60, 20, 30, -3, 0]) / 60.0
        an = -ap[::-1]
        sym_p = np.sum(ap * np.exp(1j * th * m)) / dx
        sym_n = np.sum(an * np.exp(1j * th * m)) / dx
        adv = np.array([vx[k] * (sym_p if vx[k] > 0 else sym_n) if vx[k] != 0 else 0.0 for k in range(K)])
        for dt, tau in ((2e-3, 4e-3), (5e-3, 1e-3)):
            G = _imex_linear_step_matrix(-np.diag(adv), -(np.eye(K) - _linear_E(vx, vy, w)) / tau, dt)
            steps = 40
            pred = _shear_amplitude_linear(G, vx, vy, w, U, 0, steps)
            rho, ux, uy = wl.shear_wave(nx, ny, U)
            comp, px, py, norm = wl.probe_shear(nx, ny)
            f = oracle.equilibrium(n, rho, ux, uy, mutant)
            got = []
            for _ in range(steps + 1):
                got.append(oracle.observables(f, comp, px, py, norm, mutant)[3])
                f = oracle.fd_imex_run(f, dx, dt, tau, 1, 1e30, mutant)
            rel = np.max(np.abs(np.array(got) - pred)) / U
            assert rel < 1e-7, (n, dt / tau, rel)


def check_imex_conservation(mutant=0):
    """Mass and momentum are invariant under IMEX steps at dt = 10 tau (to the
    rounding of the scheme's update, which grows with dt/tau: see
    check_imex_relaxation)."""
    n = 4
    rho, ux, uy = wl.random_smooth(16, 12, seed=170, amp_rho=0.1, amp_u=0.1)
    f = oracle.equilibrium(n, rho, ux, uy, mutant)
    f = f + wl.random_uniform(f.shape, seed=171, lo=-1e-4, hi=1e-4)
    px, py = np.ones(16), np.ones(12)
    o0 = oracle.observables(f, 0, px, py, 1.0, mutant)
    g = oracle.fd_imex_run(f, 1 / 16, 5e-3, 5e-4, 30, 1e-6, mutant)
    o1 = oracle.observables(g, 0, px, py, 1.0, mutant)
    assert abs(o1[0] - o0[0]) < 1e-12 * abs(o0[0])
    assert abs(o1[1] - o0[1]) < 1e-13 * abs(o0[0]) and abs(o1[2] - o0[2]) < 1e-13 * abs(o0[0])


def check_imex_high_precision(mutant=0):
    """The oracle's IMEX step against a 30-digit mpmath brute force written
    from the scheme's definitions (_fd_mp_ops), whose implicit stage equations
    Y = Z + dt a_ii C(Y) are solved by iterating Y <- (Z + lam f^eq(Y)) / (1 + lam)
    to convergence (no use of the collision's conservation); 16 velocities,
    6x6 rough state, two steps at dt = 5 tau."""
    import mpmath as mp
    mp.mp.dps = 30
    s6 = mp.sqrt(6)
    nodes = [-mp.sqrt(3 + s6), -mp.sqrt(3 - s6), mp.sqrt(3 - s6), mp.sqrt(3 + s6)]
    weights = [(3 - s6) / 12, (3 + s6) / 12, (3 + s6) / 12, (3 - s6) / 12]
    n, nx, ny = 4, 6, 6
    K = n * n
    rho, ux, uy = wl.random_smooth(nx, ny, seed=181, amp_rho=0.2, amp_u=0.1)
    f0 = oracle.equilibrium(n, rho, ux, uy, mutant)
    f0 = f0 * (1 + wl.random_uniform(f0.shape, seed=182, lo=-0.2, hi=0.2))
    dx, dt, tau, eps = 1.0 / nx, 0.02, 0.004, 1e-6
    A, C, feq, axpy = _fd_mp_ops(nodes, weights, nx, ny, mp.mpf(dx), mp.mpf(tau), mp.mpf(eps), mp)
    g = mp.mpf(1) - 1 / mp.sqrt(2)
    ae = [[0, 0], [1, 0]]
    ai = [[g, 0], [1 - 2 * g, g]]
    half = mp.mpf(1) / 2
    f = [[[mp.mpf(float(f0[k, y, x])) for x in range(nx)] for y in range(ny)] for k in range(K)]
    mdt = mp.mpf(dt)
    for _ in range(2):
        As, Cs = [], []
        for i in range(2):
            Z = f
            for j in range(i):
                Z = axpy(1, Z, mdt * ae[i][j], As[j])
                Z = axpy(1, Z, mdt * ai[i][j], Cs[j])
            lam = mdt * ai[i][i] / mp.mpf(tau)
            Y = Z
            for _ in range(200):   # contraction with ratio lam / (1 + lam)
                Y = axpy(1 / (1 + lam), Z, lam / (1 + lam), feq(Y))
            As.append(A(Y))
            Cs.append(C(Y))
        for i in range(2):
            f = axpy(1, f, mdt * half, As[i])
            f = axpy(1, f, mdt * half, Cs[i])
    exact = np.array([[[float(f[k][y][x]) for x in range(nx)] for y in range(ny)] for k in range(K)])
    fo = oracle.fd_imex_run(f0, dx, dt, tau, 2, eps=eps, mutant=mutant)
    err = np.max(np.abs(fo - exact)) / np.max(np.abs(exact))
    assert err < 1e-13, err


def check_fd_decay_closed_form(mutant=0):
    """FD Taylor-Green, 16 velocities, 32^2 unit domain, nu = tau_FD = 0.01
    (Eq. nu_fd): the fitted decay matches exp(-2 k^2 nu t) of Eq. (taylor)."""
    nx = 32
    tau, dt = 0.01, 2.5e-3
    rho, ux, uy = wl.taylor_green(nx, nx, 0.01)
    comp, px, py, norm = wl.probe_taylor_green(nx, nx)
    f = oracle.equilibrium(4, rho, ux, uy, mutant)
    ts, amps = [], []
    every = 40
    for s in range(0, 400 + 1, every):
        ts.append(s * dt)
        amps.append(oracle.observables(f, comp, px, py, norm, mutant)[3])
        if s < 400:
            f = oracle.fd_run(f, 1.0 / nx, dt, tau, every, 1e-6, mutant)
    gamma, _ = oracle.fit_decay(np.array(ts), np.array(amps), t_skip=0.1)
    k = 2 * math.pi
    nu_app = gamma / (2 * k * k)
    assert abs(nu_app / tau - 1.0) < 1e-2, nu_app / tau - 1.0


# --------------------------------------------------------------------------
# Units (Sec. 3) and the shock problem (Sec. 4.1): printed values
# --------------------------------------------------------------------------

def _trunc(x, digits):
    s = 10 ** digits
    return math.floor(x * s + 1e-9) / s


def check_units_tables(mutant=0):
    g = _golden("paper_values.json")
    t = g["tau_lu_tables"]
    for n, printed in t["rows"]:
        assert abs(_trunc(oracle.tau_lu_from_fd(n, t["tau_fd"]), t["digits"]) - printed) < 1e-12, n
        # the round trip and Eq. (nulu): nu_LU = N nu_FD
        tl = oracle.tau_lu_from_fd(n, t["tau_fd"])
        assert abs(oracle.tau_fd_from_lu(n, tl) - t["tau_fd"]) < 1e-15
        assert abs(oracle.nu_lu(tl) - n * oracle.nu_fd(t["tau_fd"])) < 1e-14
    s = g["tau_lu_shock"]
    for tau_fd, printed, digits in s["rows"]:
        assert abs(_trunc(oracle.tau_lu_from_fd(s["n"], tau_fd), digits) - printed) < 1e-12


def check_units_time_steps(mutant=0):
    g = _golden("paper_values.json")
    d = g["dt_fd_shock"]
    dt = oracle.dt_fd_of_cs_step(d["n"])
    assert abs(dt / d["dt_cs_in_fd"] - 1) < d["rel_tol"]
    assert abs(dt / 3 / d["dt_fd_small"] - 1) < d["rel_tol"]
    assert abs(d["cs_iters"] * dt / d["t_fd"] - 1) < d["rel_tol"]
    s = g["dt_fd_shear"]
    for n in (20, 30, 40, 50, 60):
        assert abs(oracle.dt_fd_of_cs_step(n) / (s["base"] * s["factor"] / n) - 1) < s["rel_tol"]


def check_shock_worked_example(mutant=0):
    g = _golden("paper_values.json")["shock_worked_example"]
    sol = oracle.shock_solution(g["rho_l"], g["rho_r"])
    for key in ("zeta", "xi_r", "xi_c", "u_c", "rho_c", "xi_s"):
        val, digits = g[key]
        assert abs(sol[key] - val) <= 10.0 ** (-digits) + 1e-15, (key, sol[key], val)


def check_shock_jump_conditions(mutant=0):
    """Plateau and shock satisfy the Rankine-Hugoniot conditions Eq. (shock_rh)
    with P = rho cs^2, and the fan joins the plateau continuously."""
    for rl, rr in ((1.1, 0.9), (1.5, 0.75), (3.0, 1.0)):
        s = oracle.shock_solution(rl, rr)
        rc, uc, xs = s["rho_c"], s["u_c"], s["xi_s"]
        mass = rr * (0 - xs) - rc * (uc - xs)
        mom = (rr * 0 * (0 - xs) + rr) - (rc * uc * (uc - xs) + rc)
        assert abs(mass) < 1e-12 and abs(mom) < 1e-12, (rl, rr, mass, mom)
        rho_fan, u_fan = oracle.shock_profile(np.array([s["xi_c"] - 1e-12]), rl, rr)
        assert abs(rho_fan[0] - rc) < 1e-9 and abs(u_fan[0] - uc) < 1e-9


def check_cs_shock_profile(mutant=0):
    """CS shock tube (rho_L = 1.1, rho_R = 0.9, N = 2048, tau_FD = 1e-4, 400 steps,
    Sec. 4.1) against the inviscid similarity solution: small L1 error near x0."""
    nx, x0 = 2048, 1024
    rho, ux, uy = wl.shock_tube(nx, 1, 1.1, 0.9, x0)
    f = oracle.equilibrium(3, rho, ux, uy, mutant)
    tau_lu = oracle.tau_lu_from_fd(nx, 1e-4)
    steps = 400
    f = oracle.cs_run(f, tau_lu, steps, mutant=mutant)
    r, u, _ = oracle.macro(3, f, mutant)
    t = steps * oracle.CS_DT
    x = np.arange(nx, dtype=float)
    win = np.abs(x - x0) < 400
    xi = (x[win] - (x0 + 0.5)) / t
    r_ex, u_ex = oracle.shock_profile(xi, 1.1, 0.9)
    l1_rho = np.mean(np.abs(r[0, win] - r_ex))
    l1_u = np.mean(np.abs(u[0, win] - u_ex))
    assert l1_rho < 3e-3 and l1_u < 3e-3, (l1_rho, l1_u)


ALL_CHECKS = [
    check_rule_vs_numpy, check_rule_closed_forms, check_set_moments, check_set_ordering,
    check_feq_moments, check_macro_of_equilibrium,
    check_cs_fixed_point, check_cs_streaming_direction, check_cs_periodic_return, check_cs_omega_one,
    check_cs_conservation, check_cs_exact_rational, check_cs_linear_modes, check_cs_decay_closed_form,
    check_weno_quadratic_exact, check_weno_beta, check_weno_linear_weights, check_weno_eno,
    check_fd_linear_advection, check_fd_rk3_relaxation, check_fd_conservation, check_fd_fixed_point,
    check_fd_linear_modes, check_fd_high_precision, check_fd_decay_closed_form,
    check_imex_relaxation, check_imex_stiff_limit, check_imex_linear_modes, check_imex_conservation,
    check_imex_high_precision,
    check_units_tables, check_units_time_steps, check_shock_worked_example, check_shock_jump_conditions,
    check_cs_shock_profile,
]
