/*
 * Plain FP64 CPU oracle for the two isothermal lattice Boltzmann updates of
 * Negro, Busuioc, Ambrus, Gonnella, Lamura, Sofonea, "Comparison between
 * isothermal collision-streaming and finite-difference lattice Boltzmann
 * models" (arXiv:1904.02471).
 *
 * TEST INFRASTRUCTURE ONLY. Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this code. The CUDA
 * library never includes, links or calls it, and this file takes nothing
 * from the CUDA library (no shared headers, tables or constants).
 *
 * Everything is written for reading against the paper, not for speed:
 * one loop per formula, FP64 throughout, built with -ffp-contract=off so
 * that every product is rounded before it is added.
 *
 * Lattice layout used by every routine here: f[(k*ny + y)*nx + x],
 * population k = ix + n*iy where ix, iy index the 1D Gauss-Hermite nodes
 * sorted in ascending order. Periodic in x and y (Sec. 4).
 *
 * Pins: every function below is checked by tests/test_oracle_*.py against
 * closed forms, library routines or invariants; see the header of each test.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef OR_MUTANT
#define OR_MUTANT 0 /* >0 plants a known mistake (tests/test_oracle_mutants.py) */
#endif

/* ------------------------------------------------------------------------ */
/* Velocity sets: full-range Gauss-Hermite quadrature (Sec. 1 and Sec. 2).   */
/* The 1D nodes are the roots of the probabilists' Hermite polynomial He_n,  */
/* weights normalised so that sum w = 1 for the weight exp(-v^2/2)/sqrt(2pi).*/
/* The 2D set is the tensor product, K = n^2 velocities.                     */
/* ------------------------------------------------------------------------ */

/* He_n(x) by the three-term recurrence He_{m+1} = x He_m - m He_{m-1}.
 * Returns He_n(x); *prev receives He_{n-1}(x). */
static double he_poly(int n, double x, double* prev) {
    double hm1 = 0.0, h = 1.0;
    for (int m = 0; m < n; ++m) {
        double hp1 = x * h - (double)m * hm1;
        hm1 = h;
        h = hp1;
    }
    if (prev) *prev = hm1;
    return h;
}

/* 1D rule with n nodes, ascending. Returns 0 on success, -1 otherwise.
 * Roots are bracketed on a fine grid and refined by bisection; the rule is
 * then symmetrised (the exact rule is symmetric about 0). */
int or_hermite_rule(int n, double* x, double* w) {
    if (n < 1 || n > 16) return -1;
    double lim = sqrt(4.0 * n + 2.0) + 1.0;
    int found = 0;
    double step = 1e-3;
    double a = -lim;
    double fa = he_poly(n, a, NULL);
    while (a < lim && found < n) {
        double b = a + step;
        double fb = he_poly(n, b, NULL);
        if (fa == 0.0) {
            x[found++] = a;
        } else if (fa * fb < 0.0) {
            double lo = a, hi = b, flo = fa;
            for (int it = 0; it < 200; ++it) {
                double mid = 0.5 * (lo + hi);
                double fm = he_poly(n, mid, NULL);
                if (fm == 0.0) { lo = hi = mid; break; }
                if (flo * fm < 0.0) { hi = mid; } else { lo = mid; flo = fm; }
            }
            x[found++] = 0.5 * (lo + hi);
        }
        a = b;
        fa = fb;
    }
    if (found != n) return -1;
    for (int i = 0; i < n / 2; ++i) {
        double s = 0.5 * (x[n - 1 - i] - x[i]);
        x[i] = -s;
        x[n - 1 - i] = s;
    }
    if (n % 2 == 1) x[n / 2] = 0.0;
    /* Gauss weights for the normalised weight function:
     * w_i = n! / (n^2 He_{n-1}(x_i)^2). */
    double nfact = 1.0;
    for (int m = 2; m <= n; ++m) nfact *= (double)m;
    for (int i = 0; i < n; ++i) {
        double hprev;
        he_poly(n, x[i], &hprev);
        w[i] = nfact / ((double)n * (double)n * hprev * hprev);
    }
    return 0;
}

/* 2D product set, k = ix + n*iy. */
int or_velocity_set(int n, double* vx, double* vy, double* w) {
    double x1[16], w1[16];
    if (or_hermite_rule(n, x1, w1) != 0) return -1;
    for (int iy = 0; iy < n; ++iy)
        for (int ix = 0; ix < n; ++ix) {
            int k = ix + n * iy;
#if OR_MUTANT == 4
            vx[k] = x1[iy]; /* planted: velocity components transposed */
            vy[k] = x1[ix];
#else
            vx[k] = x1[ix];
            vy[k] = x1[iy];
#endif
            w[k] = w1[ix] * w1[iy];
        }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Pointwise physics: moments (Eq. f_moments_discrete) and the second-order  */
/* Hermite equilibrium (Eq. herfeq), with T = m = 1.                          */
/* ------------------------------------------------------------------------ */

/* rho = sum_k f_k, rho*u = sum_k f_k v_k, summed in ascending k. */
static void cell_moments(int K, const double* vx, const double* vy, const double* f,
                         int64_t stride, double* rho, double* ux, double* uy) {
    double r = 0.0, jx = 0.0, jy = 0.0;
    for (int k = 0; k < K; ++k) {
        double fk = f[(int64_t)k * stride];
        r = r + fk;
        jx = jx + fk * vx[k];
        jy = jy + fk * vy[k];
    }
    *rho = r;
    *ux = jx / r;
    *uy = jy / r;
}

/* f^eq_k = w_k rho { 1 + v_k.u + 1/2 [ (v_k.u)^2 - u^2 ] } */
static double feq_k(double wk, double vxk, double vyk, double rho, double ux, double uy) {
    double vu = vxk * ux + vyk * uy;
    double usq = ux * ux + uy * uy;
#if OR_MUTANT == 1
    return wk * rho * (1.0 + vu + 0.5 * (vu * vu)); /* planted: -u^2 dropped */
#elif OR_MUTANT == 2
    return wk * rho * (1.0 - vu + 0.5 * (vu * vu - usq)); /* planted: sign of v.u */
#else
    return wk * rho * (1.0 + vu + 0.5 * (vu * vu - usq));
#endif
}

void or_feq_cell(int K, const double* vx, const double* vy, const double* w,
                 double rho, double ux, double uy, double* feq) {
    for (int k = 0; k < K; ++k) feq[k] = feq_k(w[k], vx[k], vy[k], rho, ux, uy);
}

/* Macroscopic fields of a whole lattice. */
void or_macro(int nx, int ny, int K, const double* vx, const double* vy,
              const double* f, double* rho, double* ux, double* uy) {
    int64_t plane = (int64_t)nx * ny;
    for (int64_t c = 0; c < plane; ++c) cell_moments(K, vx, vy, f + c, plane, rho + c, ux + c, uy + c);
}

/* f = f^eq(rho, u) everywhere. */
void or_equilibrium(int nx, int ny, int K, const double* vx, const double* vy, const double* w,
                    const double* rho, const double* ux, const double* uy, double* f) {
    int64_t plane = (int64_t)nx * ny;
    for (int k = 0; k < K; ++k)
        for (int64_t c = 0; c < plane; ++c) f[k * plane + c] = feq_k(w[k], vx[k], vy[k], rho[c], ux[c], uy[c]);
}

static int wrap(int i, int n) {
    int r = i % n;
    return r < 0 ? r + n : r;
}

/* ------------------------------------------------------------------------ */
/* Collision-streaming update, Eq. (sc_evolution):                            */
/*   f_k(x + v_k dt, t + dt) - f_k(x, t) = -(dt/tau) [f_k - f^eq_k](x, t).    */
/* With dx = 1 and dt = 1/sqrt(3), v_k dt is the lattice vector c_k.          */
/* fin holds the pre-collision state at t, fout receives it at t + dt.       */
/* ------------------------------------------------------------------------ */
void or_cs_step(int nx, int ny, int K, const double* vx, const double* vy, const double* w,
                const int* cx, const int* cy, double omega, const double* fin, double* fout) {
    int64_t plane = (int64_t)nx * ny;
    double feq[64];
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            int64_t c = (int64_t)y * nx + x;
            double rho, ux, uy;
            cell_moments(K, vx, vy, fin + c, plane, &rho, &ux, &uy);
            or_feq_cell(K, vx, vy, w, rho, ux, uy, feq);
            for (int k = 0; k < K; ++k) {
                double fk = fin[k * plane + c];
                double post = fk - omega * (fk - feq[k]);
#if OR_MUTANT == 3
                int xd = wrap(x - cx[k], nx), yd = wrap(y - cy[k], ny); /* planted: streams backwards */
#else
                int xd = wrap(x + cx[k], nx), yd = wrap(y + cy[k], ny);
#endif
                fout[k * plane + (int64_t)yd * nx + xd] = post;
            }
        }
}

/* Lattice vectors c_k = v_k dt / dx (integers for the D2Q9 set). Returns -1
 * if some v_k dt/dx is not an integer to 1e-9, i.e. the set is off-lattice. */
int or_lattice_vectors(int K, const double* vx, const double* vy, double dt, double dx, int* cx, int* cy) {
    for (int k = 0; k < K; ++k) {
        double sx = vx[k] * dt / dx, sy = vy[k] * dt / dx;
        double rx = floor(sx + 0.5), ry = floor(sy + 0.5);
        if (fabs(sx - rx) > 1e-9 || fabs(sy - ry) > 1e-9) return -1;
        cx[k] = (int)rx;
        cy[k] = (int)ry;
    }
    return 0;
}

/* steps CS updates; f is updated in place, tmp is scratch of the same size. */
void or_cs_run(int nx, int ny, int K, const double* vx, const double* vy, const double* w,
               const int* cx, const int* cy, double omega, int64_t steps, double* f, double* tmp) {
    int64_t n = (int64_t)K * nx * ny;
    for (int64_t s = 0; s < steps; ++s) {
        or_cs_step(nx, ny, K, vx, vy, w, cx, cy, omega, f, tmp);
        memcpy(f, tmp, (size_t)n * sizeof(double));
    }
}

/* ------------------------------------------------------------------------ */
/* Finite-difference LB (Sec. 2): Eq. (evolution) in conservative form,      */
/*   d f_k/dt = -v_kx D_x f_k - v_ky D_y f_k - (f_k - f^eq_k)/tau,           */
/* with WENO-5 advection (Jiang & Shu, the paper's ref. jiang96) and the    */
/* third-order TVD Runge-Kutta scheme (Shu & Osher, refs. shu88, gottlieb98).*/
/* ------------------------------------------------------------------------ */

/* WENO-5 interface value at i+1/2 from the five upwind-side values
 * s = (f_{i-2}, f_{i-1}, f_i, f_{i+1}, f_{i+2}) (left-biased, for v > 0).
 * detail (optional) receives q0 q1 q2 beta0 beta1 beta2 omega0 omega1 omega2. */
static double weno5(const double s[5], double eps, double* detail) {
    double a = s[0], b = s[1], c = s[2], d = s[3], e = s[4];
    /* third-order candidates on the stencils {i-2,i-1,i}, {i-1,i,i+1}, {i,i+1,i+2} */
#if OR_MUTANT == 5
    double q0 = (2.0 * a - 7.0 * b + 11.0 * c) / 6.0;
    double q1 = (-b + 5.0 * c + 2.0 * d) / 6.0;
    double q2 = (-c + 5.0 * d + 2.0 * e) / 6.0; /* planted: mirrored candidate */
#else
    double q0 = (2.0 * a - 7.0 * b + 11.0 * c) / 6.0;
    double q1 = (-b + 5.0 * c + 2.0 * d) / 6.0;
    double q2 = (2.0 * c + 5.0 * d - e) / 6.0;
#endif
    /* smoothness indicators */
    double t;
    t = a - 2.0 * b + c;
    double b0 = (13.0 / 12.0) * t * t;
    t = a - 4.0 * b + 3.0 * c;
    b0 = b0 + 0.25 * t * t;
    t = b - 2.0 * c + d;
    double b1 = (13.0 / 12.0) * t * t;
    t = b - d;
    b1 = b1 + 0.25 * t * t;
    t = c - 2.0 * d + e;
#if OR_MUTANT == 8
    double b2 = (1.0 / 12.0) * t * t; /* planted: wrong coefficient */
#else
    double b2 = (13.0 / 12.0) * t * t;
#endif
    t = 3.0 * c - 4.0 * d + e;
    b2 = b2 + 0.25 * t * t;
    /* nonlinear weights from the linear weights (1/10, 6/10, 3/10) */
    double a0 = 0.1 / ((eps + b0) * (eps + b0));
    double a1 = 0.6 / ((eps + b1) * (eps + b1));
    double a2 = 0.3 / ((eps + b2) * (eps + b2));
    double sum = a0 + a1 + a2;
    double w0 = a0 / sum, w1 = a1 / sum, w2 = a2 / sum;
    if (detail) {
        detail[0] = q0; detail[1] = q1; detail[2] = q2;
        detail[3] = b0; detail[4] = b1; detail[5] = b2;
        detail[6] = w0; detail[7] = w1; detail[8] = w2;
    }
    return w0 * q0 + w1 * q1 + w2 * q2;
}

double or_weno5_face(const double* s, double eps, double* detail) { return weno5(s, eps, detail); }

/* Interface value at i+1/2 of a periodic 1D sequence g (length n, stride st)
 * upwinded by the sign of the advection velocity v (v != 0). */
static double face_value(const double* g, int n, int64_t st, int i, double v, double eps) {
    double s[5];
    if (v > 0.0) {
        for (int m = 0; m < 5; ++m) s[m] = g[(int64_t)wrap(i - 2 + m, n) * st];
    } else {
        /* mirror image: stencil read from the right, i+3 down to i-1 */
        for (int m = 0; m < 5; ++m) s[m] = g[(int64_t)wrap(i + 3 - m, n) * st];
    }
#if OR_MUTANT == 7
    if (v > 0.0) { /* planted: downwind stencil for v > 0 */
        for (int m = 0; m < 5; ++m) s[m] = g[(int64_t)wrap(i + 3 - m, n) * st];
    }
#endif
    return weno5(s, eps, NULL);
}

/* Right-hand side L(f) of the semi-discrete FD equation. Lf has f's shape.
 * Moments (and so f^eq) are taken from the f passed in. */
#if OR_MUTANT == 9
static const double* mutant_fn = 0; /* planted: the BGK moments of every stage taken from f^n */
#endif

void or_fd_rhs(int nx, int ny, int K, const double* vx, const double* vy, const double* w,
               double dx, double tau, double eps, const double* f, double* Lf) {
    int64_t plane = (int64_t)nx * ny;
    double* rho = (double*)malloc(sizeof(double) * plane * 3);
    double* ux = rho + plane;
    double* uy = ux + plane;
#if OR_MUTANT == 9
    or_macro(nx, ny, K, vx, vy, mutant_fn ? mutant_fn : f, rho, ux, uy); /* planted */
#else
    or_macro(nx, ny, K, vx, vy, f, rho, ux, uy);
#endif
    for (int k = 0; k < K; ++k) {
        const double* g = f + k * plane;
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                int64_t c = (int64_t)y * nx + x;
                double adv = 0.0;
                if (vx[k] != 0.0) {
                    const double* row = g + (int64_t)y * nx;
                    double fp = face_value(row, nx, 1, x, vx[k], eps);
                    double fm = face_value(row, nx, 1, x - 1, vx[k], eps);
                    adv = adv - vx[k] * (fp - fm) / dx;
                }
                if (vy[k] != 0.0) {
                    const double* col = g + x;
                    double fp = face_value(col, ny, nx, y, vy[k], eps);
                    double fm = face_value(col, ny, nx, y - 1, vy[k], eps);
                    adv = adv - vy[k] * (fp - fm) / dx;
                }
                double fe = feq_k(w[k], vx[k], vy[k], rho[c], ux[c], uy[c]);
                Lf[k * plane + c] = adv - (g[c] - fe) / tau;
            }
    }
    free(rho);
}

/* One SSP-RK3 step (Shu-Osher form):
 *   f1 = f + dt L(f)
 *   f2 = 3/4 f + 1/4 (f1 + dt L(f1))
 *   f  = 1/3 f + 2/3 (f2 + dt L(f2))
 * work must hold 3 lattices. */
void or_fd_step(int nx, int ny, int K, const double* vx, const double* vy, const double* w,
                double dx, double dt, double tau, double eps, double* f, double* work) {
    int64_t n = (int64_t)K * nx * ny;
    double* L = work;
    double* f1 = work + n;
    double* f2 = work + 2 * n;
#if OR_MUTANT == 9
    mutant_fn = f; /* planted; f is not overwritten before the third stage's L */
#endif
    or_fd_rhs(nx, ny, K, vx, vy, w, dx, tau, eps, f, L);
    for (int64_t i = 0; i < n; ++i) f1[i] = f[i] + dt * L[i];
    or_fd_rhs(nx, ny, K, vx, vy, w, dx, tau, eps, f1, L);
#if OR_MUTANT == 6
    for (int64_t i = 0; i < n; ++i) f2[i] = 0.5 * f[i] + 0.5 * (f1[i] + dt * L[i]); /* planted */
#else
    for (int64_t i = 0; i < n; ++i) f2[i] = 0.75 * f[i] + 0.25 * (f1[i] + dt * L[i]);
#endif
    or_fd_rhs(nx, ny, K, vx, vy, w, dx, tau, eps, f2, L);
#if OR_MUTANT == 9
    mutant_fn = 0;
#endif
    for (int64_t i = 0; i < n; ++i) f[i] = (1.0 / 3.0) * f[i] + (2.0 / 3.0) * (f2[i] + dt * L[i]);
}

void or_fd_run(int nx, int ny, int K, const double* vx, const double* vy, const double* w,
               double dx, double dt, double tau, double eps, int64_t steps, double* f, double* work) {
    for (int64_t s = 0; s < steps; ++s) or_fd_step(nx, ny, K, vx, vy, w, dx, dt, tau, eps, f, work);
}

/* ------------------------------------------------------------------------ */
/* FD with an implicit-explicit (IMEX) Runge-Kutta step. Sec. 4.1 notes that  */
/* the restriction dt < tau of the explicit scheme can be lifted with IMEX    */
/* schemes and cites one without printing it. The scheme here is the          */
/* second-order IMEX-SSP2(2,2,2) of Pareschi and Russo (J. Sci. Comput. 25,  */
/* 2005): the advection A(f) = -v.grad f (WENO-5 flux differences, as in      */
/* or_fd_rhs) is explicit, the BGK term C(f) = -(f - f^eq(f))/tau implicit,   */
/* with the tableaux                                                          */
/*   explicit: a~21 = 1, all other a~ = 0,          b~ = (1/2, 1/2)           */
/*   implicit: a11 = a22 = g, a21 = 1 - 2g, a12 = 0, b = (1/2, 1/2)           */
/*   g = 1 - 1/sqrt(2).                                                       */
/* Stage i: Y_i = f^n + dt sum_{j<i} (a~_ij A(Y_j) + a_ij C(Y_j))             */
/*               + dt a_ii C(Y_i),                                            */
/* step:    f^{n+1} = f^n + dt sum_i (b~_i A(Y_i) + b_i C(Y_i)).              */
/* The implicit equation of a stage is solved in closed form: C conserves     */
/* rho and rho u, so Y_i has the moments of its explicit part Z_i (the first  */
/* line), f^eq(Y_i) = f^eq(Z_i), and                                          */
/*   Y_i = (Z_i + lam f^eq(Z_i)) / (1 + lam),   lam = dt a_ii / tau.          */
/* C(Y_i) is then evaluated from Y_i's own moments, as the scheme states.     */
/* ------------------------------------------------------------------------ */

/* Advection part of L(f): A(f)_k = -v_kx dF_x/dx - v_ky dF_y/dx. */
static void fd_advection(int nx, int ny, int K, const double* vx, const double* vy, double dx, double eps,
                         const double* f, double* Af) {
    int64_t plane = (int64_t)nx * ny;
    for (int k = 0; k < K; ++k) {
        const double* g = f + k * plane;
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                double adv = 0.0;
                if (vx[k] != 0.0) {
                    const double* row = g + (int64_t)y * nx;
                    adv = adv - vx[k] * (face_value(row, nx, 1, x, vx[k], eps) -
                                         face_value(row, nx, 1, x - 1, vx[k], eps)) / dx;
                }
                if (vy[k] != 0.0) {
                    const double* col = g + x;
                    adv = adv - vy[k] * (face_value(col, ny, nx, y, vy[k], eps) -
                                         face_value(col, ny, nx, y - 1, vy[k], eps)) / dx;
                }
                Af[k * plane + (int64_t)y * nx + x] = adv;
            }
    }
}

/* Collision part of L(f): C(f)_k = -(f_k - f^eq_k(f)) / tau, moments of f. */
static void fd_collision(int nx, int ny, int K, const double* vx, const double* vy, const double* w, double tau,
                         const double* f, double* Cf) {
    int64_t plane = (int64_t)nx * ny;
    for (int64_t c = 0; c < plane; ++c) {
        double rho, ux, uy;
        cell_moments(K, vx, vy, f + c, plane, &rho, &ux, &uy);
        for (int k = 0; k < K; ++k)
            Cf[k * plane + c] = -(f[k * plane + c] - feq_k(w[k], vx[k], vy[k], rho, ux, uy)) / tau;
    }
}

/* One IMEX-SSP2(2,2,2) step. work holds 7 lattices; if ystages is not NULL
 * it receives the two stage values Y_1, Y_2 (2 lattices). */
void or_fd_imex_step(int nx, int ny, int K, const double* vx, const double* vy, const double* w,
                     double dx, double dt, double tau, double eps, double* f, double* work, double* ystages) {
    const int64_t plane = (int64_t)nx * ny, n = (int64_t)K * plane;
#if OR_MUTANT == 11
    const double g = 0.5; /* planted: gamma of the implicit tableau */
#else
    const double g = 1.0 - 1.0 / sqrt(2.0);
#endif
    const double ae[2][2] = {{0.0, 0.0}, {1.0, 0.0}};
    const double ai[2][2] = {{g, 0.0}, {1.0 - 2.0 * g, g}};
    const double be[2] = {0.5, 0.5}, bi[2] = {0.5, 0.5};
    double* Y[2] = {work, work + n};
    double* A[2] = {work + 2 * n, work + 3 * n};
    double* C[2] = {work + 4 * n, work + 5 * n};
    double* Z = work + 6 * n;
    for (int i = 0; i < 2; ++i) {
        /* explicit part of the stage */
        for (int64_t m = 0; m < n; ++m) {
            double z = f[m];
            for (int j = 0; j < i; ++j) z = z + dt * (ae[i][j] * A[j][m] + ai[i][j] * C[j][m]);
            Z[m] = z;
        }
        /* implicit part in closed form */
        const double lam = dt * ai[i][i] / tau;
        for (int64_t c = 0; c < plane; ++c) {
            double rho, ux, uy;
#if OR_MUTANT == 10
            cell_moments(K, vx, vy, f + c, plane, &rho, &ux, &uy); /* planted: equilibrium of f^n */
#else
            cell_moments(K, vx, vy, Z + c, plane, &rho, &ux, &uy);
#endif
            for (int k = 0; k < K; ++k) {
                const double fe = feq_k(w[k], vx[k], vy[k], rho, ux, uy);
                Y[i][k * plane + c] = (Z[k * plane + c] + lam * fe) / (1.0 + lam);
            }
        }
        fd_advection(nx, ny, K, vx, vy, dx, eps, Y[i], A[i]);
        fd_collision(nx, ny, K, vx, vy, w, tau, Y[i], C[i]);
    }
    for (int64_t m = 0; m < n; ++m)
        f[m] = f[m] + dt * ((be[0] * A[0][m] + bi[0] * C[0][m]) + (be[1] * A[1][m] + bi[1] * C[1][m]));
    if (ystages) {
        memcpy(ystages, Y[0], sizeof(double) * n);
        memcpy(ystages + n, Y[1], sizeof(double) * n);
    }
}

void or_fd_imex_run(int nx, int ny, int K, const double* vx, const double* vy, const double* w,
                    double dx, double dt, double tau, double eps, int64_t steps, double* f, double* work) {
    for (int64_t s = 0; s < steps; ++s) or_fd_imex_step(nx, ny, K, vx, vy, w, dx, dt, tau, eps, f, work, NULL);
}

/* ------------------------------------------------------------------------ */
/* Diagnostics: global sums and the projected Fourier amplitude used to fit  */
/* the decay laws of Eq. (shear_sol) and Eq. (taylor).                        */
/* out = {sum rho, sum rho ux, sum rho uy, A} with                           */
/*   A = norm * sum_{x,y} u_comp(x,y) px[x] py[y]  (comp 0: ux, 1: uy).       */
/* Sums run over y then x in ascending order.                                */
/* ------------------------------------------------------------------------ */
void or_observables(int nx, int ny, int K, const double* vx, const double* vy, const double* f,
                    int comp, const double* px, const double* py, double norm, double* out) {
    int64_t plane = (int64_t)nx * ny;
    double m = 0.0, mx = 0.0, my = 0.0, a = 0.0;
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            int64_t c = (int64_t)y * nx + x;
            double rho = 0.0, jx = 0.0, jy = 0.0;
            for (int k = 0; k < K; ++k) {
                double fk = f[k * plane + c];
                rho = rho + fk;
                jx = jx + fk * vx[k];
                jy = jy + fk * vy[k];
            }
            m = m + rho;
            mx = mx + jx;
            my = my + jy;
            double u = comp == 0 ? jx / rho : jy / rho;
            a = a + u * px[x] * py[y];
        }
    out[0] = m;
    out[1] = mx;
    out[2] = my;
    out[3] = norm * a;
}
