// extern "C" entry points declared in include/lbm.h. Argument checking,
// error codes and the exception barrier live here; the work is in Engine.
#include <cmath>
#include <cstring>
#include <new>
#include <string>

#include "engine.h"

namespace lbm {
const char* last_error_cstr();
}

struct lbm_ctx {
    lbm::Engine e;
};
struct lbm_batch {
    lbm::Engine e;
};

#define GUARD_BEGIN try {
#define GUARD_END                                            \
    }                                                        \
    catch (const std::bad_alloc&) {                          \
        lbm::set_error("host allocation failed");            \
        return LBM_ENOMEM;                                   \
    }                                                        \
    catch (...) {                                            \
        lbm::set_error("internal error");                    \
        return LBM_EINVAL;                                   \
    }

static const double kSqrt3 = 1.73205080756887729353;

extern "C" {

const char* lbm_version(void) { return "gb300-lbm 0.1 (sm_103a; CS D2Q9 + FD WENO5/SSP-RK3)"; }

const char* lbm_strerror(int code) {
    switch (code) {
        case LBM_OK: return "ok";
        case LBM_EINVAL: return "invalid argument";
        case LBM_ECFL: return "CFL condition violated (max|v| dt/dx > 1)";
        case LBM_ESTIFF: return "stiff collision term (FD dt > tau)";
        case LBM_ENOMEM: return "out of memory or over budget";
        case LBM_ECUDA: return "CUDA error";
        case LBM_ENOTREADY: return "not ready";
        case LBM_ETIMEOUT: return "timed out";
        case LBM_EBUSY: return "busy";
        case LBM_ENONFINITE: return "non-finite state observed";
        case LBM_ECANCELLED: return "cancelled";
        case LBM_ENOTFOUND: return "not found";
    }
    return "unknown error";
}

const char* lbm_last_error(void) { return lbm::last_error_cstr(); }

// ---- unit helpers ---------------------------------------------------------
double lbm_nu(int model, double tau, double dt) {
    if (model == LBM_CS) return tau - 0.5 * dt;  // Eq. (nulu)
    if (model == LBM_FD) return tau;             // Eq. (nu_fd), T = m = 1
    return NAN;
}

double lbm_tau_lu_from_fd(int n_lu, double tau_fd) { return n_lu * tau_fd + kSqrt3 / 6.0; }

double lbm_tau_fd_from_lu(int n_lu, double tau_lu) { return (tau_lu - kSqrt3 / 6.0) / n_lu; }

double lbm_tau_star(double tau_lu) { return kSqrt3 * tau_lu; }

double lbm_fd_max_dt(int q, double dx, double tau) {
    double vmax;
    switch (q) {
        case 3: vmax = lbm::GH<3>::vmax(); break;
        case 4: vmax = lbm::GH<4>::vmax(); break;
        case 5: vmax = lbm::GH<5>::vmax(); break;
        default: return NAN;
    }
    const double cfl_dt = dx / vmax;
    return cfl_dt < tau ? cfl_dt : tau;
}

int lbm_velocity_set(int q, double* vx, double* vy, double* w) {
    if (!vx || !vy || !w) return LBM_EINVAL;
    for (int k = 0; k < q * q; ++k) {
        switch (q) {
            case 3: vx[k] = lbm::vx_of<3>(k); vy[k] = lbm::vy_of<3>(k); w[k] = lbm::w_of<3>(k); break;
            case 4: vx[k] = lbm::vx_of<4>(k); vy[k] = lbm::vy_of<4>(k); w[k] = lbm::w_of<4>(k); break;
            case 5: vx[k] = lbm::vx_of<5>(k); vy[k] = lbm::vy_of<5>(k); w[k] = lbm::w_of<5>(k); break;
            default: return LBM_EINVAL;
        }
    }
    if (q < 3 || q > 5) return LBM_EINVAL;
    return LBM_OK;
}

int lbm_fit_decay(const double* t, const double* a, int64_t n, double t_skip, double* gamma, double* a0) {
    if (!t || !a || !gamma || n < 0) return LBM_EINVAL;
    double s = 0, st = 0, sy = 0, stt = 0, sty = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (t[i] < t_skip || !(std::fabs(a[i]) > 0)) continue;
        const double y = std::log(std::fabs(a[i]));
        s += 1;
        st += t[i];
        sy += y;
        stt += t[i] * t[i];
        sty += t[i] * y;
    }
    const double den = s * stt - st * st;
    if (s < 2 || !(std::fabs(den) > 0)) {
        lbm::set_error("fit needs at least two distinct samples");
        return LBM_EINVAL;
    }
    const double slope = (s * sty - st * sy) / den;
    const double icpt = (sy - slope * st) / s;
    *gamma = -slope;
    if (a0) *a0 = std::exp(icpt);
    return LBM_OK;
}

// ---- single lattice -------------------------------------------------------
int lbm_create_spec(lbm_ctx** out, const lbm_spec* spec, void* stream) {
    GUARD_BEGIN
    if (!out) return LBM_EINVAL;
    *out = nullptr;
    lbm_ctx* c = new (std::nothrow) lbm_ctx;
    if (!c) return LBM_ENOMEM;
    const int rc = c->e.create(spec, 1, stream);
    if (rc != LBM_OK) {
        delete c;
        return rc;
    }
    *out = c;
    return LBM_OK;
    GUARD_END
}

int lbm_create(lbm_ctx** out, int model, int q, int nx, int ny, double tau, double dt, double dx, int precision,
               double rho0, void* stream) {
    lbm_spec s;
    memset(&s, 0, sizeof s);
    s.model = model;
    s.q_per_axis = q;
    s.nx = nx;
    s.ny = ny;
    s.precision = precision;
    s.tau = tau;
    s.dt = dt;
    s.dx = dx;
    s.rho0 = rho0;
    return lbm_create_spec(out, &s, stream);
}

int lbm_spec_from_nu(const lbm_spec* in, double nu, int nu_model, int n_ref, lbm_spec* out) {
    GUARD_BEGIN
    if (!in || !out) {
        lbm::set_error("lbm_spec_from_nu: null spec");
        return LBM_EINVAL;
    }
    if (!(nu > 0) || !std::isfinite(nu) || (nu_model != LBM_CS && nu_model != LBM_FD) || n_ref < 0) {
        lbm::set_error("lbm_spec_from_nu: nu must be positive and finite, nu_model LBM_CS or LBM_FD, n_ref >= 0");
        return LBM_EINVAL;
    }
    lbm_spec s = *in;
    const double n = n_ref > 0 ? (double)n_ref : (double)s.nx;
    if (!(n >= 1)) {
        lbm::set_error("lbm_spec_from_nu: the reference length needs at least one node");
        return LBM_EINVAL;
    }
    // viscosity in the target model's own units (Sec. 3: nu_LU = N nu_FD)
    double nu_m = nu;
    if (nu_model != s.model) nu_m = s.model == LBM_CS ? n * nu : nu / n;
    if (s.model == LBM_CS) {
        double dt = s.dt;  // the defaults of lbm_create: dt = 1/sqrt(3), or dx/sqrt(3)
        if (dt == 0) dt = s.dx == 0 ? 1.0 / kSqrt3 : s.dx / kSqrt3;
        s.tau = nu_m + 0.5 * dt;  // Eq. (nulu)
    } else {
        s.tau = nu_m;             // Eq. (nu_fd), T = m = 1
    }
    return lbm::Engine::validate(&s, out);
    GUARD_END
}

int lbm_create_nu(lbm_ctx** out, const lbm_spec* in, double nu, int nu_model, int n_ref, void* stream) {
    GUARD_BEGIN
    if (!out) return LBM_EINVAL;
    *out = nullptr;
    lbm_spec s;
    const int rc = lbm_spec_from_nu(in, nu, nu_model, n_ref, &s);
    if (rc != LBM_OK) return rc;
    return lbm_create_spec(out, &s, stream);
    GUARD_END
}

void lbm_destroy(lbm_ctx* c) {
    try {
        delete c;
    } catch (...) {
    }
}

int lbm_get_spec(const lbm_ctx* c, lbm_spec* out) {
    if (!c || !out) return LBM_EINVAL;
    *out = const_cast<lbm_ctx*>(c)->e.L(0).spec;
    return LBM_OK;
}

int lbm_set_weno_eps(lbm_ctx* c, double eps) {
    GUARD_BEGIN
    if (!c) return LBM_EINVAL;
    return c->e.set_eps(0, eps);
    GUARD_END
}

int lbm_init(lbm_ctx* c, const double* rho, const double* ux, const double* uy) {
    GUARD_BEGIN
    if (!c) return LBM_EINVAL;
    return c->e.init(0, rho, ux, uy);
    GUARD_END
}

int lbm_set_populations(lbm_ctx* c, const double* f) {
    GUARD_BEGIN
    if (!c) return LBM_EINVAL;
    return c->e.set_populations(0, f);
    GUARD_END
}

int lbm_step(lbm_ctx* c, int64_t n) {
    GUARD_BEGIN
    if (!c) return LBM_EINVAL;
    return c->e.step(n);
    GUARD_END
}

int lbm_inject_wait_timeout(lbm_ctx* c, int microseconds) {
    GUARD_BEGIN
    if (!c) return LBM_EINVAL;
    return c->e.inject_wait_timeout(microseconds);
    GUARD_END
}

int lbm_batch_inject_wait_timeout(lbm_batch* b, int microseconds) {
    GUARD_BEGIN
    if (!b) return LBM_EINVAL;
    return b->e.inject_wait_timeout(microseconds);
    GUARD_END
}

int lbm_sync(lbm_ctx* c) {
    GUARD_BEGIN
    if (!c) return LBM_EINVAL;
    return c->e.sync();
    GUARD_END
}

int64_t lbm_steps_done(const lbm_ctx* c) { return c ? const_cast<lbm_ctx*>(c)->e.L(0).step0 : -1; }

int lbm_moments(lbm_ctx* c, double* rho, double* ux, double* uy) {
    GUARD_BEGIN
    if (!c) return LBM_EINVAL;
    return c->e.moments(0, rho, ux, uy);
    GUARD_END
}

int lbm_populations(lbm_ctx* c, double* f) {
    GUARD_BEGIN
    if (!c) return LBM_EINVAL;
    return c->e.populations(0, f);
    GUARD_END
}

int lbm_populations_region(lbm_ctx* c, int x0, int y0, int wx, int wy, double* f) {
    GUARD_BEGIN
    if (!c) return LBM_EINVAL;
    return c->e.populations_region(0, x0, y0, wx, wy, f);
    GUARD_END
}

int lbm_set_probe(lbm_ctx* c, int comp, const double* px, const double* py, double norm) {
    GUARD_BEGIN
    if (!c) return LBM_EINVAL;
    return c->e.set_probe(0, comp, px, py, norm);
    GUARD_END
}

int lbm_observables(lbm_ctx* c, lbm_obs* out) {
    GUARD_BEGIN
    if (!c) return LBM_EINVAL;
    return c->e.observables(0, out);
    GUARD_END
}

int lbm_record(lbm_ctx* c, int64_t every, int64_t capacity) {
    GUARD_BEGIN
    if (!c) return LBM_EINVAL;
    return c->e.record(0, every, capacity);
    GUARD_END
}

int lbm_series(lbm_ctx* c, lbm_obs* out, int64_t cap, int64_t* count) {
    GUARD_BEGIN
    if (!c) return LBM_EINVAL;
    long long n = 0;
    const int rc = c->e.series(0, out, cap, &n);
    if (count) *count = n;
    return rc;
    GUARD_END
}

size_t lbm_checkpoint_size(const lbm_ctx* c) { return c ? const_cast<lbm_ctx*>(c)->e.checkpoint_size(0) : 0; }

int lbm_save(lbm_ctx* c, void* buf, size_t size) {
    GUARD_BEGIN
    if (!c) return LBM_EINVAL;
    return c->e.save(0, buf, size);
    GUARD_END
}

int lbm_load(lbm_ctx* c, const void* buf, size_t size) {
    GUARD_BEGIN
    if (!c) return LBM_EINVAL;
    return c->e.load(0, buf, size);
    GUARD_END
}

int lbm_device_view(lbm_ctx* c, lbm_view* out) {
    if (!c || !out) return LBM_EINVAL;
    lbm::Lattice& L = c->e.L(0);
    out->base = L.buf[L.state_buf()];
    out->plane = L.plane;
    out->pitch = L.pitch;
    out->elem_bytes = L.elem;
    out->cs_pull_phase = L.phase_code();
    out->reserved = 0;
    return LBM_OK;
}

// ---- batch ------------------------------------------------------------------
int lbm_batch_create(lbm_batch** out, const lbm_spec* specs, int n, void* stream) {
    GUARD_BEGIN
    if (!out) return LBM_EINVAL;
    *out = nullptr;
    lbm_batch* b = new (std::nothrow) lbm_batch;
    if (!b) return LBM_ENOMEM;
    const int rc = b->e.create(specs, n, stream);
    if (rc != LBM_OK) {
        delete b;
        return rc;
    }
    *out = b;
    return LBM_OK;
    GUARD_END
}

void lbm_batch_destroy(lbm_batch* b) {
    try {
        delete b;
    } catch (...) {
    }
}

int lbm_batch_size(const lbm_batch* b) { return b ? const_cast<lbm_batch*>(b)->e.n_lattices() : 0; }

#define BATCH_IDX_CHECK(b, i) \
    if (!(b) || !(b)->e.valid(i)) return LBM_EINVAL

int lbm_batch_init(lbm_batch* b, int i, const double* rho, const double* ux, const double* uy) {
    GUARD_BEGIN
    BATCH_IDX_CHECK(b, i);
    return b->e.init(i, rho, ux, uy);
    GUARD_END
}

int lbm_batch_set_budget(lbm_batch* b, int i, int64_t steps) {
    GUARD_BEGIN
    BATCH_IDX_CHECK(b, i);
    return b->e.set_budget(i, steps);
    GUARD_END
}

int lbm_batch_step(lbm_batch* b, int64_t n) {
    GUARD_BEGIN
    if (!b) return LBM_EINVAL;
    return b->e.step(n);
    GUARD_END
}

int lbm_batch_sync(lbm_batch* b) {
    GUARD_BEGIN
    if (!b) return LBM_EINVAL;
    return b->e.sync();
    GUARD_END
}

int64_t lbm_batch_steps_done(const lbm_batch* b, int i) {
    if (!b || i < 0 || i >= const_cast<lbm_batch*>(b)->e.n_lattices()) return -1;
    return const_cast<lbm_batch*>(b)->e.L(i).step0;
}

int lbm_batch_moments(lbm_batch* b, int i, double* rho, double* ux, double* uy) {
    GUARD_BEGIN
    BATCH_IDX_CHECK(b, i);
    return b->e.moments(i, rho, ux, uy);
    GUARD_END
}

int lbm_batch_populations(lbm_batch* b, int i, double* f) {
    GUARD_BEGIN
    BATCH_IDX_CHECK(b, i);
    return b->e.populations(i, f);
    GUARD_END
}

int lbm_batch_populations_region(lbm_batch* b, int i, int x0, int y0, int wx, int wy, double* f) {
    GUARD_BEGIN
    BATCH_IDX_CHECK(b, i);
    return b->e.populations_region(i, x0, y0, wx, wy, f);
    GUARD_END
}

int lbm_batch_set_probe(lbm_batch* b, int i, int comp, const double* px, const double* py, double norm) {
    GUARD_BEGIN
    BATCH_IDX_CHECK(b, i);
    return b->e.set_probe(i, comp, px, py, norm);
    GUARD_END
}

int lbm_batch_observables(lbm_batch* b, int i, lbm_obs* out) {
    GUARD_BEGIN
    BATCH_IDX_CHECK(b, i);
    return b->e.observables(i, out);
    GUARD_END
}

int lbm_batch_record(lbm_batch* b, int i, int64_t every, int64_t capacity) {
    GUARD_BEGIN
    BATCH_IDX_CHECK(b, i);
    return b->e.record(i, every, capacity);
    GUARD_END
}

int lbm_batch_series(lbm_batch* b, int i, lbm_obs* out, int64_t cap, int64_t* count) {
    GUARD_BEGIN
    BATCH_IDX_CHECK(b, i);
    long long n = 0;
    const int rc = b->e.series(i, out, cap, &n);
    if (count) *count = n;
    return rc;
    GUARD_END
}

int lbm_batch_groups(lbm_batch* b, int* model, int* q, int* precision, int cap) {
    if (!b) return -1;
    const int G = b->e.n_groups();
    for (int g = 0; g < G && g < cap; ++g) {
        if (model) model[g] = b->e.G(g).model;
        if (q) q[g] = b->e.G(g).q1;
        if (precision) precision[g] = b->e.G(g).precision;
    }
    return G;
}

int lbm_batch_step_profiled(lbm_batch* b, int64_t n, double* ms, int cap, double* total_ms) {
    GUARD_BEGIN
    if (!b) return LBM_EINVAL;
    return b->e.step_profiled(n, ms, cap, total_ms);
    GUARD_END
}

int lbm_batch_config(lbm_batch* b, int group, int tile, int grid) {
    GUARD_BEGIN
    if (!b) return LBM_EINVAL;
    return b->e.set_group_config(group, tile, grid);
    GUARD_END
}

int lbm_config(lbm_ctx* c, int tile, int grid) {
    GUARD_BEGIN
    if (!c) return LBM_EINVAL;
    return c->e.set_group_config(0, tile, grid);
    GUARD_END
}

int lbm_n_tiles(int model) {
    return model == LBM_CS ? (int)lbm::CS_NTILES : (model == LBM_FD ? (int)lbm::FD_NTILES : -1);
}

int64_t lbm_batch_kernel_launches(const lbm_batch* b) {
    return b ? const_cast<lbm_batch*>(b)->e.kernel_launches() : -1;
}

int64_t lbm_kernel_launches(const lbm_ctx* c) { return c ? const_cast<lbm_ctx*>(c)->e.kernel_launches() : -1; }

int lbm_batch_tune(lbm_batch* b, int trial_steps, char* report, size_t report_len) {
    GUARD_BEGIN
    if (!b) return LBM_EINVAL;
    std::string rep;
    const int rc = b->e.tune(trial_steps, &rep);
    if (report && report_len > 0) {
        strncpy(report, rep.c_str(), report_len - 1);
        report[report_len - 1] = 0;
    }
    return rc;
    GUARD_END
}

}  // extern "C"
