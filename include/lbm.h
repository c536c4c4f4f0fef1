/*
 * lbm.h - C ABI of the GB300 (sm_103a) isothermal lattice Boltzmann library.
 *
 * Two time-step updates for an ideal isothermal fluid on a periodic 2D
 * lattice, after Negro et al., "Comparison between isothermal
 * collision-streaming and finite-difference lattice Boltzmann models"
 * (arXiv:1904.02471):
 *
 *  - LBM_CS, collision-streaming: Eq. (sc_evolution) with the D2Q9
 *    Gauss-Hermite set (Sec. 2), dx = 1, dt = 1/sqrt(3), |v_ka| = sqrt(3);
 *    collision and streaming fused into one pass.
 *  - LBM_FD, finite-difference: Eq. (evolution) on a Gauss-Hermite product
 *    set with q_per_axis roots per axis (Sec. 1-2), WENO-5 advection and
 *    third-order TVD (SSP) Runge-Kutta time stepping (Sec. 2), with the BGK
 *    term and the (rho, u) moments recomputed inside every stage.
 *
 * Units are the paper's: T = m = 1, so the sound speed is 1; f^eq is the
 * second-order Hermite expansion Eq. (herfeq); rho and rho u follow
 * Eq. (f_moments_discrete).
 *
 * Conventions shared by every call:
 *  - Host field arrays are row-major [ny][nx] (x fastest), float64.
 *  - Population arrays are [K][ny][nx], K = q_per_axis^2, population
 *    k = ix + q*iy, ix / iy indexing the 1D Gauss-Hermite nodes in ascending
 *    order (for D2Q9: nodes -sqrt3, 0, sqrt3; k = 4 is the rest velocity).
 *  - Every call returns an int status (LBM_OK = 0 on success) unless stated;
 *    lbm_strerror() names a code, lbm_last_error() gives the detail of the
 *    last failure on the calling thread. No C++ exception or abort crosses
 *    this interface. Host pointers are caller-owned and only read or written
 *    during the call. Device memory is owned by the library.
 *  - A context is not thread-safe: one thread at a time per context.
 *    A server (lbm_server_*) is thread-safe.
 *  - Work is enqueued on the context's CUDA stream; calls that return data to
 *    host buffers synchronise that stream first.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
enum {
    LBM_OK = 0,
    LBM_EINVAL = 1,      /* bad argument or inconsistent parameters */
    LBM_ECFL = 2,        /* CFL = max|v_ka| dt/dx > 1 (Sec. 4.1) */
    LBM_ESTIFF = 3,      /* FD with dt > tau: stiff collision term (Sec. 4.1) */
    LBM_ENOMEM = 4,      /* device or host allocation failed, or over budget */
    LBM_ECUDA = 5,       /* a CUDA runtime call failed (see lbm_last_error) */
    LBM_ENOTREADY = 6,   /* result not available yet (lbm_poll) */
    LBM_ETIMEOUT = 7,    /* a bounded wait ran out */
    LBM_EBUSY = 8,       /* resource in use */
    LBM_ENONFINITE = 9,  /* a non-finite mass or amplitude was observed */
    LBM_ECANCELLED = 10, /* request cancelled before completion */
    LBM_ENOTFOUND = 11   /* unknown ticket or index */
};

/* ---- model and storage selectors -------------------------------------- */
enum { LBM_CS = 0, LBM_FD = 1 };
/* LBM_FP64: populations stored and updated in float64.
 * LBM_FP32_DEV: populations stored as float32 deviations g_k = f_k - w_k rho0
 * from a uniform reference state, with float32 collision and advection;
 * global sums (mass, momentum, amplitude) are accumulated in float64. */
enum { LBM_FP64 = 0, LBM_FP32_DEV = 1 };

typedef struct lbm_ctx lbm_ctx;

/* Observables of one state, Sec. 4.2-4.3 diagnostics.
 * mass = sum rho, mom_x/mom_y = sum rho u, amp = norm * sum u_c px[x] py[y]
 * (the probe set by lbm_set_probe; 0 if none). time = step * dt in the
 * context's time unit. nonfinite != 0 if mass or amp is not finite. */
typedef struct {
    int64_t step;
    double time;
    double mass;
    double mom_x;
    double mom_y;
    double amp;
    int32_t nonfinite;
    int32_t reserved;
} lbm_obs;

/* State storage of a CS lattice. LBM_STORE_AB: two buffers, pull form.
 * LBM_STORE_INPLACE: one buffer updated in place (the AA access pattern:
 * even steps collide at the node and write to the opposite velocity's slot,
 * odd steps read and write the nine locations a node owns), half the device
 * memory at the same traffic and bit-identical results. FD needs its stage
 * buffers: LBM_STORE_INPLACE with LBM_FD is LBM_EINVAL. */
#define LBM_STORE_AB 0
#define LBM_STORE_INPLACE 1

/* Time integration of an FD lattice. LBM_TS_RK3 (0, the default): the
 * third-order TVD (SSP) Runge-Kutta scheme of Sec. 2, three stages per step;
 * it needs dt <= tau (Sec. 4.1, LBM_ESTIFF otherwise). LBM_TS_IMEX: the
 * second-order IMEX-SSP2(2,2,2) Runge-Kutta scheme of Pareschi and Russo
 * (2005) with explicit WENO-5 advection and implicit BGK collision, two
 * stages per step, any dt / tau: Sec. 4.1 notes that implicit-explicit
 * schemes lift dt < tau but prints none. The CFL bound holds for both. A CS
 * lattice takes LBM_TS_RK3 (the field is ignored there and must be 0). */
#define LBM_TS_RK3 0
#define LBM_TS_IMEX 1
/* LBM_TS_RK3_FUSED: the SSP-RK3 step of LBM_TS_RK3 (same stages, same
 * dt <= tau) temporally blocked: the three stages of a step in one launch per
 * tile (the stages of Sec. 2, not a different scheme). A tile reads f^n
 * with a halo of 9 nodes, computes stage 1 on the tile plus 6 nodes and
 * stage 2 on the tile plus 3 nodes in shared memory, and writes only
 * f^(n+1): 2Q values of device memory per lattice update instead of 8Q, and
 * two state buffers instead of three, for 2.2x the stage evaluations of the
 * three stage launches (the halo nodes). Results equal LBM_TS_RK3's to
 * rounding (the same arithmetic per node and stage). FD only. */
#define LBM_TS_RK3_FUSED 2

/* Parameters of a lattice. See lbm_create for their meaning. */
typedef struct {
    int model;        /* LBM_CS or LBM_FD */
    int q_per_axis;   /* 3 for CS; 3, 4 or 5 for FD */
    int nx, ny;       /* lattice nodes per axis, >= 1 */
    int precision;    /* LBM_FP64 or LBM_FP32_DEV */
    int storage;      /* LBM_STORE_AB (0, default) or LBM_STORE_INPLACE (CS only) */
    double tau;       /* CS: tau_LU; FD: tau_FD */
    double dt;        /* time step (CS: 0 selects 1/sqrt(3)) */
    double dx;        /* node spacing (CS: 0 selects 1; FD: 0 selects 1/nx) */
    double rho0;      /* reference density of the FP32 deviation storage (0 selects 1) */
    int scheme;       /* FD time integration: LBM_TS_RK3 (0, default), LBM_TS_IMEX or LBM_TS_RK3_FUSED */
    int reserved;     /* 0 */
} lbm_spec;

/* ---- unit helpers (Sec. 3) ---------------------------------------------- */

/* Kinematic viscosity of a model in its own units:
 * CS, Eq. (nulu): nu_LU = tau_LU - dt/2; FD, Eq. (nu_fd): nu_FD = tau_FD
 * (T = m = 1). Returns NaN for an unknown model. */
double lbm_nu(int model, double tau, double dt);

/* Eq. (nu-transfer): tau_LU = N tau_FD + sqrt(3)/6 for a CS lattice of N
 * nodes along the reference length. */
double lbm_tau_lu_from_fd(int n_lu, double tau_fd);

/* Inverse of lbm_tau_lu_from_fd: tau_FD = (tau_LU - sqrt(3)/6) / N. */
double lbm_tau_fd_from_lu(int n_lu, double tau_lu);

/* Relaxation time in the usual lattice units (dt = 1, cs^2 = 1/3):
 * tau* = tau_LU / dt_LU = sqrt(3) tau_LU. */
double lbm_tau_star(double tau_lu);

/* Largest FD time step allowed by CFL <= 1 and dt <= tau (Sec. 4.1):
 * min(dx / max|v_ka|, tau). Returns NaN for q_per_axis outside 3..5. */
double lbm_fd_max_dt(int q_per_axis, double dx, double tau);

/* The velocity set used by the library (Sec. 1-2, Gauss-Hermite product
 * set): writes K = q^2 entries to each of vx, vy, w (caller-owned).
 * LBM_EINVAL for q outside 3..5. */
int lbm_velocity_set(int q_per_axis, double* vx, double* vy, double* w);

/* Least-squares fit of ln|a| = ln a0 - gamma t over the n samples with
 * t >= t_skip (Sec. 4.2: nu_app from a numerical fit of Eq. (shear_sol);
 * Sec. 4.3: of Eq. (taylor)). Writes gamma and a0. LBM_EINVAL if fewer than
 * two samples qualify. */
int lbm_fit_decay(const double* t, const double* a, int64_t n, double t_skip, double* gamma,
                  double* a0);

/* ---- a single lattice ---------------------------------------------------- */

/* Create a lattice context (Sec. 2 models, Sec. 3 units).
 *  model, q_per_axis: LBM_CS with q = 3 (D2Q9), or LBM_FD with q in 3..5.
 *  nx, ny: periodic lattice size, each >= 1, nx*ny*K < 2^40.
 *  tau: relaxation time in the model's units (CS tau_LU > dt/2; FD tau_FD > 0).
 *  dt, dx: CS requires dx/dt = sqrt(3) (0, 0 select dx = 1, dt = 1/sqrt(3));
 *      FD dx = 0 selects 1/nx (unit domain), dt must be > 0.
 *  precision: LBM_FP64 or LBM_FP32_DEV. rho0: reference density of the
 *      deviation storage (0 selects 1; ignored for LBM_FP64).
 *  cuda_stream: a cudaStream_t to enqueue work on, or NULL for a stream the
 *      library creates (the legacy default stream is never used).
 * Errors: LBM_EINVAL (bad sizes, model/q pair, tau <= dt/2 for CS, dx/dt),
 *  LBM_ECFL (max|v_ka| dt/dx > 1), LBM_ESTIFF (FD dt > tau with an RK3
 *  scheme), LBM_ENOMEM, LBM_ECUDA. On error *out is NULL. The state is zero
 *  until lbm_init. lbm_create makes RK3 lattices; lbm_create_spec takes the
 *  scheme from the spec. */
int lbm_create(lbm_ctx** out, int model, int q_per_axis, int nx, int ny, double tau, double dt,
               double dx, int precision, double rho0, void* cuda_stream);

/* Same as lbm_create with the parameters in a struct. */
int lbm_create_spec(lbm_ctx** out, const lbm_spec* spec, void* cuda_stream);

/* Resolve a spec from a kinematic viscosity instead of a relaxation time
 * (Sec. 3 unit mapping). in gives model, q_per_axis, nx, ny, precision,
 * storage, dt, dx and rho0 with the meaning and defaults of lbm_create (its
 * tau is ignored); nu > 0 is given in the units of model nu_model (LBM_CS:
 * lattice units, LBM_FD: FD units). A viscosity in the other model's units
 * is converted with nu_LU = N nu_FD (Sec. 3: nu_ref;LU = nu_ref;FD / N), N =
 * n_ref nodes of the CS lattice along the reference length (0 selects nx).
 * Then tau follows from the model's own relation: CS tau_LU = nu_LU + dt/2
 * (Eq. nulu, so an FD viscosity gives tau_LU = N tau_FD + sqrt(3)/6 with the
 * default dt, Eq. nu-transfer); FD tau_FD = nu_FD (Eq. nu_fd, T = m = 1).
 * *out receives the resolved spec, validated as lbm_create validates it
 * (same error codes). Host only: no device work. LBM_EINVAL for null
 * pointers, nu not positive and finite, a bad nu_model or n_ref < 0. */
int lbm_spec_from_nu(const lbm_spec* in, double nu, int nu_model, int n_ref, lbm_spec* out);

/* lbm_create from a viscosity: lbm_spec_from_nu, then lbm_create_spec.
 * Same errors as both; on error *out is NULL. */
int lbm_create_nu(lbm_ctx** out, const lbm_spec* in, double nu, int nu_model, int n_ref, void* cuda_stream);

/* Release all device memory of the context (after finishing its stream).
 * NULL is ignored. */
void lbm_destroy(lbm_ctx* ctx);

/* Parameters actually in use (defaults resolved). */
int lbm_get_spec(const lbm_ctx* ctx, lbm_spec* out);

/* WENO-5 smoothness regulariser epsilon (FD only, default 1e-6; Sec. 2 cites
 * Jiang-Shu WENO-5 without printing it). FP32 storage accepts [1e-8, 1e9],
 * FP64 [1e-60, 1e60]; LBM_EINVAL otherwise or for a CS context. */
int lbm_set_weno_eps(lbm_ctx* ctx, double eps);

/* Initialise f = f^eq(rho, u) (Eq. herfeq) from host fields rho, ux, uy,
 * each [ny][nx]; rho must be > 0 and finite and u finite, else LBM_EINVAL
 * (checked on the device; the state is then not initialised). The step
 * counter restarts at 0. The paper does not state its initial populations;
 * the equilibrium is the reading used here. */
int lbm_init(lbm_ctx* ctx, const double* rho, const double* ux, const double* uy);

/* Load an arbitrary state: f is [K][ny][nx] full populations (for
 * LBM_FP32_DEV they are stored as float32(f - w_k rho0)); a non-finite value
 * gives LBM_EINVAL (checked on the device; the state is then not set). The
 * step counter is kept. */
int lbm_set_populations(lbm_ctx* ctx, const double* f);

/* Enqueue n >= 0 time steps on the context stream and return. One step is
 * one application of Eq. (sc_evolution) (CS) or one RK step of the lattice's
 * scheme (FD: three stages, two with LBM_TS_IMEX; LBM_TS_RK3_FUSED runs the
 * three stages in one launch). */
int lbm_step(lbm_ctx* ctx, int64_t n);

/* Wait for all enqueued work. Returns LBM_ECUDA if a kernel failed. */
int lbm_sync(lbm_ctx* ctx);

/* Number of steps completed or enqueued since lbm_init. */
int64_t lbm_steps_done(const lbm_ctx* ctx);

/* Synchronous readout of rho, ux, uy (host [ny][nx] each, caller-owned) of
 * the current state, Eq. (f_moments_discrete). */
int lbm_moments(lbm_ctx* ctx, double* rho, double* ux, double* uy);

/* Synchronous readout of the current populations f[K][ny][nx] (host),
 * as full f in float64. For CS this is the pre-collision state f(x, t) of
 * Eq. (sc_evolution) (the kernels store another phase internally). */
int lbm_populations(lbm_ctx* ctx, double* f);

/* Synchronous readout of a window of the current populations: f[K][wy][wx]
 * (host) receives the full f at nodes (x0 + i) mod nx, (y0 + j) mod ny for
 * 0 <= i < wx, 0 <= j < wy. Requires 0 <= x0 < nx, 0 <= y0 < ny,
 * 1 <= wx <= nx, 1 <= wy <= ny (LBM_EINVAL otherwise). Same phase and
 * precision conventions as lbm_populations. */
int lbm_populations_region(lbm_ctx* ctx, int x0, int y0, int wx, int wy, double* f);

/* Amplitude probe for the observables: A = norm * sum_{x,y} u_comp px[x] py[y],
 * comp 0 = u_x, 1 = u_y; px has nx entries and py ny entries (host, copied).
 * Shear wave (Sec. 4.2): comp 1, px = sin(kx), py = 1, norm = 2/(nx ny).
 * Taylor-Green (Sec. 4.3): comp 0, px = sin(kx), py = cos(ky), norm = 4/(nx ny). */
int lbm_set_probe(lbm_ctx* ctx, int comp, const double* px, const double* py, double norm);

/* Synchronous observables of the current state (float64 global sums). */
int lbm_observables(lbm_ctx* ctx, lbm_obs* out);

/* Record the observables of every state whose step index is a multiple of
 * `every` (0 switches recording off) during later lbm_step calls, fused into
 * the step kernels, into a device series of `capacity` records. Resets the
 * series. */
int lbm_record(lbm_ctx* ctx, int64_t every, int64_t capacity);

/* Copy up to cap recorded observables (oldest first) to out; *count receives
 * the number recorded so far (capped at the capacity). Synchronous. */
int lbm_series(lbm_ctx* ctx, lbm_obs* out, int64_t cap, int64_t* count);

/* Checkpoint: lbm_checkpoint_size bytes hold the parameters, the step
 * counter and the raw state, so that lbm_load + lbm_step continues
 * bit-identically. lbm_load needs a context with the same spec. */
size_t lbm_checkpoint_size(const lbm_ctx* ctx);
int lbm_save(lbm_ctx* ctx, void* host_buf, size_t size);
int lbm_load(lbm_ctx* ctx, const void* host_buf, size_t size);

/* Device view of the storage, for zero-copy use (e.g. as torch tensors).
 * base points to plane 0 of the buffer that holds the current state;
 * element (k, y, x) is at base + k*plane + y*pitch + x, in float64
 * (LBM_FP64) or float32 deviations (LBM_FP32_DEV). cs_pull_phase says how
 * the populations sit in it: 0 node order, f_k(x, t) = stored_k(x) (FD, and
 * in-place CS after an even number of steps); 1 the pull form of two-buffer
 * CS, f_k(x, t) = stored_k(x - c_k); 2 in-place CS after an odd number of
 * steps, f_k(x, t) = stored_{8-k}(x - c_k). Valid until the next lbm_step. */
typedef struct {
    void* base;
    int64_t plane;
    int32_t pitch;
    int32_t elem_bytes;
    int32_t cs_pull_phase;
    int32_t reserved;
} lbm_view;
int lbm_device_view(lbm_ctx* ctx, lbm_view* out);

/* ---- many lattices in one launch ------------------------------------------ */

/* A batch advances n independent lattices (any mix of CS/FD, sizes,
 * precisions, tau) together: each step is one persistent launch per
 * (model, q, precision) group over a work list of (lattice, tile) items,
 * and chunks of steps are replayed from a captured CUDA graph. Every
 * lattice in a batch computes exactly what it computes alone. */
typedef struct lbm_batch lbm_batch;

int lbm_batch_create(lbm_batch** out, const lbm_spec* specs, int n, void* cuda_stream);
void lbm_batch_destroy(lbm_batch* b);
int lbm_batch_size(const lbm_batch* b);
/* Initialise lattice i from host fields (as lbm_init). */
int lbm_batch_init(lbm_batch* b, int i, const double* rho, const double* ux, const double* uy);
/* Steps still to run for lattice i; lattices with 0 left are skipped by
 * later lbm_batch_step calls (default: unlimited). */
int lbm_batch_set_budget(lbm_batch* b, int i, int64_t steps);
/* Enqueue n steps for every lattice that has budget left. */
int lbm_batch_step(lbm_batch* b, int64_t n);
int lbm_batch_sync(lbm_batch* b);
int64_t lbm_batch_steps_done(const lbm_batch* b, int i);
int lbm_batch_moments(lbm_batch* b, int i, double* rho, double* ux, double* uy);
int lbm_batch_populations(lbm_batch* b, int i, double* f);
int lbm_batch_populations_region(lbm_batch* b, int i, int x0, int y0, int wx, int wy, double* f);
int lbm_batch_set_probe(lbm_batch* b, int i, int comp, const double* px, const double* py,
                        double norm);
int lbm_batch_observables(lbm_batch* b, int i, lbm_obs* out);

/* Observables recording for lattice i of a batch (as lbm_record / lbm_series). */
int lbm_batch_record(lbm_batch* b, int i, int64_t every, int64_t capacity);
int lbm_batch_series(lbm_batch* b, int i, lbm_obs* out, int64_t cap, int64_t* count);

/* The groups of a batch (one per model, q, precision) in launch order:
 * fills up to cap entries of model/q/precision (each may be NULL) and
 * returns the number of groups (-1 for a NULL batch). */
int lbm_batch_groups(lbm_batch* b, int* model, int* q, int* precision, int cap);

/* Measurement: n steps launched one kernel at a time with CUDA events around
 * every kernel (no graph). ms[g*4 + k] (cap entries, caller-owned) receives
 * the summed device time of group g's kernels of kind k: 0..2 = CS step or FD
 * stages 1..3, 3 = observables finalisation; *total_ms the span of all n
 * steps. Computes exactly what lbm_batch_step(n) computes. Synchronous. */
int lbm_batch_step_profiled(lbm_batch* b, int64_t n, double* ms, int cap, double* total_ms);

/* Kernel configuration of group `group` of a batch (lbm_batch_groups order):
 * tile variant 0 .. lbm_n_tiles(model)-1 and grid size (blocks loop over the
 * group's work items; 0 picks the default: one block per work item, i.e. per
 * tile of every lattice of the group). Every variant computes bit-identical
 * results; only speed differs. lbm_config does the same for a context. */
int lbm_batch_config(lbm_batch* b, int group, int tile, int grid);
int lbm_config(lbm_ctx* ctx, int tile, int grid);
int lbm_n_tiles(int model);

/* Number of kernels the library has enqueued for this batch / context so
 * far (nodes of replayed graphs included). */
int64_t lbm_batch_kernel_launches(const lbm_batch* b);
int64_t lbm_kernel_launches(const lbm_ctx* ctx);

/* Autotuner: times the candidate tile shapes and grid sizes of every group
 * of the batch on its current state (state is saved and restored) and keeps
 * the fastest; results are cached per (model, q, precision, size class).
 * trial_steps > 0 steps per candidate. Writes a one-line summary into
 * report (may be NULL) of report_len bytes. */
int lbm_batch_tune(lbm_batch* b, int trial_steps, char* report, size_t report_len);

/* ---- continuous-batching run server -------------------------------------- */

/* A request: one complete run of `steps` steps from an initial state:
 * init 0: Taylor-Green vortex, Sec. 4.3 Eq. (tg), density from the steady
 *         pressure balance; 1: shear wave, Sec. 4.2; 2: shock tube, Sec. 4.1,
 *         rho_l for x <= nx/2 else rho_r, fluid at rest.
 * U is the velocity amplitude in the model's units. obs_every > 0 records the
 * observables every obs_every steps (fused into the step kernels) and fits
 * the apparent viscosity of the decay (init 0 and 1); 0 records only the
 * first and last state. keep_moments != 0 keeps the final rho, u fields
 * (host memory, 24 bytes per node) for lbm_result_moments until the ticket
 * is released. user_tag is returned unchanged. */
typedef struct {
    lbm_spec spec;
    int64_t steps;
    int init;
    int obs_every;
    int keep_moments;
    int reserved;
    double U;
    double rho_l, rho_r;
    uint64_t user_tag;
} lbm_request;

/* Result of a finished request. status: LBM_OK, LBM_ENONFINITE, LBM_ECANCELLED,
 * LBM_ENOMEM (admission failed), LBM_ECUDA. Times are seconds on the server's
 * clock (since creation): latency = t_done - t_submit. nu_fit: apparent
 * viscosity gamma/(m k^2) from a log-linear fit of the recorded amplitude
 * (m = 1 shear, 2 Taylor-Green; Sec. 4.2-4.3), in the model's units; 0 when
 * not available. */
typedef struct {
    int status;
    int reserved;
    uint64_t user_tag;
    int64_t steps;
    lbm_obs first, last;
    double nu_fit;
    double t_submit, t_admit, t_done;
    int64_t n_series;
} lbm_result;

typedef struct lbm_server lbm_server;

/* Start a server. hbm_budget_bytes bounds the summed device footprint of
 * resident runs (admission control); max_slots bounds their number. Runs go
 * to one of two lanes by an estimate of their step's device time (from the
 * lattice size, model, velocity set and precision): large runs (a step of
 * about 0.5 ms or more, e.g. a 16-velocity FD lattice from 2048^2 nodes) and
 * small runs. Each lane has a worker thread and its own CUDA stream, the
 * small runs' at the device's highest priority and the large runs' at the
 * lowest, so the two lanes' kernels share the GPU at the same time and a
 * large run is not throttled by the small runs' rounds. Within a lane,
 * resident runs advance together in scheduling rounds that give each run
 * about the same device time: the run with the cheapest step advances the
 * lane's chunk (chunk_steps for small runs, chunk_steps / 8 for large ones)
 * per round, a run whose step costs m times as much advances chunk / m (at
 * least 1), none more than it has left. Requests admitted while others run
 * join their lane's next round. cuda_stream: NULL for the two streams the
 * server creates, or a cudaStream_t on which the server then runs a single
 * lane for all runs. A server is thread-safe. LBM_EINVAL for a null out, a
 * zero budget, max_slots < 1 or chunk_steps < 1; LBM_ENOMEM or LBM_ECUDA if
 * the engines cannot be set up (*out is then null). */
int lbm_server_create(lbm_server** out, size_t hbm_budget_bytes, int max_slots, int chunk_steps,
                      void* cuda_stream);
/* Queue a request and return at once with its ticket. LBM_EINVAL / LBM_ECFL /
 * LBM_ESTIFF for a bad spec (as lbm_create), LBM_ENOMEM if its footprint
 * exceeds the whole budget. */
int lbm_submit(lbm_server* s, const lbm_request* req, uint64_t* ticket);
/* LBM_ENOTREADY until the run finished, then LBM_OK and *out filled;
 * LBM_ENOTFOUND for an unknown ticket. */
int lbm_poll(lbm_server* s, uint64_t ticket, lbm_result* out);
/* Copy up to cap recorded observables of a finished run; *count receives how
 * many there are. */
int lbm_result_series(lbm_server* s, uint64_t ticket, lbm_obs* out, int64_t cap, int64_t* count);
/* Final fields of a finished run submitted with keep_moments: rho, ux, uy
 * (host [ny][nx] each, caller-owned), Eq. (f_moments_discrete) of its last
 * state. LBM_ENOTREADY while the run is not finished, LBM_ENOTFOUND for an
 * unknown or released ticket or a run without kept fields (or one that
 * failed before its end). */
int lbm_result_moments(lbm_server* s, uint64_t ticket, double* rho, double* ux, double* uy);
/* Forget a finished request: its result, series and kept fields are freed
 * and later calls with its ticket return LBM_ENOTFOUND. A server keeps every
 * finished result until it is released (or the server is destroyed), so a
 * long-lived server should release what it has read. LBM_ENOTREADY for a
 * queued or running request, LBM_ENOTFOUND for an unknown ticket. */
int lbm_release(lbm_server* s, uint64_t ticket);
/* Cancel a queued or running request (a running one stops at the end of the
 * current round with status LBM_ECANCELLED). */
int lbm_cancel(lbm_server* s, uint64_t ticket);
/* Wait until every submitted request finished, or timeout_s (LBM_ETIMEOUT). */
int lbm_server_drain(lbm_server* s, double timeout_s);
/* Queued, running and finished (not yet released) counts and resident
 * device bytes. */
int lbm_server_stats(lbm_server* s, int64_t* queued, int64_t* running, int64_t* finished,
                     size_t* resident_bytes);
/* Cancel what is left, stop the worker and free everything. */
void lbm_server_destroy(lbm_server* s);
/* The steps each of n runs advances in one scheduling round of a server with
 * chunk_steps (the rule of lbm_server_create): specs[i] the run's lattice,
 * left[i] >= 0 the steps it has still to run; steps[i] receives its
 * allotment (0 only when left[i] is 0). Host arrays, caller-owned; no device
 * work. For callers that schedule their own batches (lbm_batch_set_budget)
 * the same way. LBM_EINVAL for n < 0, chunk_steps < 1, a null array with
 * n > 0 or a negative left[i]; a bad spec returns what lbm_create returns. */
int lbm_server_plan_round(const lbm_spec* specs, const int64_t* left, int n, int chunk_steps, int64_t* steps);
/* Device bytes a lattice of this spec holds (its state buffers and the
 * per-lattice observables scratch): the footprint the server admits runs by
 * against its HBM budget, and what lbm_create allocates for the state.
 * Host only (no device work). Two-buffer CS keeps two copies of the 9
 * planes, in-place CS one; FD three copies of the Q^2 planes (RK3: f^n and
 * two stage buffers; IMEX: f^n, Z and P) and two with LBM_TS_RK3_FUSED.
 * A bad spec returns what lbm_create returns; *bytes is then not written. */
int lbm_footprint(const lbm_spec* spec, size_t* bytes);

/* Test injection of a device-side wait that runs out (no counterpart in the
 * paper; failure detection of the library itself). The CS bulk-copy kernel
 * (the default CS kernel; the only one with device-side waits) bounds every
 * mbarrier wait by 2 s of device time; with microseconds > 0, every wait of
 * the following CS launches is bounded by that many microseconds and the
 * first block skips the copies of its first row, so that row's consumers wait
 * on a barrier that nothing completes. The wait runs out, the launch sets the
 * group's error word and finishes (no fault, no unbounded wait, copies in
 * flight land first), and lbm_sync / lbm_batch_sync return LBM_ETIMEOUT; the
 * state of that step is invalid. 0 turns the injection off. Range 0..1e6,
 * else LBM_EINVAL. The server variant applies from the next round and fails
 * the runs of that round with LBM_ETIMEOUT (reported by lbm_poll). */
int lbm_inject_wait_timeout(lbm_ctx* ctx, int microseconds);
int lbm_batch_inject_wait_timeout(lbm_batch* b, int microseconds);
int lbm_server_inject_wait_timeout(lbm_server* s, int microseconds);

/* ---- observables without allocation ------------------------------------------
 * The paper has no counterpart to this entry point; it serves callers that
 * cannot allocate device memory: hosts that hand the library a fixed memory
 * arena and forbid any further allocation (an embedding application that
 * owns all device memory), and latency-sensitive loops where a cudaMalloc
 * would synchronise the device and stall the work in flight.
 *
 * It computes what lbm_observables computes (float64 mass, momentum and
 * probe amplitude) for a state in caller-owned device memory, and allocates
 * nothing: no cudaMalloc, cudaFree or allocating library call. Its scratch
 * (block partial sums) is a file-scope device array of 1024 x 4 doubles
 * (32 KiB) that every GPU loading the library holds until the process exits;
 * larger lattices are covered by fewer, longer-striding blocks.
 *
 *  state: device pointer; element (k, y, x) at state + k*plane + y*pitch + x,
 *      float64 full f (LBM_FP64) or float32 f - w_k rho0 (LBM_FP32_DEV).
 *  cs_phase: how the populations sit in state, the value lbm_device_view
 *      reports in cs_pull_phase: 0 node order, f_k(x) = stored_k(x) (FD, and
 *      in-place CS after an even number of steps); 1 pull form of two-buffer
 *      CS, f_k(x) = stored_k(x - c_k); 2 in-place CS after an odd number of
 *      steps, f_k(x) = stored_{8-k}(x - c_k). LBM_EINVAL outside 0..2, or
 *      non-zero for FD.
 *  comp: -1 for no probe, else 0 (u_x) / 1 (u_y) with device tables px[nx],
 *      py[ny] and norm as in lbm_set_probe.
 *  step, dt: copied into the record (time = step * dt).
 *  out: device pointer to one lbm_obs, written asynchronously on cuda_stream
 *      (NULL = legacy default stream); the call returns after enqueueing.
 * Limits: nx*ny < 2^31, pitch >= nx, plane >= pitch*ny; LBM_EINVAL otherwise.
 * The first call on a device looks up the array's device address with that
 * device current (once per device); make that first call before any stream
 * capture. Every call shares the one array and overwrites all of it that it
 * reads, so calls do not depend on each other's leftovers, but calls that
 * overlap on the GPU (different streams, no ordering) race on the array. */
int lbm_observables_noalloc(int model, int q_per_axis, int precision, int nx, int ny, const void* state,
                            int64_t plane, int32_t pitch, int32_t cs_phase, double rho0, int comp, const double* px,
                            const double* py, double norm, int64_t step, double dt, lbm_obs* out,
                            void* cuda_stream);

/* ---- measurement support ------------------------------------------------------
 * Measured FP32 rate of the current device (no counterpart in the paper; the
 * denominator of the FD stage kernel's arithmetic roofline): independent
 * chains of fused multiply-adds on every SM, two per instruction (packed
 * FP32x2, as the FD kernel uses) when packed != 0, else one; timed with CUDA
 * events over 10 launches after a warm-up. Writes flops per second (two per
 * multiply-add), the device's SM count (may be NULL) and the mean launch time
 * (may be NULL). Synchronous; allocates and frees a small output buffer. */
int lbm_probe_fp32(int packed, double* flops_per_s, int* sm_count, double* ms_per_launch);

/* ---- errors ---------------------------------------------------------------- */
const char* lbm_strerror(int code);
const char* lbm_last_error(void);
/* Library version string. */
const char* lbm_version(void);

#ifdef __cplusplus
}
#endif
#endif /* LBM_H */
