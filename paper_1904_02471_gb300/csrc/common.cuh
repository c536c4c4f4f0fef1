// Device-side definitions shared by the CS and FD kernels.
//
// Work model: a "group" is a set of lattices with the same model, velocity
// set and storage type. Every kernel is persistent over a flat list of work
// items (one item = one tile of one lattice); item -> lattice by binary
// search of the lattices' first items. A single lattice is a group of one.
//
// Per-lattice dynamic state (which CS buffer is current, steps done, steps
// left) lives in the device descriptor and is advanced on the device at the
// end of every chunk of steps, so a captured chunk can be replayed as a CUDA
// graph any number of times.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/lbm.h"

namespace lbm {

constexpr int NOBS = 4;  // sum rho (minus the storage offset), sum j_x, sum j_y, probe sum

struct LatDesc {
    void* buf[3];           // CS: buf[0]/buf[1] ping-pong; FD: f^n, f^(1), f^(2)
    int nx, ny;
    int pitch;              // row pitch in elements (multiple of 32)
    int tiles_x;            // tiles along x for the group's tile shape
    long long plane;        // elements per population plane
    int item_begin;         // first work item of this lattice in its group
    int items;              // number of work items
    int cur;                // CS: index (0/1) of the buffer holding the state; in place: the phase
    int inplace;            // CS: one buffer updated in place (AA pattern)
    int obs_every;          // record observables when (step - obs_base) % obs_every == 0 (0: off)
    long long obs_base;     // step at which recording started
    long long step0;        // steps completed
    long long remaining;    // steps still to run (skipped when exhausted)
    double omega;           // CS: dt / tau_LU
    double cdx;             // FD: dt / dx
    double dt_tau;          // FD: dt / tau_FD
    double rho0;            // storage offset: populations stored as f - w_k rho0 (0 for FP64)
    double eps;             // FD: WENO epsilon
    double dt;              // time step, for time stamps
    int probe_comp;         // 0: u_x, 1: u_y, -1: no probe
    int obs_cap;            // capacity of the series
    double probe_norm;
    const double* probe_px;   // [nx]
    const double* probe_py;   // [ny]
    const float* probe_pxf;   // float copies for FP32 kernels
    const float* probe_pyf;
    double* partials;       // [items][NOBS], this lattice's slice
    lbm_obs* series;        // [obs_cap]
    double* snap;           // [NOBS] result of a one-off observables reduction
    // float copies of omega, cdx, dt_tau, rho0, eps for the FP32 kernels (a
    // conversion from double would run on the narrow FP64 pipe every tile)
    float omega_f, cdx_f, dt_tau_f, rho0_f, eps_f;
    int* err;               // the group's error word (header word 2)
};

// State buffers: element (0, 0) of a buffer sits STATE_HEAD elements into its
// slot of the lattice's allocation and every slot ends with STATE_TAIL spare
// elements (row segments of bulk copies may reach into them).
constexpr long long STATE_HEAD = 4, STATE_TAIL = 1024;

// Error bits of the group error word: an access outside a state buffer caught
// by the bounds-checked build; an input value rejected by the state
// initialisation kernels (rho <= 0 or a non-finite value).
constexpr int ERR_BOUNDS = 2;
constexpr int ERR_INPUT = 4;

// Bounds-checked build (-DLBM_BOUNDS_CHECK; compute-sanitizer stand-in): a
// single-element access to a state buffer must hit a node of the lattice
// (population < K, row < ny, column < nx), a bulk row copy must stay inside
// the buffer's slot of the allocation. A failing check skips the access and
// sets ERR_BOUNDS; nothing traps. Without the flag the checks compile away.
#ifdef LBM_BOUNDS_CHECK
__device__ __forceinline__ bool bc_report(const LatDesc* d) {
    atomicOr(d->err, ERR_BOUNDS);
    return false;
}
__device__ __forceinline__ bool bc_node(const LatDesc* d, int K, long long off) {
    bool ok = off >= 0 && off < (long long)K * d->plane;
    if (ok) {
        const long long r = off % d->plane;
        ok = (r % d->pitch) < d->nx && (r / d->pitch) < d->ny;
    }
    return ok || bc_report(d);
}
__device__ __forceinline__ bool bc_span(const LatDesc* d, int K, long long off, long long n) {
    return (off >= -STATE_HEAD && off + n <= (long long)K * d->plane + STATE_TAIL) || bc_report(d);
}
#define LBM_BC_NODE(d, K, off) bc_node((d), (K), (off))
#define LBM_BC_SPAN(d, K, off, n) bc_span((d), (K), (off), (n))
#else
#define LBM_BC_NODE(d, K, off) true
#define LBM_BC_SPAN(d, K, off, n) true
#endif

// A per-lattice constant in the kernel's precision.
template <typename T>
__device__ __forceinline__ T lat_val(double d, float f);
template <>
__device__ __forceinline__ double lat_val<double>(double d, float) { return d; }
template <>
__device__ __forceinline__ float lat_val<float>(double, float f) { return f; }

// ---------------------------------------------------------------------------
// Gauss-Hermite nodes and weights (probabilists', weights summing to 1):
//   3 nodes: 0, +-sqrt(3); w = 2/3, 1/6 (the D2Q9 set of Sec. 2)
//   4 nodes: +-sqrt(3 -+ sqrt 6); w = (3 +- sqrt 6)/12
//   5 nodes: 0, +-sqrt(5 -+ sqrt 10); w = 8/15, (7 +- 2 sqrt 10)/60
// Values are the closed forms evaluated to 21 digits. Index i runs over the
// nodes in ascending order. All functions fold to immediates when i is a
// compile-time constant (fully unrolled population loops).
// ---------------------------------------------------------------------------
template <int Q1>
struct GH;

template <>
struct GH<3> {
    static __host__ __device__ constexpr double v(int i) {
        return i == 0 ? -1.73205080756887729353 : (i == 1 ? 0.0 : 1.73205080756887729353);
    }
    static __host__ __device__ constexpr double w(int i) { return i == 1 ? 2.0 / 3.0 : 1.0 / 6.0; }
    static __host__ __device__ constexpr double vmax() { return 1.73205080756887729353; }
};

template <>
struct GH<4> {
    static __host__ __device__ constexpr double v(int i) {
        return i == 0 ? -2.33441421833897723932
                      : (i == 1 ? -0.741963784302725857649
                                : (i == 2 ? 0.741963784302725857649 : 2.33441421833897723932));
    }
    static __host__ __device__ constexpr double w(int i) {
        return (i == 0 || i == 3) ? 0.0458758547680684918169 : 0.454124145231931508183;
    }
    static __host__ __device__ constexpr double vmax() { return 2.33441421833897723932; }
};

template <>
struct GH<5> {
    static __host__ __device__ constexpr double v(int i) {
        return i == 0 ? -2.85697001387280565416
                      : (i == 1 ? -1.35562617997426586583
                                : (i == 2 ? 0.0
                                          : (i == 3 ? 1.35562617997426586583 : 2.85697001387280565416)));
    }
    static __host__ __device__ constexpr double w(int i) {
        return (i == 0 || i == 4) ? 0.0112574113277206889334
                                  : ((i == 1 || i == 3) ? 0.2220759220056126444 : 0.533333333333333333333);
    }
    static __host__ __device__ constexpr double vmax() { return 2.85697001387280565416; }
};

// Population k = ix + Q1*iy of the product set.
template <int Q1>
__host__ __device__ constexpr double vx_of(int k) { return GH<Q1>::v(k % Q1); }
template <int Q1>
__host__ __device__ constexpr double vy_of(int k) { return GH<Q1>::v(k / Q1); }
template <int Q1>
__host__ __device__ constexpr double w_of(int k) { return GH<Q1>::w(k % Q1) * GH<Q1>::w(k / Q1); }
// D2Q9 lattice vector c_k = v_k dt/dx in {-1, 0, 1}.
__host__ __device__ constexpr int c3_of(int i) { return i - 1; }

// ---------------------------------------------------------------------------
// Work-item lookup: the lattice whose item range holds `item`.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int find_lattice(const int* __restrict__ item_begin, int n, int item) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (__ldg(item_begin + mid) <= item) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Last item of this block's sequence (first item `item`, stride gridDim.x)
// that still belongs to lattice d. A lattice that sits out a step (its step
// budget is spent) is passed over in one jump: the item loop continues from
// there, so its tiles cost nothing however many there are.
__device__ __forceinline__ int last_item_of(const LatDesc& d, int item) {
    const int stride = (int)gridDim.x;
    return item + (d.item_begin + d.items - 1 - item) / stride * stride;
}

// Observe the state at sub-step j of this chunk?
__device__ __forceinline__ bool observe_now(const LatDesc& d, int j) {
    if (d.obs_every <= 0) return false;
    const long long s = d.step0 + j - d.obs_base;
    return s >= 0 && (s % d.obs_every) == 0 && (s / d.obs_every) < d.obs_cap;
}


// Block reduction of NOBS per-thread partial sums into out[NOBS] (double).
// Warp level in T (for FP32 storage: at most 32 per-thread sums in float),
// across warps in double, fixed order (deterministic).
// Must be called by all threads of the block. With TRAILING_SYNC false the
// caller guarantees a barrier before `smem` is written again.
template <typename T, int NT, bool TRAILING_SYNC = true>
__device__ __forceinline__ void block_reduce_obs(const T (&v)[NOBS], double* out, double* smem) {
    constexpr int NW = NT / 32;
    T r[NOBS];
#pragma unroll
    for (int q = 0; q < NOBS; ++q) {
        T x = v[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        r[q] = x;
    }
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    if (lane == 0) {
#pragma unroll
        for (int q = 0; q < NOBS; ++q) smem[warp * NOBS + q] = (double)r[q];
    }
    __syncthreads();
    if (tid < NOBS) {
        double s = 0.0;
        for (int w = 0; w < NW; ++w) s += smem[w * NOBS + tid];
        out[tid] = s;
    }
    if constexpr (TRAILING_SYNC) __syncthreads();
}

}  // namespace lbm
