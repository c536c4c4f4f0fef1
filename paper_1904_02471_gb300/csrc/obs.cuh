// Device helpers of the observables readouts (the library's snapshot and
// the allocation-free entry point share them): where a state keeps each
// population, per-node moments, deterministic row sums and the record.
#pragma once

#include "common.cuh"

namespace lbm {

// ---------------------------------------------------------------------------
// Where a state keeps f_k(x) (the phases lbm_view::cs_pull_phase names):
//   phase 0, node order: plane k, node x (FD; in-place CS after an even
//            number of steps);
//   phase 1, pull form: plane k, node x - c_k (two-buffer CS);
//   phase 2, mirrored pull form: plane K-1-k (the opposite velocity), node
//            x - c_k (in-place CS after an odd number of steps).
// c_k is the D2Q9 lattice vector; shifts exist only for the 3-node set.
// ---------------------------------------------------------------------------
struct StoreMap {
    bool shift;
    bool mirror;
};
__host__ __device__ constexpr StoreMap store_map_of_phase(int phase) {
    return StoreMap{phase != 0, phase == 2};
}
// Phase of a lattice descriptor's current state; pull = CS.
__device__ __forceinline__ int desc_phase(const LatDesc* d, bool pull) {
    return !pull ? 0 : (!d->inplace ? 1 : (d->cur ? 2 : 0));
}

// Offset of f_k at node (x, y) in a buffer of the given layout.
template <int Q1>
__device__ __forceinline__ long long stored_offset(StoreMap m, int k, int x, int y, int nx, int ny,
                                                   long long plane, int pitch) {
    constexpr int K = Q1 * Q1;
    int xs = x, ys = y;
    if (Q1 == 3 && m.shift) {
        xs = x - c3_of(k % Q1);
        ys = y - c3_of(k / Q1);
        xs = xs < 0 ? xs + nx : (xs >= nx ? xs - nx : xs);
        ys = ys < 0 ? ys + ny : (ys >= ny ? ys - ny : ys);
    }
    return (long long)(m.mirror ? K - 1 - k : k) * plane + (long long)ys * pitch + xs;
}

// Moments of one node in the storage precision, Eq. (f_moments_discrete):
// dr = sum of stored values (rho minus the storage offset), j = sum v_k
// times stored value, population k ascending. ok(off) is the bounds check of
// an access (a skipped access reads 0).
template <typename T, int Q1, typename OK>
__device__ __forceinline__ void stored_node_moments(const T* __restrict__ in, StoreMap m, int x, int y, int nx,
                                                    int ny, long long plane, int pitch, T& dr, T& jx, T& jy,
                                                    OK ok) {
    constexpr int K = Q1 * Q1;
    dr = T(0);
    jx = T(0);
    jy = T(0);
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const long long off = stored_offset<Q1>(m, k, x, y, nx, ny, plane, pitch);
        const T s = ok(off) ? in[off] : T(0);
        dr += s;
        if (vx_of<Q1>(k) != 0.0) jx += s * (T)vx_of<Q1>(k);
        if (vy_of<Q1>(k) != 0.0) jy += s * (T)vy_of<Q1>(k);
    }
}

// Deterministic block sum of n rows of NOBS doubles into out[NOBS]
// (sm: blockDim.x * NOBS doubles). Called by every thread of the block.
__device__ __forceinline__ void sum_rows(const double* __restrict__ p, long long n, double* out, double* sm) {
    double a[NOBS] = {0.0, 0.0, 0.0, 0.0};
    for (long long i = threadIdx.x; i < n; i += blockDim.x)
#pragma unroll
        for (int q = 0; q < NOBS; ++q) a[q] += p[i * NOBS + q];
#pragma unroll
    for (int q = 0; q < NOBS; ++q) sm[threadIdx.x * NOBS + q] = a[q];
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s)
#pragma unroll
            for (int q = 0; q < NOBS; ++q) sm[threadIdx.x * NOBS + q] += sm[(threadIdx.x + s) * NOBS + q];
        __syncthreads();
    }
    if (threadIdx.x < NOBS) out[threadIdx.x] = sm[threadIdx.x];
}

// The observables record of a state from its NOBS global sums.
__device__ __forceinline__ lbm_obs make_obs(long long step, double dt, int nx, int ny, double rho0, int probe_comp,
                                            double probe_norm, const double* tot) {
    lbm_obs o;
    o.step = step;
    o.time = (double)step * dt;
    o.mass = (double)nx * (double)ny * rho0 + tot[0];
    o.mom_x = tot[1];
    o.mom_y = tot[2];
    o.amp = probe_comp >= 0 ? probe_norm * tot[3] : 0.0;
    o.nonfinite = (isfinite(o.mass) && isfinite(o.amp) && isfinite(o.mom_x) && isfinite(o.mom_y)) ? 0 : 1;
    o.reserved = 0;
    return o;
}

}  // namespace lbm
