// State initialisation, readout and observables reductions.
//
// CS lattices with two buffers are stored in the pull phase: stored_k(m) =
// f*_k(m, t-1), the post-collision value at m that streams to m + c_k, so the
// pre-collision state of Eq. (sc_evolution) is f_k(x, t) = stored_k(x - c_k).
// Writing a state f therefore stores f_k(x) at x - c_k; reading gathers from
// x - c_k. In-place CS lattices (one buffer) hold f_k(x) at plane k, node x
// after an even number of steps and at plane 8 - k, node x - c_k after an odd
// number. FD lattices store f^n as is. Deviation storage adds / removes w_k rho0.
//
// Global sums (mass, momentum, probe amplitude) are float64 from the first
// addition on here, reduced block-wise into partials and then in a fixed
// order by a single block (deterministic).
#include "kernels.h"
#include "obs.cuh"

namespace lbm {

// Buffer that holds a lattice's current state: the current one of the pair
// (two-buffer CS, temporally blocked FD); buffer 0 for in-place CS, and for
// RK3 / IMEX FD, whose cur stays 0.
template <bool PULL>
__device__ __forceinline__ int store_buf(const LatDesc* d) {
    return PULL && d->inplace ? 0 : d->cur;
}

template <typename T, int Q1, bool PULL>
__global__ void init_eq_kernel(const LatDesc* d, int nx, int ny, const double* __restrict__ rho,
                               const double* __restrict__ ux, const double* __restrict__ uy) {
    constexpr int K = Q1 * Q1;
    const long long plane = d->plane;
    const int pitch = d->pitch;
    const double r0 = d->rho0;
    const StoreMap m = store_map_of_phase(desc_phase(d, PULL));
    T* __restrict__ out = static_cast<T*>(d->buf[store_buf<PULL>(d)]);
    const long long n = (long long)nx * ny;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(c % nx), y = (int)(c / nx);
        const double rd = rho[c], ud = ux[c], vd = uy[c];
        // input check on the device (every value is read here anyway)
        if (!(rd > 0.0) || !isfinite(rd) || !isfinite(ud) || !isfinite(vd)) atomicOr(d->err, ERR_INPUT);
        // arithmetic in the storage precision: float for the deviation
        // storage, whose rho - rho0 is formed in double first
        const T dr = (T)(rd - r0), r = (T)rd, u = (T)ud, v = (T)vd;
        const T usq = u * u + v * v;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const T xi = (T)vx_of<Q1>(k) * u + (T)vy_of<Q1>(k) * v;
            // Eq. (herfeq) minus the storage offset w_k rho0
            const T dev = (T)w_of<Q1>(k) * (dr + r * (xi + T(0.5) * (xi * xi - usq)));
            const long long off = stored_offset<Q1>(m, k, x, y, nx, ny, plane, pitch);
            if (LBM_BC_NODE(d, K, off)) out[off] = (T)dev;
        }
    }
}

template <typename T, int Q1, bool PULL>
__global__ void set_pop_kernel(const LatDesc* d, int nx, int ny, const double* __restrict__ f) {
    constexpr int K = Q1 * Q1;
    const long long plane = d->plane;
    const int pitch = d->pitch;
    const double r0 = d->rho0;
    const StoreMap m = store_map_of_phase(desc_phase(d, PULL));
    T* __restrict__ out = static_cast<T*>(d->buf[store_buf<PULL>(d)]);
    const long long n = (long long)nx * ny;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(c % nx), y = (int)(c / nx);
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const long long off = stored_offset<Q1>(m, k, x, y, nx, ny, plane, pitch);
            const double fv = f[k * n + c];
            if (!isfinite(fv)) atomicOr(d->err, ERR_INPUT);
            if (LBM_BC_NODE(d, K, off)) out[off] = (T)(fv - w_of<Q1>(k) * r0);
        }
    }
}

constexpr int IO_THREADS = 256;

template <typename T, int Q1, bool PULL>
__global__ void __launch_bounds__(IO_THREADS) readout_kernel(const LatDesc* d, int nx, int ny, int x0, int y0, int wx,
                                                             int wy, double* __restrict__ f, double* __restrict__ rho,
                                                             double* __restrict__ ux, double* __restrict__ uy,
                                                             double* __restrict__ part) {
    constexpr int K = Q1 * Q1;
    __shared__ double red[(IO_THREADS / 32) * NOBS];
    const long long plane = d->plane;
    const int pitch = d->pitch;
    const double r0 = d->rho0;
    const StoreMap m = store_map_of_phase(desc_phase(d, PULL));
    const T* __restrict__ in = static_cast<const T*>(d->buf[store_buf<PULL>(d)]);
    const int pc = d->probe_comp;
    const long long n = (long long)wx * wy;
    double acc[NOBS] = {0.0, 0.0, 0.0, 0.0};
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        int x = x0 + (int)(c % wx), y = y0 + (int)(c / wx);
        x %= nx;
        y %= ny;
        double dr = 0.0, jx = 0.0, jy = 0.0;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const long long off = stored_offset<Q1>(m, k, x, y, nx, ny, plane, pitch);
            const double s = LBM_BC_NODE(d, K, off) ? (double)in[off] : 0.0;
            if (f) f[k * n + c] = s + w_of<Q1>(k) * r0;
            dr += s;
            jx += s * vx_of<Q1>(k);
            jy += s * vy_of<Q1>(k);
        }
        const double r = r0 + dr;
        const double u = jx / r, v = jy / r;
        if (rho) {
            rho[c] = r;
            ux[c] = u;
            uy[c] = v;
        }
        acc[0] += dr;
        acc[1] += jx;
        acc[2] += jy;
        if (pc >= 0) acc[3] += (pc == 0 ? u : v) * d->probe_px[x] * d->probe_py[y];
    }
    if (part) block_reduce_obs<double, IO_THREADS>(acc, part + (long long)blockIdx.x * NOBS, red);
}

// Observables of the whole lattice (no readout): per node the moments in the
// storage precision and, for the probed component only, the velocity; from
// there on float64 (per-thread sums, block reduction, two-level finalise).
template <typename T, int Q1, bool PULL>
__global__ void __launch_bounds__(IO_THREADS) obs_snapshot_kernel(const LatDesc* d, int nx, int ny,
                                                                  double* __restrict__ part) {
    [[maybe_unused]] constexpr int K = Q1 * Q1;   // used by the bounds-checked build
    __shared__ double red[(IO_THREADS / 32) * NOBS];
    const long long plane = d->plane;
    const int pitch = d->pitch;
    const T r0 = (T)d->rho0;
    const StoreMap m = store_map_of_phase(desc_phase(d, PULL));
    const T* __restrict__ in = static_cast<const T*>(d->buf[store_buf<PULL>(d)]);
    const int pc = d->probe_comp;
    const long long n = (long long)nx * ny;
    double acc[NOBS] = {0.0, 0.0, 0.0, 0.0};
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(c % nx), y = (int)(c / nx);
        T dr, jx, jy;
        stored_node_moments<T, Q1>(in, m, x, y, nx, ny, plane, pitch, dr, jx, jy,
                                   [&](long long off) { return LBM_BC_NODE(d, K, off); });
        acc[0] += (double)dr;
        acc[1] += (double)jx;
        acc[2] += (double)jy;
        if (pc >= 0) acc[3] += (double)((pc == 0 ? jx : jy) / (r0 + dr)) * d->probe_px[x] * d->probe_py[y];
    }
    block_reduce_obs<double, IO_THREADS>(acc, part + (long long)blockIdx.x * NOBS, red);
}

constexpr int FIN_THREADS = 256;

__global__ void __launch_bounds__(FIN_THREADS) snap_finalize_kernel(LatDesc* d, const double* part, int nblocks) {
    __shared__ double sm[FIN_THREADS * NOBS];
    __shared__ double tot[NOBS];
    sum_rows(part, nblocks, tot, sm);
    __syncthreads();
    if (threadIdx.x < NOBS) d->snap[threadIdx.x] = tot[threadIdx.x];
}

__device__ void write_record(LatDesc* d, long long step, const double* tot) {
    d->series[(step - d->obs_base) / d->obs_every] =
        make_obs(step, d->dt, d->nx, d->ny, d->rho0, d->probe_comp, d->probe_norm, tot);
}

// Two-level reduction of the tile partials of every lattice observing at
// sub-step j: chunk sums (grid max_lat x nchunks), then one block per lattice
// sums its chunks in order and writes the record.
__global__ void __launch_bounds__(FIN_THREADS) obs_chunk_kernel(GroupDev g, int j, int nchunks, double* chunks) {
    __shared__ double sm[FIN_THREADS * NOBS];
    __shared__ double tot[NOBS];
    const int li = blockIdx.x / nchunks, ch = blockIdx.x - li * nchunks;
    if (li >= g.hdr[0]) return;
    const LatDesc* d = g.desc + li;
    if ((long long)j >= d->remaining || !observe_now(*d, j)) return;
    const long long len = (d->items + nchunks - 1) / nchunks;
    const long long lo = ch * len;
    const long long hi = lo + len < d->items ? lo + len : d->items;
    sum_rows(d->partials + lo * NOBS, hi > lo ? hi - lo : 0, tot, sm);
    __syncthreads();
    if (threadIdx.x < NOBS) chunks[((long long)li * nchunks + ch) * NOBS + threadIdx.x] = tot[threadIdx.x];
}

__global__ void __launch_bounds__(FIN_THREADS) obs_finalize_kernel(GroupDev g, int j, int nchunks, const double* chunks) {
    __shared__ double sm[FIN_THREADS * NOBS];
    __shared__ double tot[NOBS];
    const int li = blockIdx.x;
    if (li >= g.hdr[0]) return;
    LatDesc* d = g.desc + li;
    if ((long long)j >= d->remaining || !observe_now(*d, j)) return;
    sum_rows(chunks + (long long)li * nchunks * NOBS, nchunks, tot, sm);
    __syncthreads();
    if (threadIdx.x == 0) write_record(d, d->step0 + j, tot);
}

__global__ void advance_kernel(GroupDev g, int c, int flip) {
    const int li = blockIdx.x * blockDim.x + threadIdx.x;
    if (li >= g.hdr[0]) return;
    LatDesc* d = g.desc + li;
    const long long adv = d->remaining < (long long)c ? d->remaining : (long long)c;
    d->step0 += adv;
    d->remaining -= adv;
    if (flip && (adv & 1)) d->cur ^= 1;
}

// ---------------------------------------------------------------------------
static int io_grid(long long n) {
    long long b = (n + IO_THREADS - 1) / IO_THREADS;
    if (b > 4096) b = 4096;
    return (int)(b < 1 ? 1 : b);
}

#define LBM_DISPATCH_Q(q1, pull, PREC, BODY)                            \
    do {                                                                \
        if (precision == LBM_FP64) {                                    \
            using T = double;                                           \
            if (q1 == 3 && pull) { constexpr int Q = 3; constexpr bool P = true; BODY; } \
            else if (q1 == 3) { constexpr int Q = 3; constexpr bool P = false; BODY; }   \
            else if (q1 == 4) { constexpr int Q = 4; constexpr bool P = false; BODY; }   \
            else if (q1 == 5) { constexpr int Q = 5; constexpr bool P = false; BODY; }   \
            else return cudaErrorInvalidValue;                          \
        } else {                                                        \
            using T = float;                                            \
            if (q1 == 3 && pull) { constexpr int Q = 3; constexpr bool P = true; BODY; } \
            else if (q1 == 3) { constexpr int Q = 3; constexpr bool P = false; BODY; }   \
            else if (q1 == 4) { constexpr int Q = 4; constexpr bool P = false; BODY; }   \
            else if (q1 == 5) { constexpr int Q = 5; constexpr bool P = false; BODY; }   \
            else return cudaErrorInvalidValue;                          \
        }                                                               \
    } while (0)

cudaError_t launch_init_equilibrium(int precision, int q1, int pull, const LatDesc* d, int nx, int ny,
                                    const double* rho, const double* ux, const double* uy, cudaStream_t s) {
    const int grid = io_grid((long long)nx * ny);
    LBM_DISPATCH_Q(q1, pull, precision, (init_eq_kernel<T, Q, P><<<grid, IO_THREADS, 0, s>>>(d, nx, ny, rho, ux, uy)));
    return cudaGetLastError();
}

cudaError_t launch_set_populations(int precision, int q1, int pull, const LatDesc* d, int nx, int ny,
                                   const double* f, cudaStream_t s) {
    const int grid = io_grid((long long)nx * ny);
    LBM_DISPATCH_Q(q1, pull, precision, (set_pop_kernel<T, Q, P><<<grid, IO_THREADS, 0, s>>>(d, nx, ny, f)));
    return cudaGetLastError();
}

cudaError_t launch_readout(int precision, int q1, int pull, const LatDesc* d, int nx, int ny, int x0, int y0, int wx,
                           int wy, double* f, double* rho, double* ux, double* uy, double* part, int nblocks,
                           cudaStream_t s) {
    int grid = io_grid((long long)wx * wy);
    if (part && grid > nblocks) grid = nblocks;
    if (part && !f && !rho && x0 == 0 && y0 == 0 && wx == nx && wy == ny)
        LBM_DISPATCH_Q(q1, pull, precision, (obs_snapshot_kernel<T, Q, P><<<grid, IO_THREADS, 0, s>>>(d, nx, ny, part)));
    else
        LBM_DISPATCH_Q(q1, pull, precision,
                       (readout_kernel<T, Q, P><<<grid, IO_THREADS, 0, s>>>(d, nx, ny, x0, y0, wx, wy, f, rho, ux, uy,
                                                                              part)));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !part) return e;
    snap_finalize_kernel<<<1, FIN_THREADS, 0, s>>>(const_cast<LatDesc*>(d), part, grid);
    return cudaGetLastError();
}

cudaError_t launch_obs_finalize(const GroupDev& g, int max_lat, int nchunks, double* chunks, int j, cudaStream_t s) {
    if (max_lat <= 0) return cudaSuccess;
    obs_chunk_kernel<<<max_lat * nchunks, FIN_THREADS, 0, s>>>(g, j, nchunks, chunks);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    obs_finalize_kernel<<<max_lat, FIN_THREADS, 0, s>>>(g, j, nchunks, chunks);
    return cudaGetLastError();
}

cudaError_t launch_advance(const GroupDev& g, int max_lat, int c, int flip_phase, cudaStream_t s) {
    if (max_lat <= 0) return cudaSuccess;
    advance_kernel<<<(max_lat + 127) / 128, 128, 0, s>>>(g, c, flip_phase);
    return cudaGetLastError();
}

}  // namespace lbm
