// Allocation-free observables of a lattice state held in caller memory.
//
// Some callers cannot call cudaMalloc: code running while a stream is being
// captured into a CUDA graph (allocation is not a capturable operation),
// hosts that hand the library a fixed arena and forbid further allocation,
// and latency-sensitive loops where cudaMalloc would synchronise the device.
// For them this file offers lbm_observables_noalloc: the same float64
// reduction as lbm_observables, but its block partial sums live in a
// file-scope device array (NOALLOC_MAX_BLOCKS x 4 doubles = 32 KiB) that
// every GPU loading the library holds until the process exits. The caller
// passes the state and the output record; nothing is allocated or freed.
#include <mutex>

#include "engine.h"

namespace lbm {
namespace {

constexpr int NOALLOC_MAX_BLOCKS = 1024;
constexpr int NOALLOC_THREADS = 256;
constexpr int NOALLOC_MAX_DEVICES = 64;

static __device__ __align__(256) double g_noalloc_partials[NOALLOC_MAX_BLOCKS * NOBS];

// Device address of g_noalloc_partials, looked up once per device.
std::mutex g_noalloc_mutex;
double* g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {};

struct NoallocArgs {
    const void* state;
    long long plane;
    int pitch, nx, ny;
    double rho0;
    int comp;
    const double* px;
    const double* py;
    double norm;
    long long step;
    double dt;
};

template <int Q1>
__device__ __forceinline__ int noalloc_c(int i) {
    return Q1 == 3 ? c3_of(i) : 0;
}

template <typename T, int Q1, bool PULL>
__global__ void __launch_bounds__(NOALLOC_THREADS) noalloc_partials_kernel(NoallocArgs a, double* part) {
    constexpr int K = Q1 * Q1;
    __shared__ double red[(NOALLOC_THREADS / 32) * NOBS];
    const T* in = static_cast<const T*>(a.state);
    const long long n = (long long)a.nx * a.ny;
    double acc[NOBS] = {0.0, 0.0, 0.0, 0.0};
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n;
         c += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(c % a.nx), y = (int)(c / a.nx);
        // per node in the storage precision, then float64 (as lbm_observables)
        T dr = T(0), jx = T(0), jy = T(0);
#pragma unroll
        for (int k = 0; k < K; ++k) {
            int xs = x, ys = y;
            if (PULL) {  // CS storage phase: f_k(x) = stored_k(x - c_k)
                xs = x - noalloc_c<Q1>(k % Q1);
                ys = y - noalloc_c<Q1>(k / Q1);
                xs = xs < 0 ? xs + a.nx : (xs >= a.nx ? xs - a.nx : xs);
                ys = ys < 0 ? ys + a.ny : (ys >= a.ny ? ys - a.ny : ys);
            }
            const T s = in[k * a.plane + (long long)ys * a.pitch + xs];
            dr += s;
            if (vx_of<Q1>(k) != 0.0) jx += s * (T)vx_of<Q1>(k);
            if (vy_of<Q1>(k) != 0.0) jy += s * (T)vy_of<Q1>(k);
        }
        acc[0] += (double)dr;
        acc[1] += (double)jx;
        acc[2] += (double)jy;
        if (a.comp >= 0) acc[3] += (double)((a.comp == 0 ? jx : jy) / ((T)a.rho0 + dr)) * a.px[x] * a.py[y];
    }
    block_reduce_obs<double, NOALLOC_THREADS>(acc, part + (long long)blockIdx.x * NOBS, red);
}

__global__ void __launch_bounds__(NOALLOC_THREADS) noalloc_finalize_kernel(NoallocArgs a, const double* part,
                                                                          int nblocks, lbm_obs* out) {
    __shared__ double sm[NOALLOC_THREADS * NOBS];
    double v[NOBS] = {0.0, 0.0, 0.0, 0.0};
    for (int i = threadIdx.x; i < nblocks; i += blockDim.x)
#pragma unroll
        for (int q = 0; q < NOBS; ++q) v[q] += part[i * NOBS + q];
#pragma unroll
    for (int q = 0; q < NOBS; ++q) sm[threadIdx.x * NOBS + q] = v[q];
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s)
#pragma unroll
            for (int q = 0; q < NOBS; ++q) sm[threadIdx.x * NOBS + q] += sm[(threadIdx.x + s) * NOBS + q];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        lbm_obs o;
        o.step = a.step;
        o.time = (double)a.step * a.dt;
        o.mass = (double)a.nx * (double)a.ny * a.rho0 + sm[0];
        o.mom_x = sm[1];
        o.mom_y = sm[2];
        o.amp = a.comp >= 0 ? a.norm * sm[3] : 0.0;
        o.nonfinite = (isfinite(o.mass) && isfinite(o.amp) && isfinite(o.mom_x) && isfinite(o.mom_y)) ? 0 : 1;
        o.reserved = 0;
        *out = o;
    }
}

// Looks up (once per device, with that device current) the device address
// of the static partials array.
int noalloc_scratch(double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) {
        set_error("device index beyond the supported range");
        return LBM_EINVAL;
    }
    std::lock_guard<std::mutex> lk(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        double* p = nullptr;
        e = cudaGetSymbolAddress((void**)&p, g_noalloc_partials);
        if (e != cudaSuccess || !p) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_partials)");
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return LBM_OK;
}

}  // namespace
}  // namespace lbm

extern "C" int lbm_observables_noalloc(int model, int q_per_axis, int precision, int nx, int ny, const void* state,
                                       int64_t plane, int32_t pitch, double rho0, int comp, const double* px,
                                       const double* py, double norm, int64_t step, double dt, lbm_obs* out,
                                       void* cuda_stream) {
    using namespace lbm;
    try {
        if ((model != LBM_CS && model != LBM_FD) || (model == LBM_CS && q_per_axis != 3) || q_per_axis < 3 ||
            q_per_axis > 5 || (precision != LBM_FP64 && precision != LBM_FP32_DEV) || !state || !out) {
            set_error("lbm_observables_noalloc: bad model, velocity set, precision or null pointer");
            return LBM_EINVAL;
        }
        if (nx < 1 || ny < 1 || (long long)nx * ny > 2147483647LL || pitch < nx ||
            plane < (long long)pitch * ny) {
            set_error("lbm_observables_noalloc: lattice size beyond the maximum (nx*ny < 2^31) or bad layout");
            return LBM_EINVAL;
        }
        if (comp >= 0 && (comp > 1 || !px || !py)) {
            set_error("lbm_observables_noalloc: probe needs comp 0/1 and device tables px, py");
            return LBM_EINVAL;
        }
        double* part = nullptr;
        int rc = noalloc_scratch(&part);
        if (rc != LBM_OK) return rc;
        NoallocArgs a{state, (long long)plane, pitch, nx, ny, precision == LBM_FP64 ? 0.0 : rho0,
                      comp >= 0 ? comp : -1, px, py, norm, (long long)step, dt};
        const long long n = (long long)nx * ny;
        long long nb = (n + NOALLOC_THREADS - 1) / NOALLOC_THREADS;
        const int grid = (int)(nb < NOALLOC_MAX_BLOCKS ? nb : NOALLOC_MAX_BLOCKS);
        cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
        const bool pull = model == LBM_CS;
        if (precision == LBM_FP64) {
            if (pull) noalloc_partials_kernel<double, 3, true><<<grid, NOALLOC_THREADS, 0, s>>>(a, part);
            else if (q_per_axis == 3) noalloc_partials_kernel<double, 3, false><<<grid, NOALLOC_THREADS, 0, s>>>(a, part);
            else if (q_per_axis == 4) noalloc_partials_kernel<double, 4, false><<<grid, NOALLOC_THREADS, 0, s>>>(a, part);
            else noalloc_partials_kernel<double, 5, false><<<grid, NOALLOC_THREADS, 0, s>>>(a, part);
        } else {
            if (pull) noalloc_partials_kernel<float, 3, true><<<grid, NOALLOC_THREADS, 0, s>>>(a, part);
            else if (q_per_axis == 3) noalloc_partials_kernel<float, 3, false><<<grid, NOALLOC_THREADS, 0, s>>>(a, part);
            else if (q_per_axis == 4) noalloc_partials_kernel<float, 4, false><<<grid, NOALLOC_THREADS, 0, s>>>(a, part);
            else noalloc_partials_kernel<float, 5, false><<<grid, NOALLOC_THREADS, 0, s>>>(a, part);
        }
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "noalloc_partials_kernel");
        noalloc_finalize_kernel<<<1, NOALLOC_THREADS, 0, s>>>(a, part, grid, out);
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "noalloc_finalize_kernel");
        return LBM_OK;
    } catch (...) {
        set_error("lbm_observables_noalloc: internal error");
        return LBM_EINVAL;
    }
}
