// Allocation-free observables of a lattice state held in caller memory.
//
// Some callers cannot call cudaMalloc: hosts that hand the library a fixed
// arena and forbid further allocation (an embedding application that owns
// all device memory), and latency-sensitive loops where cudaMalloc would
// synchronise the device and stall the work in flight.
// For them this file offers lbm_observables_noalloc: the same float64
// reduction as lbm_observables, but its block partial sums live in a
// file-scope device array (NOALLOC_MAX_BLOCKS x 4 doubles = 32 KiB) that
// every GPU loading the library holds until the process exits. The caller
// passes the state and the output record; nothing is allocated or freed.
#include <mutex>

#include "engine.h"
#include "obs.cuh"

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
    int phase;   // storage phase of a CS state (lbm_view::cs_pull_phase); 0 for FD
    double rho0;
    int comp;
    const double* px;
    const double* py;
    double norm;
    long long step;
    double dt;
};

// Per-node moments read through the state's storage phase (the helpers the
// library's own observables snapshot uses), then float64 block partials.
template <typename T, int Q1>
__global__ void __launch_bounds__(NOALLOC_THREADS) noalloc_partials_kernel(NoallocArgs a, double* part) {
    __shared__ double red[(NOALLOC_THREADS / 32) * NOBS];
    const T* in = static_cast<const T*>(a.state);
    const StoreMap m = store_map_of_phase(a.phase);
    const long long n = (long long)a.nx * a.ny;
    double acc[NOBS] = {0.0, 0.0, 0.0, 0.0};
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n;
         c += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(c % a.nx), y = (int)(c / a.nx);
        T dr, jx, jy;
        stored_node_moments<T, Q1>(in, m, x, y, a.nx, a.ny, a.plane, a.pitch, dr, jx, jy,
                                   [](long long) { return true; });
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
    __shared__ double tot[NOBS];
    sum_rows(part, nblocks, tot, sm);
    __syncthreads();
    if (threadIdx.x == 0) *out = make_obs(a.step, a.dt, a.nx, a.ny, a.rho0, a.comp, a.norm, tot);
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
                                       int64_t plane, int32_t pitch, int32_t cs_phase, double rho0, int comp, const double* px,
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
        if (cs_phase < 0 || cs_phase > 2 || (model == LBM_FD && cs_phase != 0)) {
            set_error("lbm_observables_noalloc: cs_phase must be 0, 1 or 2 for CS and 0 for FD");
            return LBM_EINVAL;
        }
        if (comp >= 0 && (comp > 1 || !px || !py)) {
            set_error("lbm_observables_noalloc: probe needs comp 0/1 and device tables px, py");
            return LBM_EINVAL;
        }
        double* part = nullptr;
        int rc = noalloc_scratch(&part);
        if (rc != LBM_OK) return rc;
        NoallocArgs a{state, (long long)plane, pitch, nx, ny, cs_phase, precision == LBM_FP64 ? 0.0 : rho0,
                      comp >= 0 ? comp : -1, px, py, norm, (long long)step, dt};
        const long long n = (long long)nx * ny;
        long long nb = (n + NOALLOC_THREADS - 1) / NOALLOC_THREADS;
        const int grid = (int)(nb < NOALLOC_MAX_BLOCKS ? nb : NOALLOC_MAX_BLOCKS);
        cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
        if (precision == LBM_FP64) {
            if (q_per_axis == 3) noalloc_partials_kernel<double, 3><<<grid, NOALLOC_THREADS, 0, s>>>(a, part);
            else if (q_per_axis == 4) noalloc_partials_kernel<double, 4><<<grid, NOALLOC_THREADS, 0, s>>>(a, part);
            else noalloc_partials_kernel<double, 5><<<grid, NOALLOC_THREADS, 0, s>>>(a, part);
        } else {
            if (q_per_axis == 3) noalloc_partials_kernel<float, 3><<<grid, NOALLOC_THREADS, 0, s>>>(a, part);
            else if (q_per_axis == 4) noalloc_partials_kernel<float, 4><<<grid, NOALLOC_THREADS, 0, s>>>(a, part);
            else noalloc_partials_kernel<float, 5><<<grid, NOALLOC_THREADS, 0, s>>>(a, part);
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
