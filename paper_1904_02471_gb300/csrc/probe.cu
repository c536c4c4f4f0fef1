// Measured FP32 throughput of this GPU: the denominator of the FD stage
// kernel's arithmetic roofline. Independent chains of fused multiply-adds on
// every SM, packed two per instruction (FFMA2, as the FD kernel's WENO-5
// faces) or one per instruction, timed with CUDA events. The paper has no
// counterpart; this is measurement support for the library's kernels.
#include "engine.h"

namespace lbm {
namespace {

constexpr int PROBE_THREADS = 256;
constexpr int PROBE_CHAINS = 8;

template <bool PACKED>
__global__ void __launch_bounds__(PROBE_THREADS) fp32_probe_kernel(int iters, float seed, float* out) {
    // a <- a * m + c with m slightly below 1: the values stay normal and
    // bounded for any iteration count
    const float m = 0.999999f, c = 1e-6f;
    if constexpr (PACKED) {
        float2 a[PROBE_CHAINS];
#pragma unroll
        for (int i = 0; i < PROBE_CHAINS; ++i) a[i] = make_float2(seed + i, seed - i);
        const float2 m2 = make_float2(m, m), c2 = make_float2(c, c);
        for (int it = 0; it < iters; ++it)
#pragma unroll
            for (int i = 0; i < PROBE_CHAINS; ++i) a[i] = __ffma2_rn(a[i], m2, c2);
        float s = 0.f;
#pragma unroll
        for (int i = 0; i < PROBE_CHAINS; ++i) s += a[i].x + a[i].y;
        out[blockIdx.x * PROBE_THREADS + threadIdx.x] = s;
    } else {
        float a[2 * PROBE_CHAINS];
#pragma unroll
        for (int i = 0; i < 2 * PROBE_CHAINS; ++i) a[i] = seed + i;
        for (int it = 0; it < iters; ++it)
#pragma unroll
            for (int i = 0; i < 2 * PROBE_CHAINS; ++i) a[i] = __fmaf_rn(a[i], m, c);
        float s = 0.f;
#pragma unroll
        for (int i = 0; i < 2 * PROBE_CHAINS; ++i) s += a[i];
        out[blockIdx.x * PROBE_THREADS + threadIdx.x] = s;
    }
}

}  // namespace
}  // namespace lbm

extern "C" int lbm_probe_fp32(int packed, double* flops_per_s, int* sm_count, double* ms_per_launch) {
    using namespace lbm;
    if (!flops_per_s) return LBM_EINVAL;
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev);
    if (e != cudaSuccess) return cuda_fail(e, "device attributes");
    const int blocks = sms * (per_sm / PROBE_THREADS);
    const int iters = 4096;
    float* out = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    cudaStream_t s = nullptr;
    int rc = LBM_OK;
    e = cudaMalloc(&out, sizeof(float) * (size_t)blocks * PROBE_THREADS);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    if (e == cudaSuccess) {
        auto launch = [&]() {
            if (packed) fp32_probe_kernel<true><<<blocks, PROBE_THREADS, 0, s>>>(iters, 1.0f, out);
            else fp32_probe_kernel<false><<<blocks, PROBE_THREADS, 0, s>>>(iters, 1.0f, out);
        };
        launch();  // warm-up
        constexpr int reps = 10;
        e = cudaEventRecord(a, s);
        for (int r = 0; r < reps && e == cudaSuccess; ++r) {
            launch();
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaEventRecord(b, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(b);
        float t = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, a, b);
        if (e == cudaSuccess) {
            // two flops per fused multiply-add, 2 * PROBE_CHAINS per thread and iteration
            const double fmas = (double)blocks * PROBE_THREADS * iters * 2.0 * PROBE_CHAINS;
            *flops_per_s = 2.0 * fmas / (t / reps * 1e-3);
            if (ms_per_launch) *ms_per_launch = t / reps;
            if (sm_count) *sm_count = sms;
        }
    }
    if (e != cudaSuccess) rc = cuda_fail(e, "lbm_probe_fp32");
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (s) cudaStreamDestroy(s);
    if (out) cudaFree(out);
    return rc;
}
