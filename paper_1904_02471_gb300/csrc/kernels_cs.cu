// Collision-streaming D2Q9 update, Eq. (sc_evolution), collision and
// streaming fused into one pass.
//
// Pull form. The buffer holding "the state" stores the post-collision values
// of the previous step, so the pre-collision population at node x is
//     f_k(x, t) = stored_k(x - c_k),
// gathered with periodic wrap. The kernel collides at x,
//     f*_k = f_k - omega (f_k - f^eq_k),  omega = dt / tau_LU,
// and writes f*_k to x in the other buffer (aligned, coalesced stores).
// Reads are one row up/down and one element left/right of the aligned
// position (adjacent lanes of the same warp), so DRAM traffic stays at one
// read + one write per population and node: 18 values per lattice update.
//
// Storage: buffers hold f_k - w_k rho0 (FP32 deviation form, rho0 the
// reference density) or f_k itself (FP64, rho0 = 0). With s_k the stored
// values: rho = rho0 + sum s_k, j = sum s_k v_k (sum w_k v_k = 0), and the
// stored equilibrium is w_k [ (rho - rho0) + rho (xi + (xi^2 - u^2)/2) ],
// xi = v_k . u, i.e. Eq. (herfeq) minus w_k rho0 (Sec. 2).
#include "kernels.h"

namespace lbm {

template <typename T, int TX, int RY>
__global__ void __launch_bounds__(TX) cs_step_kernel(GroupDev g, int j) {
    __shared__ double red[(TX / 32) * NOBS];
    const int n_lat = g.hdr[0];
    const int total = g.hdr[1];
    for (int item = blockIdx.x; item < total; item += gridDim.x) {
        const int li = find_lattice(g.item_begin, n_lat, item);
        const LatDesc* dp = g.desc + li;
        if ((long long)j >= dp->remaining) continue;
        const int nx = dp->nx, ny = dp->ny, pitch = dp->pitch;
        const long long plane = dp->plane;
        const int local = item - dp->item_begin;
        const int bx = local % dp->tiles_x, by = local / dp->tiles_x;
        const int cur = dp->cur ^ (j & 1);
        const T* __restrict__ in = static_cast<const T*>(dp->buf[cur]);
        T* __restrict__ out = static_cast<T*>(dp->buf[cur ^ 1]);
        const T omega = (T)dp->omega;
        const T r0 = (T)dp->rho0;
        const bool obs = observe_now(*dp, j);
        const int pc = dp->probe_comp;
        T acc[NOBS] = {T(0), T(0), T(0), T(0)};

        const int x = bx * TX + threadIdx.x;
        if (x < nx) {
            const int xm = (x == 0) ? nx - 1 : x - 1;
            const int xp = (x + 1 >= nx) ? x + 1 - nx : x + 1;
            T pxv = T(0);
            if (obs && pc >= 0) {
                if constexpr (sizeof(T) == 4) pxv = dp->probe_pxf[x]; else pxv = (T)dp->probe_px[x];
            }
#pragma unroll
            for (int r = 0; r < RY; ++r) {
                const int y = by * RY + r;
                if (y >= ny) break;
                const int ym = (y == 0) ? ny - 1 : y - 1;
                const int yp = (y + 1 >= ny) ? y + 1 - ny : y + 1;
                const long long rowm = (long long)ym * pitch, row0 = (long long)y * pitch,
                                rowp = (long long)yp * pitch;
                T s[9];
#pragma unroll
                for (int k = 0; k < 9; ++k) {
                    const int cx = c3_of(k % 3), cy = c3_of(k / 3);
                    const int sx = cx == 1 ? xm : (cx == -1 ? xp : x);
                    const long long sr = cy == 1 ? rowm : (cy == -1 ? rowp : row0);
                    s[k] = in[k * plane + sr + sx];
                }
                // moments, Eq. (f_moments_discrete), ascending k
                T dr = T(0), jx = T(0), jy = T(0);
#pragma unroll
                for (int k = 0; k < 9; ++k) {
                    dr += s[k];
                    if (vx_of<3>(k) != 0.0) jx += s[k] * (T)vx_of<3>(k);
                    if (vy_of<3>(k) != 0.0) jy += s[k] * (T)vy_of<3>(k);
                }
                const T rho = r0 + dr;
                const T inv = T(1) / rho;
                const T ux = jx * inv, uy = jy * inv;
                const T usq = ux * ux + uy * uy;
#pragma unroll
                for (int k = 0; k < 9; ++k) {
                    const T xi = (T)vx_of<3>(k) * ux + (T)vy_of<3>(k) * uy;
                    const T geq = (T)w_of<3>(k) * (dr + rho * (xi + T(0.5) * (xi * xi - usq)));
                    out[k * plane + row0 + x] = s[k] - omega * (s[k] - geq);
                }
                if (obs) {
                    acc[0] += dr;
                    acc[1] += jx;
                    acc[2] += jy;
                    if (pc >= 0) {
                        T pyv;
                        if constexpr (sizeof(T) == 4) pyv = dp->probe_pyf[y]; else pyv = (T)dp->probe_py[y];
                        acc[3] += (pc == 0 ? ux : uy) * pxv * pyv;
                    }
                }
            }
        }
        if (obs) block_reduce_obs<T, TX>(acc, dp->partials + (long long)local * NOBS, red);
    }
}

int cs_tile_tx(int v) {
    switch (v) {
        case CS_T128x1: case CS_T128x2: return 128;
        case CS_T256x1: case CS_T256x2: return 256;
        case CS_T64x4: return 64;
    }
    return 0;
}
int cs_tile_ty(int v) {
    switch (v) {
        case CS_T128x1: case CS_T256x1: return 1;
        case CS_T128x2: case CS_T256x2: return 2;
        case CS_T64x4: return 4;
    }
    return 0;
}

template <typename T>
static const void* cs_kernel_ptr(int tile) {
    switch (tile) {
        case CS_T128x1: return (const void*)cs_step_kernel<T, 128, 1>;
        case CS_T128x2: return (const void*)cs_step_kernel<T, 128, 2>;
        case CS_T256x1: return (const void*)cs_step_kernel<T, 256, 1>;
        case CS_T256x2: return (const void*)cs_step_kernel<T, 256, 2>;
        case CS_T64x4: return (const void*)cs_step_kernel<T, 64, 4>;
    }
    return nullptr;
}

cudaError_t launch_cs_step(int precision, int tile, int grid, const GroupDev& g, int j, cudaStream_t s) {
    const void* fn = precision == LBM_FP64 ? cs_kernel_ptr<double>(tile) : cs_kernel_ptr<float>(tile);
    if (!fn || grid <= 0) return cudaErrorInvalidValue;
    GroupDev gg = g;
    int jj = j;
    void* args[] = {&gg, &jj};
    return cudaLaunchKernel(fn, dim3(grid), dim3(cs_tile_tx(tile)), args, 0, s);
}

int cs_blocks_per_sm(int precision, int tile) {
    const void* fn = precision == LBM_FP64 ? cs_kernel_ptr<double>(tile) : cs_kernel_ptr<float>(tile);
    int n = 0;
    if (!fn || cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, cs_tile_tx(tile), 0) != cudaSuccess) return 1;
    return n > 0 ? n : 1;
}

}  // namespace lbm
