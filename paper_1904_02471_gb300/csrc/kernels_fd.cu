// Finite-difference LB update (Sec. 2): Eq. (evolution) in conservative form
//     d f_k/dt = L(f)_k = -v_kx D_x f_k - v_ky D_y f_k - (f_k - f^eq_k) / tau,
// advected with WENO-5 (Jiang-Shu) and advanced with the three-stage TVD
// (SSP) Runge-Kutta scheme in Shu-Osher form:
//     f1 = f + dt L(f);  f2 = 3/4 f + 1/4 (f1 + dt L(f1));
//     f^{n+1} = 1/3 f + 2/3 (f2 + dt L(f2)).
// One launch = one stage for every lattice of the group. The moments (rho, u)
// and so f^eq are taken from that stage's input, as the BGK term belongs to L.
//
// Per tile (TX x TY nodes) and population k:
//   1. the stage input plane k is staged in shared memory with a periodic
//      halo of 3 nodes (the WENO-5 stencil reach),
//   2. every interface value is computed once and stored: (TX+1) x TY faces
//      normal to x and TX x (TY+1) normal to y (a face is shared by the two
//      nodes it separates, which also makes the flux form conservative),
//   3. each node takes its flux differences, adds the BGK term and combines
//      with f^n for the stage.
// The WENO-5 face value is upwinded by the sign of the (constant) velocity
// component: for v > 0 the face i+1/2 is reconstructed from f_{i-2..i+2},
// for v < 0 from f_{i+3..i-1} (mirror image). Components equal to 0 (the
// 3- and 5-node sets) do not advect along that axis.
//
// Buffers: buf[0] = f^n (updated in place by stage 3: it is read only at the
// node being written, by the thread writing it), buf[1] = f^(1),
// buf[2] = f^(2). Storage offset as in the CS kernel (deviation form for
// FP32, full f for FP64): WENO differences and the stage combination are
// unchanged by the constant offset w_k rho0.
#include "kernels.h"

namespace lbm {

// 1D nodes and weights, indexed [q1 - 3][i] (see GH<> in common.cuh).
__constant__ double c_node_d[3][5] = {
    {GH<3>::v(0), GH<3>::v(1), GH<3>::v(2), 0.0, 0.0},
    {GH<4>::v(0), GH<4>::v(1), GH<4>::v(2), GH<4>::v(3), 0.0},
    {GH<5>::v(0), GH<5>::v(1), GH<5>::v(2), GH<5>::v(3), GH<5>::v(4)}};
__constant__ double c_wt_d[3][5] = {
    {GH<3>::w(0), GH<3>::w(1), GH<3>::w(2), 0.0, 0.0},
    {GH<4>::w(0), GH<4>::w(1), GH<4>::w(2), GH<4>::w(3), 0.0},
    {GH<5>::w(0), GH<5>::w(1), GH<5>::w(2), GH<5>::w(3), GH<5>::w(4)}};
__constant__ float c_node_f[3][5] = {
    {(float)GH<3>::v(0), (float)GH<3>::v(1), (float)GH<3>::v(2), 0.f, 0.f},
    {(float)GH<4>::v(0), (float)GH<4>::v(1), (float)GH<4>::v(2), (float)GH<4>::v(3), 0.f},
    {(float)GH<5>::v(0), (float)GH<5>::v(1), (float)GH<5>::v(2), (float)GH<5>::v(3), (float)GH<5>::v(4)}};
__constant__ float c_wt_f[3][5] = {
    {(float)GH<3>::w(0), (float)GH<3>::w(1), (float)GH<3>::w(2), 0.f, 0.f},
    {(float)GH<4>::w(0), (float)GH<4>::w(1), (float)GH<4>::w(2), (float)GH<4>::w(3), 0.f},
    {(float)GH<5>::w(0), (float)GH<5>::w(1), (float)GH<5>::w(2), (float)GH<5>::w(3), (float)GH<5>::w(4)}};

template <typename T>
__device__ __forceinline__ T node1(int q1, int i);
template <>
__device__ __forceinline__ double node1<double>(int q1, int i) { return c_node_d[q1 - 3][i]; }
template <>
__device__ __forceinline__ float node1<float>(int q1, int i) { return c_node_f[q1 - 3][i]; }
template <typename T>
__device__ __forceinline__ T wt1(int q1, int i);
template <>
__device__ __forceinline__ double wt1<double>(int q1, int i) { return c_wt_d[q1 - 3][i]; }
template <>
__device__ __forceinline__ float wt1<float>(int q1, int i) { return c_wt_f[q1 - 3][i]; }

// WENO-5 interface value from the upwind-ordered stencil (a, b, c, d, e) =
// (f_{i-2}, f_{i-1}, f_i, f_{i+1}, f_{i+2}) for the face i+1/2.
// Candidates q_r on {i-2..i}, {i-1..i+1}, {i..i+2}; smoothness indicators
// beta_r; nonlinear weights alpha_r = d_r / (eps + beta_r)^2 with linear
// weights d = (1/10, 6/10, 3/10). The normalisation sum_r alpha_r q_r /
// sum_r alpha_r is evaluated after multiplying numerator and denominator by
// s0 s1 s2 (s_r = (eps + beta_r)^2), which needs one division instead of four.
template <typename T>
__device__ __forceinline__ T weno5(T a, T b, T c, T d, T e, T eps) {
    const T q0 = (T(2) * a - T(7) * b + T(11) * c) * T(1.0 / 6.0);
    const T q1 = (-b + T(5) * c + T(2) * d) * T(1.0 / 6.0);
    const T q2 = (T(2) * c + T(5) * d - e) * T(1.0 / 6.0);
    T t0 = a - T(2) * b + c, u0 = a - T(4) * b + T(3) * c;
    T t1 = b - T(2) * c + d, u1 = b - d;
    T t2 = c - T(2) * d + e, u2 = T(3) * c - T(4) * d + e;
    const T b0 = T(13.0 / 12.0) * t0 * t0 + T(0.25) * u0 * u0;
    const T b1 = T(13.0 / 12.0) * t1 * t1 + T(0.25) * u1 * u1;
    const T b2 = T(13.0 / 12.0) * t2 * t2 + T(0.25) * u2 * u2;
    T s0 = eps + b0, s1 = eps + b1, s2 = eps + b2;
    s0 *= s0;
    s1 *= s1;
    s2 *= s2;
    const T a0 = T(0.1) * (s1 * s2);
    const T a1 = T(0.6) * (s0 * s2);
    const T a2 = T(0.3) * (s0 * s1);
    return fdiv(a0 * q0 + a1 * q1 + a2 * q2, a0 + a1 + a2);
}

__device__ __forceinline__ int wrapi(int i, int n) {
    i %= n;
    return i < 0 ? i + n : i;
}

// Shared memory of one block: the K halo tiles of the stage input, two face
// buffers (double-buffered across populations) and the reduction scratch.
template <typename T, int TX, int TY>
__host__ __device__ constexpr size_t fd_smem_bytes(int K) {
    return sizeof(T) * ((size_t)K * (TX + 6) * (TY + 6) + 2 * ((TX + 1) * TY + TX * (TY + 1))) +
           sizeof(double) * (TX * TY / 32) * NOBS;
}

template <typename T, int TX, int TY>
__global__ void __launch_bounds__(TX* TY) fd_stage_kernel(GroupDev g, int q1, int j, int stage) {
    constexpr int NT = TX * TY;
    constexpr int HX = TX + 6, HY = TY + 6, HXY = HX * HY;
    constexpr int NFX = (TX + 1) * TY;   // faces normal to x
    constexpr int NFY = TX * (TY + 1);   // faces normal to y
    constexpr int NF = NFX + NFY;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int K = q1 * q1;
    T* tiles = reinterpret_cast<T*>(smem_raw);          // [K][HY][HX]
    T* faces = tiles + (size_t)K * HXY;                  // [2][NF]
    double* red = reinterpret_cast<double*>(faces + 2 * NF);

    const int n_lat = g.hdr[0];
    const int total = g.hdr[1];
    const int tid = threadIdx.y * TX + threadIdx.x;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int in_idx = stage == 1 ? 0 : (stage == 2 ? 1 : 2);
    const int out_idx = stage == 1 ? 1 : (stage == 2 ? 2 : 0);
    const T ca = stage == 1 ? T(0) : (stage == 2 ? T(0.75) : T(1.0 / 3.0));
    const T cb = stage == 1 ? T(1) : (stage == 2 ? T(0.25) : T(2.0 / 3.0));

    for (int item = blockIdx.x; item < total; item += gridDim.x) {
        const int li = find_lattice(g.item_begin, n_lat, item);
        const LatDesc* dp = g.desc + li;
        if ((long long)j >= dp->remaining) continue;
        const int nx = dp->nx, ny = dp->ny, pitch = dp->pitch;
        const long long plane = dp->plane;
        const int local = item - dp->item_begin;
        const int bx = local % dp->tiles_x, by = local / dp->tiles_x;
        const int x0 = bx * TX, y0 = by * TY;
        const int x = x0 + tx, y = y0 + ty;
        const bool active = x < nx && y < ny;
        const T* __restrict__ U = static_cast<const T*>(dp->buf[in_idx]);
        const T* __restrict__ Fn = static_cast<const T*>(dp->buf[0]);
        T* __restrict__ out = static_cast<T*>(dp->buf[out_idx]);
        const T r0 = (T)dp->rho0;
        const T cdx = (T)dp->cdx;
        const T dtt = (T)dp->dt_tau;
        const T eps = (T)dp->eps;
        const long long cell = (long long)y * pitch + x;
        const bool interior = x0 >= 3 && x0 + TX + 3 <= nx && y0 >= 3 && y0 + TY + 3 <= ny;

        // 1. stage all K halo tiles of the stage input (periodic halo of 3)
        __syncthreads();  // previous item finished reading the tiles
        if (interior) {
            const T* src = U + (long long)(y0 - 3) * pitch + (x0 - 3);
            for (int k = 0; k < K; ++k) {
                const T* sk = src + k * plane;
                T* dk = tiles + k * HXY;
                for (int i = tid; i < HXY; i += NT) {
                    const int r = i / HX, c = i - r * HX;
                    dk[i] = sk[(long long)r * pitch + c];
                }
            }
        } else {
            for (int k = 0; k < K; ++k) {
                const T* sk = U + k * plane;
                T* dk = tiles + k * HXY;
                for (int i = tid; i < HXY; i += NT) {
                    const int r = i / HX, c = i - r * HX;
                    dk[i] = sk[(long long)wrapi(y0 - 3 + r, ny) * pitch + wrapi(x0 - 3 + c, nx)];
                }
            }
        }
        T fn_next = (stage != 1 && active) ? Fn[cell] : T(0);
        __syncthreads();

        // 2. moments of the stage input at this node, Eq. (f_moments_discrete)
        const int cidx = (ty + 3) * HX + tx + 3;
        T dr = T(0), jx = T(0), jy = T(0);
        for (int k = 0; k < K; ++k) {
            const T u = tiles[k * HXY + cidx];
            dr += u;
            jx += u * node1<T>(q1, k % q1);
            jy += u * node1<T>(q1, k / q1);
        }
        const T rho = r0 + dr;
        const T inv = active ? T(1) / rho : T(0);
        const T ux = jx * inv, uy = jy * inv;
        const T usq = ux * ux + uy * uy;

        if (stage == 1 && observe_now(*dp, j)) {
            T acc[NOBS] = {T(0), T(0), T(0), T(0)};
            if (active) {
                acc[0] = dr;
                acc[1] = jx;
                acc[2] = jy;
                const int pc = dp->probe_comp;
                if (pc >= 0) {
                    T pxv, pyv;
                    if constexpr (sizeof(T) == 4) {
                        pxv = dp->probe_pxf[x];
                        pyv = dp->probe_pyf[y];
                    } else {
                        pxv = dp->probe_px[x];
                        pyv = dp->probe_py[y];
                    }
                    acc[3] = (pc == 0 ? ux : uy) * pxv * pyv;
                }
            }
            block_reduce_obs<T, NT>(acc, dp->partials + (long long)local * NOBS, red);
        }

        // 3. per population: interface values, then the node update
        for (int k = 0; k < K; ++k) {
            const T* tk = tiles + k * HXY;
            T* fx = faces + (k & 1) * NF;
            T* fy = fx + NFX;
            const T vx = node1<T>(q1, k % q1), vy = node1<T>(q1, k / q1);
            // Upwind stencil of a face, as (first point, step) in the tile:
            // v > 0: f_{i-2..i+2} (first = left node - 2, step +1);
            // v < 0: f_{i+3..i-1} (first = left node + 3, step -1); the same
            // with rows (step +-HX) for faces normal to y.
            const int ox = vx > T(0) ? -2 : 3, sx = vx > T(0) ? 1 : -1;
            const int oy = vy > T(0) ? -2 * HX : 3 * HX, sy = vy > T(0) ? HX : -HX;
            const int fbeg = vx == T(0) ? NFX : 0;
            const int fend = vy == T(0) ? NFX : NF;
            for (int f = fbeg + tid; f < fend; f += NT) {
                const T* t;
                int st;
                if (f < NFX) {
                    const int row = f / (TX + 1), col = f - row * (TX + 1);
                    t = tk + (row + 3) * HX + (col + 2) + ox;  // left node of the face, shifted
                    st = sx;
                } else {
                    const int f2 = f - NFX;
                    const int row = f2 / TX, col = f2 - row * TX;
                    t = tk + (row + 2) * HX + (col + 3) + oy;  // lower node of the face, shifted
                    st = sy;
                }
                fx[f] = weno5<T>(t[0], t[st], t[2 * st], t[3 * st], t[4 * st], eps);
            }
            const T fn = fn_next;
            if (stage != 1 && active && k + 1 < K) fn_next = Fn[(k + 1) * plane + cell];
            __syncthreads();
            if (active) {
                T adv = T(0);
                if (vx != T(0)) adv -= (vx * cdx) * (fx[ty * (TX + 1) + tx + 1] - fx[ty * (TX + 1) + tx]);
                if (vy != T(0)) adv -= (vy * cdx) * (fy[(ty + 1) * TX + tx] - fy[ty * TX + tx]);
                const T uk = tk[cidx];
                const T xi = vx * ux + vy * uy;
                const T wk = wt1<T>(q1, k % q1) * wt1<T>(q1, k / q1);
                const T geq = wk * (dr + rho * (xi + T(0.5) * (xi * xi - usq)));
                const T upd = uk + (adv - (uk - geq) * dtt);
                out[k * plane + cell] = stage == 1 ? upd : ca * fn + cb * upd;
            }
        }
    }
}

int fd_tile_tx(int v) {
    switch (v) {
        case FD_T32x8: case FD_T32x4: case FD_T32x16: return 32;
        case FD_T64x4: return 64;
    }
    return 0;
}
int fd_tile_ty(int v) {
    switch (v) {
        case FD_T32x8: return 8;
        case FD_T32x4: case FD_T64x4: return 4;
        case FD_T32x16: return 16;
    }
    return 0;
}

template <typename T>
static const void* fd_kernel_ptr(int tile) {
    switch (tile) {
        case FD_T32x8: return (const void*)fd_stage_kernel<T, 32, 8>;
        case FD_T32x4: return (const void*)fd_stage_kernel<T, 32, 4>;
        case FD_T64x4: return (const void*)fd_stage_kernel<T, 64, 4>;
        case FD_T32x16: return (const void*)fd_stage_kernel<T, 32, 16>;
    }
    return nullptr;
}

template <typename T>
static size_t fd_smem(int tile, int K) {
    switch (tile) {
        case FD_T32x8: return fd_smem_bytes<T, 32, 8>(K);
        case FD_T32x4: return fd_smem_bytes<T, 32, 4>(K);
        case FD_T64x4: return fd_smem_bytes<T, 64, 4>(K);
        case FD_T32x16: return fd_smem_bytes<T, 32, 16>(K);
    }
    return 0;
}

static const void* fd_fn(int precision, int tile) {
    return precision == LBM_FP64 ? fd_kernel_ptr<double>(tile) : fd_kernel_ptr<float>(tile);
}
static size_t fd_bytes(int precision, int tile, int q1) {
    return precision == LBM_FP64 ? fd_smem<double>(tile, q1 * q1) : fd_smem<float>(tile, q1 * q1);
}

// Opt every variant into the largest dynamic shared memory it can need (25
// populations); done once per process.
static cudaError_t fd_prepare(int precision, int tile) {
    static bool done[2][FD_NTILES] = {};
    const int p = precision == LBM_FP64 ? 0 : 1;
    if (done[p][tile]) return cudaSuccess;
    const size_t need = fd_bytes(precision, tile, 5);
    cudaError_t e = cudaFuncSetAttribute(fd_fn(precision, tile), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need);
    if (e == cudaSuccess) done[p][tile] = true;
    return e;
}

cudaError_t launch_fd_stage(int precision, int q1, int tile, int grid, const GroupDev& g, int j, int stage,
                            cudaStream_t s) {
    if (tile < 0 || tile >= FD_NTILES || grid <= 0 || q1 < 3 || q1 > 5 || stage < 1 || stage > 3)
        return cudaErrorInvalidValue;
    const void* fn = fd_fn(precision, tile);
    cudaError_t e = fd_prepare(precision, tile);
    if (e != cudaSuccess) return e;
    GroupDev gg = g;
    int qq = q1, jj = j, ss = stage;
    void* args[] = {&gg, &qq, &jj, &ss};
    return cudaLaunchKernel(fn, dim3(grid), dim3(fd_tile_tx(tile), fd_tile_ty(tile)), args, fd_bytes(precision, tile, q1), s);
}

int fd_blocks_per_sm(int precision, int q1, int tile) {
    if (tile < 0 || tile >= FD_NTILES || fd_prepare(precision, tile) != cudaSuccess) return 1;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fd_fn(precision, tile), fd_tile_tx(tile) * fd_tile_ty(tile),
                                                      fd_bytes(precision, tile, q1)) != cudaSuccess)
        return 1;
    return n > 0 ? n : 1;
}

}  // namespace lbm
