// Finite-difference LB update (Sec. 2): Eq. (evolution) in conservative form
//     d f_k/dt = L(f)_k = -v_kx D_x f_k - v_ky D_y f_k - (f_k - f^eq_k) / tau,
// advected with WENO-5 (Jiang-Shu) and advanced with the three-stage TVD
// (SSP) Runge-Kutta scheme in Shu-Osher form:
//     f1 = f + dt L(f);  f2 = 3/4 f + 1/4 (f1 + dt L(f1));
//     f^{n+1} = 1/3 f + 2/3 (f2 + dt L(f2)).
// One launch = one stage for every lattice of the group. The moments (rho, u)
// and so f^eq are taken from that stage's input, as the BGK term belongs to L.
//
// Per tile (TX x TY nodes):
//   1. every population plane of the stage input is staged in shared memory
//      with a periodic halo of 3 nodes (the WENO-5 stencil reach); the
//      moments come from there,
//   then per group of G populations:
//   2. per group of G populations, every interface value is computed once
//      and stored: (TX+1) x TY faces normal to x and TX x (TY+1) normal to y
//      (a face is shared by the two nodes it separates, which also makes the
//      flux form conservative),
//   3. after one barrier each node takes its flux differences, adds the BGK
//      term and combines with f^n for the stage.
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
#include "fd_common.cuh"
#include "kernels.h"
#include "ptx.cuh"

namespace lbm {

// Column sums cs[ix] = sum_iy g(ix + Q1 iy) and row sums rs[iy] =
// sum_ix g(ix + Q1 iy) of a quantity over the product set.
template <typename T, int Q1, typename Fn>
__device__ __forceinline__ void sum_cols_rows(Fn g, T (&cs)[Q1], T (&rs)[Q1]) {
#pragma unroll
    for (int iy = 0; iy < Q1; ++iy)
#pragma unroll
        for (int ix = 0; ix < Q1; ++ix) {
            const T v = g(ix + Q1 * iy);
            cs[ix] = iy == 0 ? v : cs[ix] + v;
            rs[iy] = ix == 0 ? v : rs[iy] + v;
        }
}
// Zeroth and first moments from column and row sums: sum g, sum g v_x,
// sum g v_y (v_x depends on ix only, v_y on iy only).
template <typename T, int Q1>
__device__ __forceinline__ void moments_of_sums(const T (&cs)[Q1], const T (&rs)[Q1], T& m0, T& mx, T& my) {
    m0 = cs[0];
#pragma unroll
    for (int i = 1; i < Q1; ++i) m0 += cs[i];
    mx = T(0);
    my = T(0);
#pragma unroll
    for (int i = 0; i < Q1; ++i) {
        if (GH<Q1>::v(i) != 0.0) {
            mx += (T)GH<Q1>::v(i) * cs[i];
            my += (T)GH<Q1>::v(i) * rs[i];
        }
    }
}
// v_k . u and v_k . j + d of population k from per-axis products: the 1D set
// is symmetric (v_{Q1-1-i} = -v_i), so v_i u_x and v_i j_x are formed for
// the upper half of the nodes and negated for the lower half; v_iy u_y and
// v_iy j_y + d once per row (shared by the Q1 populations of the row).
template <typename T, int Q1>
struct EqTerms {
    T ux, uy, jx, jy, d;
    __device__ __forceinline__ T xu(int ix) const {
        return GH<Q1>::v(ix) == 0.0 ? T(0)
               : (2 * ix >= Q1 ? (T)GH<Q1>::v(ix) * ux : -((T)GH<Q1>::v(Q1 - 1 - ix) * ux));
    }
    __device__ __forceinline__ T xj(int ix) const {
        return GH<Q1>::v(ix) == 0.0 ? T(0)
               : (2 * ix >= Q1 ? (T)GH<Q1>::v(ix) * jx : -((T)GH<Q1>::v(Q1 - 1 - ix) * jx));
    }
    __device__ __forceinline__ T xi(int k) const {
        const int ix = k % Q1, iy = k / Q1;
        if (GH<Q1>::v(iy) == 0.0) return xu(ix);
        const T yv = (T)GH<Q1>::v(iy) * uy;
        return GH<Q1>::v(ix) == 0.0 ? yv : xu(ix) + yv;
    }
    __device__ __forceinline__ T lin(int k) const {
        const int ix = k % Q1, iy = k / Q1;
        const T yl = GH<Q1>::v(iy) == 0.0 ? d : (T)GH<Q1>::v(iy) * jy + d;
        return GH<Q1>::v(ix) == 0.0 ? yl : xj(ix) + yl;
    }
};

// Tile geometry: TX = 32 nodes along x (one warp per row), TY rows. The
// staged halo tile of a population has HY = TY + 6 rows of HXP = 40 values,
// columns x0 - 4 .. x0 + 35 (16-byte aligned rows; the stencil needs
// x0 - 3 .. x0 + 34), rows y0 - 3 .. y0 + TY + 2.
constexpr int FD_TX = 32;
constexpr int FD_HXP = 40;

// Populations whose faces are evaluated between two barriers (a group): 4,
// or 2 where four face groups would not fit next to the halo tiles (FP64, 25
// velocities), or 8 for FP32 32 x 8 tiles: warp p evaluates the edge faces of
// the group's p-th population, so a group of as many populations as the tile
// has warps gives every warp the same work between two barriers.
template <typename T, int Q1, int TY>
__host__ __device__ constexpr int fd_group() {
    return (sizeof(T) == 8 && Q1 == 5) ? 2 : (sizeof(T) == 4 && TY == 8 ? 8 : 4);
}
// Face buffers: two alternate between groups (one barrier per group); a
// group of 8 has one (two barriers per group, the same shared memory).
template <typename T, int Q1, int TY>
__host__ __device__ constexpr int fd_face_bufs() { return fd_group<T, Q1, TY>() == 8 ? 1 : 2; }

template <typename T, int Q1, int TY>
__host__ __device__ constexpr size_t fd_smem_bytes() {
    return sizeof(T) * ((size_t)Q1 * Q1 * (TY + 6) * FD_HXP +
                        fd_face_bufs<T, Q1, TY>() * fd_group<T, Q1, TY>() * ((FD_TX + 1) * TY + FD_TX * (TY + 1))) +
           sizeof(double) * (FD_TX * TY / 32) * NOBS;
}

// Resident blocks per SM the register allocation is bounded for: 1024
// threads per SM for FP32, i.e. at most 64 registers per thread (shared
// memory, 53.5 KiB per 256-thread block for 16 populations, allows as many:
// four blocks in 228 KiB); 512 threads (128 registers) for FP64.
// The IMEX stage kernels hold more values per thread (the stage input and P
// at the node): their FP32 variants are bounded for 512 threads per SM (128
// registers) instead.
template <typename T, int TY, bool IMEX = false>
constexpr int fd_min_blocks() {
    return ((sizeof(T) == 4 ? (IMEX ? 512 : 1024) : 512) / (FD_TX * TY)) > 0
               ? (sizeof(T) == 4 ? (IMEX ? 512 : 1024) : 512) / (FD_TX * TY)
               : 1;
}

// IMEX-SSP2(2,2,2) (LBM_TS_IMEX): gamma of the implicit tableau, 1 - 1/sqrt 2.
constexpr double IMEX_GAMMA = 0.29289321881345247560;

// IMEX: the implicit BGK part of a stage in closed form, at every staged node
// of the tile. The stage value Y solves Y = u + dt g C(Y), C(Y) = -(Y -
// f^eq(Y)) / tau; the collision conserves rho and rho u (Eq. herfeq has the
// moments of Eq. f_moments_discrete), so Y has the moments of u, f^eq(Y) =
// f^eq(u), and Y = (u + lam f^eq(u)) / (1 + lam), lam = g dt / tau. Values
// in the storage form (deviations from w_k rho0 for FP32, r0 = rho0; full f
// for FP64, r0 = 0): the map is linear, the offsets carry over.
template <typename T, int Q1>
__device__ __forceinline__ void imex_stage_values(T* tiles, int hxy, T r0, T lam, T il, int tid, int nt) {
    constexpr int K = Q1 * Q1;
    for (int pos = tid; pos < hxy; pos += nt) {
        T dr = T(0), jx = T(0), jy = T(0);
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const T u = tiles[k * hxy + pos];
            dr += u;
            if (vx_of<Q1>(k) != 0.0) jx += u * (T)vx_of<Q1>(k);
            if (vy_of<Q1>(k) != 0.0) jy += u * (T)vy_of<Q1>(k);
        }
        const T rho = r0 + dr;
        const T inv = T(1) / rho;
        const T ux = jx * inv, uy = jy * inv;
        const T usq = ux * ux + uy * uy, hr = T(0.5) * rho;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const T vx = (T)vx_of<Q1>(k), vy = (T)vy_of<Q1>(k);
            const T xi = vx * ux + vy * uy;
            const T geq = (T)w_of<Q1>(k) * (hr * (xi * xi - usq) + (vx * jx + (vy * jy + dr)));
            tiles[k * hxy + pos] = (tiles[k * hxy + pos] + lam * geq) * il;
        }
    }
}

// One stage of the FD update. IMEX = false: SSP-RK3 stage `stage` (1..3).
// IMEX = true: stage 1 or 2 of IMEX-SSP2(2,2,2) with explicit WENO-5
// advection A and implicit BGK C. With Y_i the stage values (above), the
// scheme's
//   Y_2 = f^n + dt A(Y_1) + (1 - 2g) dt C(Y_1) + g dt C(Y_2),
//   f^{n+1} = f^n + dt/2 (A(Y_1) + A(Y_2) + C(Y_1) + C(Y_2))
// are evaluated as: stage 1 stages f^n, maps it to Y_1, and writes
//   Z = f^n + dt A(Y_1) + (1 - 2g) dt C(Y_1)      (buffer 1)
//   P = f^n + 2g dt C(Y_1)                          (buffer 2);
// stage 2 stages Z, maps it to Y_2, and writes
//   f^{n+1} = P + ((Z - P) + dt A(Y_2) + dt C(Y_2)) / 2   (buffer 0),
// with dt C(Y_i) = -(dt/tau) (u_i - f^eq(u_i)) / (1 + lam), u_i the stage's
// input (f^n or Z): no difference of nearly equal values is multiplied by
// dt/tau, so the rounding stays small however stiff the collision is.
template <typename T, int Q1, int TY, bool IMEX>
__global__ void __launch_bounds__(FD_TX* TY, (fd_min_blocks<T, TY, IMEX>())) fd_stage_kernel(GroupDev g, int j, int stage) {
    using P = Pr<T>;
    using V = typename P::V;
    constexpr int K = Q1 * Q1;
    constexpr int TX = FD_TX, HXP = FD_HXP;
    constexpr int NT = TX * TY;
    constexpr int HY = TY + 6, HXY = HY * HXP;
    constexpr int NFX = (TX + 1) * TY;   // faces normal to x: [TY][TX + 1]
    constexpr int NFY = TX * (TY + 1);   // faces normal to y: [TY + 1][TX]
    constexpr int NF = NFX + NFY;
    constexpr int VEC = 16 / sizeof(T);   // values per 16-byte copy
    constexpr int RV = HXP / VEC;         // 16-byte chunks per staged row
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int G = fd_group<T, Q1, TY>();
    constexpr int FB = fd_face_bufs<T, Q1, TY>();
    // 16-velocity set: populations 2q and 2q+1 (nodes ix = 0, 1 or 2, 3 of
    // one row of the product set) have the same signs of both velocity
    // components, so the same upwind stencils: their faces are evaluated and
    // stored side by side
    constexpr bool PAIRS = Q1 == 4;
    static_assert(!PAIRS || (GH<4>::v(0) < 0 && GH<4>::v(1) < 0 && GH<4>::v(2) > 0 && GH<4>::v(3) > 0 && G % 2 == 0),
                  "pairs (2q, 2q+1) must share their upwind directions");
    T* tiles = reinterpret_cast<T*>(smem_raw);          // [K][HY][HXP]
    T* faces = tiles + (size_t)K * HXY;                  // [FB][G][NF]
    double* red = reinterpret_cast<double*>(faces + FB * G * NF);
    __shared__ long long s_row[HY];                      // wrapped row offsets (edge tiles)
    __shared__ int s_col[HXP];                           // wrapped columns (edge tiles)
    __shared__ int s_obs;                                // record observables for this item

    const int n_lat = g.hdr[0];
    const int total = g.hdr[1];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tid = ty * TX + tx;
    const int in_idx = IMEX ? (stage == 1 ? 0 : 1) : (stage == 1 ? 0 : (stage == 2 ? 1 : 2));
    const int out_idx = IMEX ? (stage == 1 ? 1 : 0) : (stage == 1 ? 1 : (stage == 2 ? 2 : 0));
    // the stage reads its input at its own node from global memory too (IMEX:
    // the staged tile holds the stage values Y instead), and f^n (RK3 stages 2, 3)
    const bool node_in = IMEX || stage != 1;
    // stage weights: f^(s) = f^n + cb ((u - f^n) + dt L(u)), i.e. the Shu-Osher
    // combinations 3/4 f^n + 1/4 (u + dt L(u)) and 1/3 f^n + 2/3 (u + dt L(u))
    const T cb = stage == 1 ? T(1) : (stage == 2 ? T(0.25) : T(2.0 / 3.0));
    // warp p of a group of G populations also evaluates the faces on the
    // tile's right and top edges for the group's p-th population:
    // lane l < TY: x-face right of node (TX-1, l); every lane: y-face above (l, TY-1)
    const int ex_row = tx < TY ? tx : TY - 1;
    // per-thread bases in the staged tile (all stencil offsets are immediates)
    const int cidx = (ty + 3) * HXP + tx + 4;           // the node itself
    const int xrow = (ty + 3) * HXP + tx;                // row of the node, column tx
    const int ycol = ty * HXP + tx + 4;                  // column of the node, row ty
    const int exrow = (ex_row + 3) * HXP + TX;           // extra x-face: virtual node (TX, ex_row)
    const int eycol = TY * HXP + tx + 4;                 // extra y-face: virtual node (tx, TY)

    for (int item = blockIdx.x; item < total; item += gridDim.x) {
        const int li = find_lattice(g.item_begin, n_lat, item);
        const LatDesc* dp = g.desc + li;
        if ((long long)j >= dp->remaining) {
            item = last_item_of(*dp, item);
            continue;
        }
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
        const T r0 = lat_val<T>(dp->rho0, dp->rho0_f);
        const T cdx = lat_val<T>(dp->cdx, dp->cdx_f);
        const T dtt = lat_val<T>(dp->dt_tau, dp->dt_tau_f);
        const V eps = P::sp(lat_val<T>(dp->eps, dp->eps_f) * T(12.0 / 13.0));
        const long long cell = (long long)y * pitch + x;
        const bool interior = x0 >= 4 && x0 + TX + 4 <= nx && y0 >= 3 && y0 + TY + 3 <= ny;
        // 16-byte asynchronous copies of the K halo tiles: a thread owns one
        // (row, 16-byte column chunk) of the tile and copies it for every
        // SK-th population, stepping by whole planes (no index arithmetic per
        // copy); row_src(r, c) is the source of population 0
        auto stage_rows16 = [&](int t, auto row_src) {
            constexpr int CHUNKS = HY * RV;   // (row, 16-byte chunk) positions of a tile
            if constexpr (NT >= CHUNKS) {
                constexpr int SK = NT / CHUNKS;
                if (t < SK * CHUNKS) {
                    const int pr = t % CHUNKS, k0 = t / CHUNKS;
                    const int r = pr / RV, c = pr - r * RV;
                    const T* sp = row_src(r, c) + k0 * plane;
                    T* dp16 = tiles + k0 * HXY + r * HXP + c * VEC;
#pragma unroll 4
                    for (int k = k0; k < K; k += SK, sp += SK * plane, dp16 += SK * HXY)
                        if (LBM_BC_NODE(dp, K, sp - U) && LBM_BC_NODE(dp, K, sp - U + VEC - 1)) cp_async16(dp16, sp);
                }
            } else {
                for (int pr = t; pr < CHUNKS; pr += NT) {
                    const int r = pr / RV, c = pr - r * RV;
                    const T* sp = row_src(r, c);
                    T* dp16 = tiles + r * HXP + c * VEC;
#pragma unroll 4
                    for (int k = 0; k < K; ++k, sp += plane, dp16 += HXY)
                        if (LBM_BC_NODE(dp, K, sp - U) && LBM_BC_NODE(dp, K, sp - U + VEC - 1)) cp_async16(dp16, sp);
                }
            }
        };

        // 1. stage all K halo tiles of the stage input
        __syncthreads();  // the previous item is done with the tiles (and s_obs)
        if (tid == 0) s_obs = stage == 1 && observe_now(*dp, j);
        if (interior) {
            // rows are 16-byte aligned (x0 - 4 is a multiple of 4, pitch of
            // 32): every thread issues all its 16-byte asynchronous copies,
            // then waits once
            const T* src = U + (long long)(y0 - 3) * pitch + (x0 - 4);
            stage_rows16(tid, [&](int r, int c) { return src + (long long)r * pitch + c * VEC; });
            cp_async_wait_all();
        } else {
            // periodic edge: wrapped row offsets and columns once per tile,
            // then asynchronous copies from the wrapped positions
            for (int i = tid; i < HY + HXP; i += NT) {
                if (i < HY) s_row[i] = (long long)wrapi(y0 - 3 + i, ny) * pitch;
                else s_col[i - HY] = wrapi(x0 - 4 + (i - HY), nx);
            }
            __syncthreads();
            if (nx % VEC == 0) {
                // a 16-byte column chunk starts at a multiple of VEC and the
                // wrap point nx is one, so no chunk straddles it: one copy
                // per chunk from its wrapped start column
                stage_rows16(tid, [&](int r, int c) { return U + s_row[r] + s_col[c * VEC]; });
            } else {
                for (int i = tid; i < K * HXY; i += NT) {
                    const int k = i / HXY, rem = i - k * HXY;
                    const int r = rem / HXP, c = rem - r * HXP;
                    if (LBM_BC_NODE(dp, K, k * plane + s_row[r] + s_col[c]))
                        cp_async_small<sizeof(T)>(tiles + i, U + k * plane + s_row[r] + s_col[c]);
                }
            }
            cp_async_wait_all();
        }
        const T* __restrict__ fnp = (IMEX ? U : Fn) + cell;   // node values of f^n (RK3) / of the input (IMEX)
        const T* __restrict__ ppn = static_cast<const T*>(dp->buf[2]) + cell;   // IMEX stage 2: P
        T* __restrict__ pout = static_cast<T*>(dp->buf[2]) + cell;              // IMEX stage 1: P
        // IMEX constants: lam = g dt/tau, il = 1/(1 + lam), c1 = (dt/tau) il
        const T lam = T(IMEX_GAMMA) * dtt, il = T(1) / (T(1) + lam), c1 = dtt * il;
        T* __restrict__ op = out + cell;
        __syncthreads();
        if constexpr (IMEX) {
            imex_stage_values<T, Q1>(tiles, HXY, r0, lam, il, tid, NT);
            __syncthreads();
        }

        // 2. moments of the stage input at this node, Eq. (f_moments_discrete)
        //    (ascending k; FP32 with 16 velocities: through the column sums
        //    over iy and the row sums over ix of the product set, fewer
        //    operations)
        T dr = T(0), jx = T(0), jy = T(0);
        if constexpr (sizeof(T) == 4 && Q1 == 4) {
            T cs[Q1], rs[Q1];
            sum_cols_rows<T, Q1>([&](int k) { return tiles[k * HXY + cidx]; }, cs, rs);
            moments_of_sums<T, Q1>(cs, rs, dr, jx, jy);
        } else {
#pragma unroll
            for (int k = 0; k < K; ++k) {
                const T u = tiles[k * HXY + cidx];
                dr += u;
                if (vx_of<Q1>(k) != 0.0) jx += u * (T)vx_of<Q1>(k);
                if (vy_of<Q1>(k) != 0.0) jy += u * (T)vy_of<Q1>(k);
            }
        }
        const T rho = r0 + dr;
        const T inv = active ? T(1) / rho : T(0);
        const T ux = jx * inv, uy = jy * inv;
        const T usq = ux * ux + uy * uy;

        if (s_obs) {
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
            // no trailing barrier: `red` is next written after the next
            // item's staging barrier
            block_reduce_obs<T, NT, false>(acc, dp->partials + (long long)local * NOBS, red);
        }

        // FP32: residual moments of the collision term. In exact arithmetic
        // sum_k (u_k - geq_k) (1, v_k) = 0; in float32 the rounding of the
        // moments and of geq leaves a residual of ~1e-7 of the momentum per
        // stage, which is not small next to the viscous decay per stage of a
        // slowly decaying flow. It is computed from the differences u_k - geq_k
        // (accurate) and removed below with w_k (R0 + v_k . R1), which has
        // exactly these moments (quadrature identities of the set).
        // The stored equilibrium is written w_k (dr + v_k . j + rho/2 ((v_k . u)^2
        // - u^2)), i.e. Eq. (herfeq) minus w_k rho0 with rho (v_k . u) = v_k . j.
        const T hr = T(0.5) * rho;
        T R0 = T(0), R1x = T(0), R1y = T(0);
        if constexpr (sizeof(T) == 4) {
            // v_k . u and v_k . j + dr from per-axis terms (v_x u_x for each
            // node of the 1D set, v_y u_y + ... for each row of the product set)
            const EqTerms<T, Q1> e{ux, uy, jx, jy, dr};
            auto dk = [&](int k) {
                T geq;
                if constexpr (Q1 == 4) {
                    const T xi = e.xi(k);
                    geq = (T)w_of<Q1>(k) * (hr * (xi * xi - usq) + e.lin(k));
                } else {
                    const T vx = (T)vx_of<Q1>(k), vy = (T)vy_of<Q1>(k);
                    const T xi = vx * ux + vy * uy;
                    geq = (T)w_of<Q1>(k) * (hr * (xi * xi - usq) + (vx * jx + (vy * jy + dr)));
                }
                // the stage input at the node (IMEX: from global memory, the
                // tile holds the stage values)
                const T uin = IMEX ? ((active && LBM_BC_NODE(dp, K, cell + k * plane)) ? fnp[k * plane] : T(0))
                                   : tiles[k * HXY + cidx];
                return uin - geq;
            };
            if constexpr (Q1 == 4) {
                // sums through the columns and rows of the product set
                T cs[Q1], rs[Q1];
                sum_cols_rows<T, Q1>(dk, cs, rs);
                moments_of_sums<T, Q1>(cs, rs, R0, R1x, R1y);
            } else {
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    const T d = dk(k);
                    R0 += d;
                    if (vx_of<Q1>(k) != 0.0) R1x += d * (T)vx_of<Q1>(k);
                    if (vy_of<Q1>(k) != 0.0) R1y += d * (T)vy_of<Q1>(k);
                }
            }
        }
        // the correction w_k (R0 + v_k . R1) enters the equilibrium as
        // shifted moments: dr + R0, j + R1
        const T drc = dr + R0, jxc = jx + R1x, jyc = jy + R1y;
        const EqTerms<T, Q1> ec{ux, uy, jxc, jyc, drc};

        // 3. per group of G populations: every thread evaluates the x- and
        //    y-face on the low side of its node for each population of the
        //    group (one packed pair each), the tile's right- and top-edge
        //    faces are added (below), one barrier, then every node updates
        //    those G populations from the four faces around it. Two face
        //    buffers alternate between groups; with one, a barrier also
        //    precedes each group's faces. With the 16-velocity set the packed
        //    pairs are two populations' x-faces and then their y-faces instead
        //    of one population's x- and y-face, and faces are stored and read
        //    back as pairs (half the shared-memory instructions for them); its
        //    edge faces are evaluated through one copy of the code for all the
        //    group's pairs (an unrolled copy per pair and axis had made the
        //    kernel's instructions outgrow the instruction cache: the warps
        //    stalled on instruction fetch), the x-edges of all pairs packed one
        //    (pair, row) per lane.
#pragma unroll
        for (int k0 = 0; k0 < K; k0 += G) {
            T* fg = faces + (FB == 2 ? ((k0 / G) & 1) * G * NF : 0);
            if (FB == 1 && k0 > 0) __syncthreads();  // the previous group's update is done with the faces
            T fnv[G];
            T pv[IMEX ? G : 1];   // IMEX stage 2: P at the node
            if constexpr (PAIRS) {
                // populations 2q and 2q+1 of the group side by side: the x-faces
                // of both as one packed pair, then the y-faces of both; faces
                // stored as pairs [TY][TX + 1] and [TY + 1][TX] of V per q
#pragma unroll
                for (int q = 0; q < G / 2; ++q) {
                    const int ka = k0 + 2 * q;
                    const T* ta = tiles + ka * HXY;
                    const T* tb = ta + HXY;
                    V* fx2 = reinterpret_cast<V*>(fg) + q * NF;
                    V* fy2 = fx2 + NFX;
                    const double vxd = vx_of<Q1>(ka), vyd = vy_of<Q1>(ka);   // also the signs of ka + 1
                    const int xo = vxd > 0 ? 1 : 6, xs = vxd > 0 ? 1 : -1;
                    const int yo = vyd > 0 ? 0 : 5 * HXP, ys = vyd > 0 ? HXP : -HXP;
                    auto face = [&](int base, int o, int st) {
                        const T* a = ta + base + o;
                        const T* b = tb + base + o;
                        return weno5_pair<T>(P::mk(a[0], b[0]), P::mk(a[st], b[st]), P::mk(a[2 * st], b[2 * st]),
                                             P::mk(a[3 * st], b[3 * st]), P::mk(a[4 * st], b[4 * st]), eps);
                    };
                    fx2[ty * (TX + 1) + tx] = face(xrow, xo, xs);
                    fy2[ty * TX + tx] = face(ycol, yo, ys);
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int k = ka + h;
                        fnv[2 * q + h] = (node_in && active && LBM_BC_NODE(dp, K, cell + k * plane)) ? fnp[k * plane] : T(0);
                        if constexpr (IMEX)
                            pv[2 * q + h] = (stage == 2 && active && LBM_BC_NODE(dp, K, cell + k * plane)) ? ppn[k * plane] : T(0);
                    }
                }
                // the tile's right-edge x-faces and top-edge y-faces of the
                // group's pairs, through one copy of the code (pair and stencil
                // direction selected at run time): edge tasks e < NXE are the
                // right-edge x-faces of all pairs and rows, one (pair, row) per
                // lane; task NXE + q is pair q's top-edge y-faces, one column
                // per lane; task e is evaluated by warp e mod TY
                constexpr int NPR = G / 2;
                constexpr int NXE = (NPR * TY + 31) / 32;
                for (int e = ty; e < NXE + NPR; e += TY) {
                    const bool xax = e < NXE;
                    const int lx = e * 32 + tx;                    // x task: (pair, row) of this lane
                    const bool xok = lx < NPR * TY;
                    const int q = xax ? (xok ? lx / TY : 0) : e - NXE;
                    const int row = xax ? (xok ? lx % TY : 0) : 0;
                    const T* ta = tiles + (k0 + 2 * q) * HXY;
                    const T* tb = ta + HXY;
                    V* fx2 = reinterpret_cast<V*>(fg) + q * NF;
                    // pair q's nodes along x are (2q mod Q1, +1): both below the
                    // middle of the 1D set (v_x < 0) or both above (v_x > 0);
                    // v_y has one sign in the whole group (whole rows)
                    const bool xpos = 2 * ((2 * q) % Q1) >= Q1;
                    const bool ypos = vy_of<Q1>(k0) > 0;
                    const int st = xax ? (xpos ? 1 : -1) : (ypos ? HXP : -HXP);
                    const int base = xax ? (row + 3) * HXP + TX + (xpos ? 1 : 6) : eycol + (ypos ? 0 : 5 * HXP);
                    const T* a = ta + base;
                    const T* b = tb + base;
                    const V f = weno5_pair<T>(P::mk(a[0], b[0]), P::mk(a[st], b[st]), P::mk(a[2 * st], b[2 * st]),
                                              P::mk(a[3 * st], b[3 * st]), P::mk(a[4 * st], b[4 * st]), eps);
                    if (xax) {
                        if (xok) fx2[row * (TX + 1) + TX] = f;
                    } else {
                        fx2[NFX + TY * TX + tx] = f;
                    }
                }
            } else {
#pragma unroll
                for (int p = 0; p < G; ++p) {
                    const int k = k0 + p;
                    if (k >= K) break;
                    const T* tk = tiles + k * HXY;
                    T* fx = fg + p * NF;            // [TY][TX + 1]
                    T* fy = fx + NFX;               // [TY + 1][TX]
                    const double vxd = vx_of<Q1>(k), vyd = vy_of<Q1>(k);
                    // upwind stencil of the face on the low side of node (c, r):
                    // x, v > 0: cols c+1..c+5 of row r+3; v < 0: cols c+6..c+2
                    // y, v > 0: rows r..r+4 of col c+4; v < 0: rows r+5..r+1
                    const int xo = vxd > 0 ? 1 : 6, xs = vxd > 0 ? 1 : -1;
                    const int yo = vyd > 0 ? 0 : 5 * HXP, ys = vyd > 0 ? HXP : -HXP;
                    {
                        const T* px = tk + xrow + xo;
                        const T* py = tk + ycol + yo;
                        const V f = weno5_pair<T>(P::mk(px[0], py[0]), P::mk(px[xs], py[ys]), P::mk(px[2 * xs], py[2 * ys]),
                                                  P::mk(px[3 * xs], py[3 * ys]), P::mk(px[4 * xs], py[4 * ys]), eps);
                        fx[ty * (TX + 1) + tx] = f.x;
                        fy[ty * TX + tx] = f.y;
                    }
                    if (ty == p % TY) {
                        const T* px = tk + exrow + xo;
                        const T* py = tk + eycol + yo;
                        const V f = weno5_pair<T>(P::mk(px[0], py[0]), P::mk(px[xs], py[ys]), P::mk(px[2 * xs], py[2 * ys]),
                                                  P::mk(px[3 * xs], py[3 * ys]), P::mk(px[4 * xs], py[4 * ys]), eps);
                        if (tx < TY) fx[tx * (TX + 1) + TX] = f.x;
                        fy[TY * TX + tx] = f.y;
                    }
                    fnv[p] = (node_in && active && LBM_BC_NODE(dp, K, cell + k * plane)) ? fnp[k * plane] : T(0);
                    if constexpr (IMEX)
                        pv[p] = (stage == 2 && active && LBM_BC_NODE(dp, K, cell + k * plane)) ? ppn[k * plane] : T(0);
                }
            }
            __syncthreads();
            if (active) {
                V pxl, pxr, pyb, pyt;   // face pairs of populations 2q, 2q+1 (PAIRS)
#pragma unroll
                for (int p = 0; p < G; ++p) {
                    const int k = k0 + p;
                    if (k >= K) break;
                    const T* tk = tiles + k * HXY;
                    const T* fx = fg + p * NF;
                    const T* fy = fx + NFX;
                    const double vxd = vx_of<Q1>(k), vyd = vy_of<Q1>(k);
                    // the four faces around the node: low/high x, low/high y
                    T fxl, fxh, fyl, fyh;
                    if constexpr (PAIRS) {
                        if ((p & 1) == 0) {
                            const V* fx2 = reinterpret_cast<const V*>(fg) + (p >> 1) * NF;
                            const V* fy2 = fx2 + NFX;
                            pxl = fx2[ty * (TX + 1) + tx];
                            pxr = fx2[ty * (TX + 1) + tx + 1];
                            pyb = fy2[ty * TX + tx];
                            pyt = fy2[(ty + 1) * TX + tx];
                        }
                        fxl = (p & 1) ? pxl.y : pxl.x;
                        fxh = (p & 1) ? pxr.y : pxr.x;
                        fyl = (p & 1) ? pyb.y : pyb.x;
                        fyh = (p & 1) ? pyt.y : pyt.x;
                    } else {
                        fxl = fx[ty * (TX + 1) + tx];
                        fxh = fx[ty * (TX + 1) + tx + 1];
                        fyl = fy[ty * TX + tx];
                        fyh = fy[(ty + 1) * TX + tx];
                    }
                    // flux difference F(i+1/2) - F(i-1/2) = (c+ - c-) + (d+ - d-)/12:
                    // the upwind node values c differ by one node (exact for
                    // close values), the stored corrections d = 12 (face - c) are small
                    const T vx = (T)vxd, vy = (T)vyd;
                    const T uk = tk[cidx];
                    // a = v_x dF_x + v_y dF_y (zero components drop out)
                    T a = T(0);
                    if (vxd != 0.0) {
                        const T dc = vxd > 0 ? uk - tk[cidx - 1] : tk[cidx + 1] - uk;
                        a = vx * ((fxh - fxl) * T(1.0 / 12.0) + dc);
                    }
                    if (vyd != 0.0) {
                        const T dc = vyd > 0 ? uk - tk[cidx - HXP] : tk[cidx + HXP] - uk;
                        a += vy * ((fyh - fyl) * T(1.0 / 12.0) + dc);
                    }
                    T xi, geq;
                    if constexpr (sizeof(T) == 4 && Q1 == 4) {
                        xi = ec.xi(k);
                        geq = (T)w_of<Q1>(k) * (hr * (xi * xi - usq) + ec.lin(k));
                    } else {
                        xi = vx * ux + vy * uy;
                        geq = (T)w_of<Q1>(k) * (hr * (xi * xi - usq) + (vx * jxc + (vy * jyc + drc)));
                    }
                    if constexpr (IMEX) {
                        // dt A(Y)_k and dt C(Y)_k (from the stage input at the node)
                        const T dta = -(a * cdx);
                        const T dtc = -(c1 * (fnv[p] - geq));
                        if (LBM_BC_NODE(dp, K, cell + k * plane)) {
                            if (stage == 1) {
                                op[k * plane] = fnv[p] + (dta + T(1.0 - 2.0 * IMEX_GAMMA) * dtc);   // Z
                                pout[k * plane] = fnv[p] + T(2.0 * IMEX_GAMMA) * dtc;             // P
                            } else {
                                op[k * plane] = pv[p] + T(0.5) * ((fnv[p] - pv[p]) + (dta + dtc));
                            }
                        }
                    } else {
                        // dt L(u)_k = -(dt/dx) a - (u - geq) dt/tau
                        const T inc = (geq - uk) * dtt - a * cdx;
                        // stage combination in increment form: one rounding of the
                        // stored value per stage (u - f^n is exact for close values)
                        if (LBM_BC_NODE(dp, K, cell + k * plane))
                            op[k * plane] = stage == 1 ? uk + inc : fnv[p] + cb * ((uk - fnv[p]) + inc);
                    }
                }
            }
        }
    }
}

int fd_tile_tx(int v) { return (v >= 0 && v < FD_NTILES) ? FD_TX : 0; }
int fd_tile_ty(int v) {
    switch (v) {
        case FD_T32x8: return 8;
        case FD_T32x4: return 4;
        case FD_T32x16: return 16;
        case FD_T32x2: return 2;
    }
    return 0;
}

template <typename T, int Q1, bool IMEX>
static const void* fd_kernel_ptr_q(int tile) {
    switch (tile) {
        case FD_T32x8: return (const void*)fd_stage_kernel<T, Q1, 8, IMEX>;
        case FD_T32x4: return (const void*)fd_stage_kernel<T, Q1, 4, IMEX>;
        case FD_T32x16: return (const void*)fd_stage_kernel<T, Q1, 16, IMEX>;
        case FD_T32x2: return (const void*)fd_stage_kernel<T, Q1, 2, IMEX>;
    }
    return nullptr;
}

template <typename T, bool IMEX>
static const void* fd_kernel_ptr(int tile, int q1) {
    switch (q1) {
        case 3: return fd_kernel_ptr_q<T, 3, IMEX>(tile);
        case 4: return fd_kernel_ptr_q<T, 4, IMEX>(tile);
        case 5: return fd_kernel_ptr_q<T, 5, IMEX>(tile);
    }
    return nullptr;
}

template <typename T, int Q1>
static size_t fd_smem_q(int tile) {
    switch (tile) {
        case FD_T32x8: return fd_smem_bytes<T, Q1, 8>();
        case FD_T32x4: return fd_smem_bytes<T, Q1, 4>();
        case FD_T32x16: return fd_smem_bytes<T, Q1, 16>();
        case FD_T32x2: return fd_smem_bytes<T, Q1, 2>();
    }
    return 0;
}

template <typename T>
static size_t fd_smem(int tile, int q1) {
    switch (q1) {
        case 3: return fd_smem_q<T, 3>(tile);
        case 4: return fd_smem_q<T, 4>(tile);
        case 5: return fd_smem_q<T, 5>(tile);
    }
    return 0;
}

static const void* fd_fn(int precision, int tile, int q1, int scheme) {
    if (scheme == LBM_TS_IMEX)
        return precision == LBM_FP64 ? fd_kernel_ptr<double, true>(tile, q1) : fd_kernel_ptr<float, true>(tile, q1);
    return precision == LBM_FP64 ? fd_kernel_ptr<double, false>(tile, q1) : fd_kernel_ptr<float, false>(tile, q1);
}
static size_t fd_bytes(int precision, int tile, int q1) {
    return precision == LBM_FP64 ? fd_smem<double>(tile, q1) : fd_smem<float>(tile, q1);
}

// Opt each variant (both schemes' kernels) into the dynamic shared memory it
// needs; once per process. A variant that cannot fit on this device is
// refused (and the CUDA error state cleared).
static cudaError_t fd_prepare(int precision, int tile, int q1) {
    static int state[2][FD_NTILES][3] = {};  // 0 unknown, 1 ready, 2 does not fit
    const int p = precision == LBM_FP64 ? 0 : 1;
    int& st = state[p][tile][q1 - 3];
    if (st == 1) return cudaSuccess;
    if (st == 2) return cudaErrorInvalidConfiguration;
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
        cudaGetLastError();
        return cudaErrorInvalidConfiguration;
    }
    const size_t need = fd_bytes(precision, tile, q1);
    if (need > (size_t)optin) {
        st = 2;
        return cudaErrorInvalidConfiguration;
    }
    for (int scheme : {LBM_TS_RK3, LBM_TS_IMEX}) {
        cudaError_t e = cudaFuncSetAttribute(fd_fn(precision, tile, q1, scheme),
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need);
        if (e != cudaSuccess) {
            cudaGetLastError();
            st = 2;
            return cudaErrorInvalidConfiguration;
        }
    }
    st = 1;
    return cudaSuccess;
}

cudaError_t launch_fd_stage(int precision, int q1, int scheme, int tile, int grid, const GroupDev& g, int j,
                            int stage, cudaStream_t s) {
    if (tile < 0 || tile >= FD_NTILES || grid <= 0 || q1 < 3 || q1 > 5 ||
        (scheme != LBM_TS_RK3 && scheme != LBM_TS_IMEX && scheme != LBM_TS_RK3_FUSED) || stage < 1 ||
        stage > fd_stages(scheme))
        return cudaErrorInvalidValue;
    if (scheme == LBM_TS_RK3_FUSED) return launch_fd_fused(precision, q1, tile, grid, g, j, s);
    const void* fn = fd_fn(precision, tile, q1, scheme);
    cudaError_t e = fd_prepare(precision, tile, q1);
    if (e != cudaSuccess) return e;
    GroupDev gg = g;
    int jj = j, ss = stage;
    void* args[] = {&gg, &jj, &ss};
    return cudaLaunchKernel(fn, dim3(grid), dim3(fd_tile_tx(tile), fd_tile_ty(tile)), args, fd_bytes(precision, tile, q1), s);
}

bool fd_variant_fits(int precision, int q1, int tile, int scheme) {
    if (scheme == LBM_TS_RK3_FUSED) return fd_fused_fits(precision, q1, tile);
    return tile >= 0 && tile < FD_NTILES && q1 >= 3 && q1 <= 5 && fd_prepare(precision, tile, q1) == cudaSuccess;
}

int fd_blocks_per_sm(int precision, int q1, int tile, int scheme) {
    if (scheme == LBM_TS_RK3_FUSED) return fd_fused_blocks_per_sm(precision, q1, tile);
    if (!fd_variant_fits(precision, q1, tile, scheme)) return 1;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fd_fn(precision, tile, q1, LBM_TS_RK3),
                                                      fd_tile_tx(tile) * fd_tile_ty(tile),
                                                      fd_bytes(precision, tile, q1)) != cudaSuccess)
        return 1;
    return n > 0 ? n : 1;
}

}  // namespace lbm
