// Temporally blocked FD step (LBM_TS_RK3_FUSED): the three SSP-RK3 stages of
// one step of Eq. (evolution) (Sec. 2: WENO-5 advection, BGK collision from
// each stage's own moments, TVD Runge-Kutta in Shu-Osher form) for one tile
// of 32 x TY nodes in a single launch. Each stage widens the stencil by 3
// nodes, so a tile reads f^n on a halo of 9 nodes and computes
//   stage 1 on the tile + 6 nodes   (region R1, 44 x (TY + 12) nodes),
//   stage 2 on the tile + 3 nodes   (region R2, 38 x (TY + 6) nodes),
//   stage 3 on the tile              (32 x TY nodes),
// keeping f^(1) and f^(2) in shared memory: per lattice update it reads Q and
// writes Q values of device memory (2Q, against 8Q for the three stage
// launches), at the price of the halo's extra node-stages (6.5 per tile node
// for 32 x 8 tiles instead of 3).
//
// The arithmetic of every stage is that of the stage kernels (kernels_fd.cu):
// the same WENO-5 interface values (12 (face - c), c the upwind node value),
// flux differences (c+ - c-) + (d+ - d-)/12, BGK term with moments of the
// stage input and, for FP32 deviation storage, the moment-exact collision
// (residual moments of u - f^eq removed through shifted moments), and the
// increment-form stage combinations f^n + cb ((u - f^n) + dt L(u)).
//
// State: two buffers; a step reads buf[cur] and writes buf[cur ^ 1] (a tile
// cannot write f^(n+1) over f^n, which neighbouring tiles still read for
// their halos); cur flips with every step, as for two-buffer CS lattices.
//
// Per tile and stage, populations go in groups of G: faces of the group's
// populations on the stage's region (one packed x/y pair per position), one
// barrier, the node updates, one barrier. f^n is staged per group (the halo
// tile of the group's populations); the moments of the stage input are
// formed once per stage and node, before the groups. Stage 2 updates f^(1)
// into f^(2) in place: a group's new values are held in registers until every
// thread has read the group's old neighbour values, then written.
#include <atomic>

#include "fd_common.cuh"
#include "kernels.h"
#include "ptx.cuh"

namespace lbm {

// cp.async groups: close the group of copies issued so far; wait until at
// most N groups are still in flight
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait_prior() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

template <typename T, int Q1, int TY>
struct FusedGeo {
    static constexpr int K = Q1 * Q1;
    // threads per block (FP32 with 1024 threads, 64 registers each: 2.5%
    // slower at 32 x 16 tiles)
    static constexpr int NT = sizeof(T) == 4 ? 512 : 256;
    static constexpr int G = sizeof(T) == 4 ? 4 : 2;        // populations per face group
    static constexpr int VEC = 16 / (int)sizeof(T);         // values per 16-byte copy
    // staged f^n of a group: columns x0 - 12 .. x0 + 43 (16-byte aligned
    // rows; the stencils need x0 - 9 .. x0 + 40), rows y0 - 9 .. y0 + TY + 8
    static constexpr int W0 = 56, H0 = TY + 18;
    // stage 1 region R1 (also the layout of the f^(1) / f^(2) buffer):
    // columns x0 - 6 .. x0 + 37, rows y0 - 6 .. y0 + TY + 5
    static constexpr int W1 = 44, H1 = TY + 12;
    // stage 2 region R2: columns x0 - 3 .. x0 + 34, rows y0 - 3 .. y0 + TY + 2
    static constexpr int W2 = 38, H2 = TY + 6;
    // face arrays [G][FH][FW]: x-face (r, c) is the face on the low-x side of
    // node (r, c) (c = W: the high face of the last column), y-face (r, c)
    // the face below node (r, c) (r = H: above the last row)
    static constexpr int FW = W1 + 1, FH = H1 + 1;
    static constexpr int NM = 6;   // per-node moments kept: ux, uy, rho/2, drc, jxc, jyc
    static constexpr size_t n_s1 = (size_t)K * H1 * W1;
    static constexpr size_t n_r0 = (size_t)G * H0 * W0;
    static constexpr size_t n_f = (size_t)G * FH * FW;
    static constexpr size_t n_m = (size_t)NM * H1 * W1;
    static constexpr size_t n_red = sizeof(double) * (NT / 32) * NOBS;
    // two staging buffers (the next group's f^n is copied while the current
    // group computes) where they fit next to the rest (opt-in limit of the
    // device, 227 KiB, less 2 KiB for the static shared variables), else one
    static constexpr int NB = sizeof(T) * (n_s1 + 2 * n_r0 + 2 * n_f + n_m) + n_red <= 227 * 1024 - 2048 ? 2 : 1;
    static constexpr size_t bytes = sizeof(T) * (n_s1 + NB * n_r0 + 2 * n_f + n_m) + n_red;
    // stage 2 nodes per thread (results held before the in-place write)
    static constexpr int NR2 = (H2 * W2 + NT - 1) / NT;
    static_assert((n_s1 * sizeof(T)) % 16 == 0 && (W0 * sizeof(T)) % 16 == 0, "16-byte aligned staging rows");
    static_assert(((n_s1 + n_r0 + 2 * n_f + n_m) * sizeof(T)) % 8 == 0 && (n_r0 * sizeof(T)) % 16 == 0,
                  "aligned staging buffers and reduction scratch");
};

// x- and y-face on the low side of the node at (R, C) of a region stored
// with row width W, for one population whose velocity components are
// positive (xp, yp) or not: the upwind stencils of the stage kernels
// (v > 0: f_{i-3..i+1}; v <= 0: f_{i+2..i-2}).
template <typename T>
__device__ __forceinline__ typename Pr<T>::V fused_faces(const T* in, int W, int R, int C, bool xp, bool yp,
                                                         typename Pr<T>::V eps) {
    using P = Pr<T>;
    const int bx = R * W + (xp ? C - 3 : C + 2), sx = xp ? 1 : -1;
    const int by = (yp ? R - 3 : R + 2) * W + C, sy = yp ? W : -W;
    return weno5_pair<T>(P::mk(in[bx], in[by]), P::mk(in[bx + sx], in[by + sy]), P::mk(in[bx + 2 * sx], in[by + 2 * sy]),
                         P::mk(in[bx + 3 * sx], in[by + 3 * sy]), P::mk(in[bx + 4 * sx], in[by + 4 * sy]), eps);
}

template <typename T, int Q1, int TY>
__global__ void __launch_bounds__(FusedGeo<T, Q1, TY>::NT, 1) fd_fused_kernel(GroupDev g, int j) {
    using Ge = FusedGeo<T, Q1, TY>;
    using P = Pr<T>;
    using V = typename P::V;
    constexpr int K = Ge::K, NT = Ge::NT, G = Ge::G, VEC = Ge::VEC;
    constexpr int W0 = Ge::W0, H0 = Ge::H0, W1 = Ge::W1, H1 = Ge::H1, W2 = Ge::W2, H2 = Ge::H2;
    constexpr int FW = Ge::FW;
    constexpr int N1 = H1 * W1;   // nodes of R1 (plane of the f^(1) buffer)
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* s1 = reinterpret_cast<T*>(smem_raw);   // [K][H1][W1]: f^(1) on R1, then f^(2) on R2
    T* r0 = s1 + Ge::n_s1;                     // [NB][G][H0][W0]: f^n of a group's populations
    T* fxs = r0 + Ge::NB * Ge::n_r0;           // [G][FH][FW]
    T* fys = fxs + Ge::n_f;                    // [G][FH][FW]
    T* mom = fys + Ge::n_f;                    // [NM][N1]
    double* red = reinterpret_cast<double*>(mom + Ge::n_m);
    __shared__ long long s_row[H0];            // wrapped row offsets of the staged rows
    __shared__ int s_col[W0];                  // wrapped columns of the staged columns
    __shared__ int s_obs;
    __shared__ T s_vx[K], s_vy[K], s_w[K];

    const int n_lat = g.hdr[0];
    const int total = g.hdr[1];
    const int tid = threadIdx.x;
    if (tid < K) {
        s_vx[tid] = (T)vx_of<Q1>(tid);
        s_vy[tid] = (T)vy_of<Q1>(tid);
        s_w[tid] = (T)w_of<Q1>(tid);
    }

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
        const int x0 = bx * 32, y0 = by * TY;
        const int cur = dp->cur ^ (j & 1);
        const T* __restrict__ Fn = static_cast<const T*>(dp->buf[cur]);
        T* __restrict__ out = static_cast<T*>(dp->buf[cur ^ 1]);
        const T rz = lat_val<T>(dp->rho0, dp->rho0_f);
        const T cdx = lat_val<T>(dp->cdx, dp->cdx_f);
        const T dtt = lat_val<T>(dp->dt_tau, dp->dt_tau_f);
        const V eps = P::sp(lat_val<T>(dp->eps, dp->eps_f) * T(12.0 / 13.0));
        const bool interior = x0 >= 12 && x0 + 44 <= nx && y0 >= 9 && y0 + TY + 9 <= ny;

        __syncthreads();   // the previous item is done with shared memory
        if (tid == 0) s_obs = observe_now(*dp, j);
        for (int i = tid; i < H0 + W0; i += NT) {
            if (i < H0) s_row[i] = (long long)wrapi(y0 - 9 + i, ny) * pitch;
            else s_col[i - H0] = wrapi(x0 - 12 + (i - H0), nx);
        }
        __syncthreads();

        // Moments of a stage input at one node (Eq. f_moments_discrete,
        // ascending k) into mom[.][p]; FP32: shifted by the residual moments
        // of u - f^eq (the stage kernels' moment-exact collision).
        auto node_moments = [&](const T (&u)[K], int p, T& dr, T& jx, T& jy, T& ux, T& uy) {
            dr = T(0);
            jx = T(0);
            jy = T(0);
#pragma unroll
            for (int k = 0; k < K; ++k) {
                dr += u[k];
                if (vx_of<Q1>(k) != 0.0) jx += u[k] * (T)vx_of<Q1>(k);
                if (vy_of<Q1>(k) != 0.0) jy += u[k] * (T)vy_of<Q1>(k);
            }
            const T rho = rz + dr;
            const T inv = T(1) / rho;
            ux = jx * inv;
            uy = jy * inv;
            const T usq = ux * ux + uy * uy;
            const T hr = T(0.5) * rho;
            T R0 = T(0), R1x = T(0), R1y = T(0);
            if constexpr (sizeof(T) == 4) {
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    const T vx = (T)vx_of<Q1>(k), vy = (T)vy_of<Q1>(k);
                    const T xi = vx * ux + vy * uy;
                    const T geq = (T)w_of<Q1>(k) * (hr * (xi * xi - usq) + (vx * jx + (vy * jy + dr)));
                    const T d = u[k] - geq;
                    R0 += d;
                    if (vx_of<Q1>(k) != 0.0) R1x += d * (T)vx_of<Q1>(k);
                    if (vy_of<Q1>(k) != 0.0) R1y += d * (T)vy_of<Q1>(k);
                }
            }
            mom[0 * N1 + p] = ux;
            mom[1 * N1 + p] = uy;
            mom[2 * N1 + p] = hr;
            mom[3 * N1 + p] = dr + R0;
            mom[4 * N1 + p] = jx + R1x;
            mom[5 * N1 + p] = jy + R1y;
        };
        // the stored moments of a node (formed once per node and stage)
        struct NodeM {
            T ux, uy, usq, hr, drc, jxc, jyc;
        };
        auto load_m = [&](int p) {
            NodeM m;
            m.ux = mom[0 * N1 + p];
            m.uy = mom[1 * N1 + p];
            m.hr = mom[2 * N1 + p];
            m.drc = mom[3 * N1 + p];
            m.jxc = mom[4 * N1 + p];
            m.jyc = mom[5 * N1 + p];
            m.usq = m.ux * m.ux + m.uy * m.uy;
            return m;
        };
        // velocity components and weights of a group's populations (uniform
        // across the block), loaded once per group
        struct GroupC {
            T vx[G], vy[G], w[G];
        };
        auto group_consts = [&](int k0) {
            GroupC gc;
#pragma unroll
            for (int pp = 0; pp < G; ++pp) {
                const int k = k0 + pp < K ? k0 + pp : K - 1;
                gc.vx[pp] = s_vx[k];
                gc.vy[pp] = s_vy[k];
                gc.w[pp] = s_w[k];
            }
            return gc;
        };
        // faces of the group's populations on a region of W x H nodes whose
        // node (r, c) sits at (r + OY, c + OX) of the input `in` (row width
        // WI, population planes `pl` apart): positions outer, populations inner
        auto group_faces = [&](const GroupC& gc, const T* in, long long pl, int WI, int OY, int OX, int W, int H,
                               int ng) {
            const int npos = (H + 1) * (W + 1);
            for (int pos = tid; pos < npos; pos += NT) {
                const int r = pos / (W + 1), c = pos - r * (W + 1);
#pragma unroll
                for (int pp = 0; pp < G; ++pp) {
                    if (pp < ng) {
                        const V f = fused_faces<T>(in + pp * pl, WI, r + OY, c + OX, gc.vx[pp] > T(0), gc.vy[pp] > T(0),
                                                   eps);
                        if (r < H) fxs[pp * Ge::FH * FW + r * FW + c] = f.x;
                        if (c < W) fys[pp * Ge::FH * FW + r * FW + c] = f.y;
                    }
                }
            }
        };
        // dt L(u)_k of population pp of the group at node (r, c) of a region
        // (input as in group_faces) from its four faces, its upwind
        // neighbours and the node's moments (the stage kernels' formulas);
        // uk = the stage input at the node
        auto node_inc = [&](const GroupC& gc, const NodeM& m, const T* tk, int WI, int OY, int OX, int pp, int r, int c,
                            T& uk) {
            const int R = r + OY, C = c + OX;
            uk = tk[R * WI + C];
            const T vx = gc.vx[pp], vy = gc.vy[pp];
            const T dcx = vx > T(0) ? uk - tk[R * WI + C - 1] : tk[R * WI + C + 1] - uk;
            const T dcy = vy > T(0) ? uk - tk[(R - 1) * WI + C] : tk[(R + 1) * WI + C] - uk;
            const T* fx = fxs + pp * Ge::FH * FW;
            const T* fy = fys + pp * Ge::FH * FW;
            T a = T(0);
            if (vx != T(0)) a = vx * ((fx[r * FW + c + 1] - fx[r * FW + c]) * T(1.0 / 12.0) + dcx);
            if (vy != T(0)) a += vy * ((fy[(r + 1) * FW + c] - fy[r * FW + c]) * T(1.0 / 12.0) + dcy);
            const T xi = vx * m.ux + vy * m.uy;
            const T geq = gc.w[pp] * (m.hr * (xi * xi - m.usq) + (vx * m.jxc + (vy * m.jyc + m.drc)));
            return (geq - uk) * dtt - a * cdx;
        };

        // asynchronous copies of the halo tiles of f^n (rows y0 - 9 .., columns
        // x0 - 12 ..) of populations k0 .. k0 + G - 1 into dst
        auto stage_group = [&](int k0, T* dst) {
            const int ng = K - k0 < G ? K - k0 : G;
            constexpr int RV = W0 / VEC;   // 16-byte chunks per staged row
            if (interior || nx % VEC == 0) {
                // interior: rows are 16-byte aligned (x0 - 12 is a multiple of
                // VEC, the pitch of 32); periodic edge with nx a multiple of
                // VEC: no chunk straddles the wrap point
                for (int t = tid; t < ng * H0 * RV; t += NT) {
                    const int pp = t / (H0 * RV), rem = t - pp * (H0 * RV);
                    const int r = rem / RV, cc = rem - r * RV;
                    const long long src = (long long)(k0 + pp) * plane +
                                          (interior ? (long long)(y0 - 9 + r) * pitch + (x0 - 12 + cc * VEC)
                                                    : s_row[r] + s_col[cc * VEC]);
                    if (LBM_BC_NODE(dp, K, src) && LBM_BC_NODE(dp, K, src + VEC - 1))
                        cp_async16(dst + pp * H0 * W0 + r * W0 + cc * VEC, Fn + src);
                }
            } else {
                for (int t = tid; t < ng * H0 * W0; t += NT) {
                    const int pp = t / (H0 * W0), rem = t - pp * (H0 * W0);
                    const int r = rem / W0, c = rem - r * W0;
                    const long long src = (long long)(k0 + pp) * plane + s_row[r] + s_col[c];
                    if (LBM_BC_NODE(dp, K, src)) cp_async_small<sizeof(T)>(dst + rem + pp * H0 * W0, Fn + src);
                }
            }
        };

        // ---- stage 1: f^(1) = f^n + dt L(f^n) on R1 ----
        // the first group's f^n tiles are copied while the moments are formed
        stage_group(0, r0);
        cp_async_commit();
        // moments of f^n at the R1 nodes (read from device memory), and the
        // observables of f^n over the tile's own nodes
        {
            T acc[NOBS] = {T(0), T(0), T(0), T(0)};
            for (int p = tid; p < N1; p += NT) {
                const int r = p / W1, c = p - r * W1;
                const long long off = s_row[r + 3] + s_col[c + 6];
                T u[K];
#pragma unroll
                for (int k = 0; k < K; ++k)
                    u[k] = LBM_BC_NODE(dp, K, k * plane + off) ? Fn[k * plane + off] : T(0);
                T dr, jx, jy, ux, uy;
                node_moments(u, p, dr, jx, jy, ux, uy);
                const int x = x0 + c - 6, y = y0 + r - 6;
                if (s_obs && r >= 6 && r < 6 + TY && c >= 6 && c < 38 && x < nx && y < ny) {
                    acc[0] += dr;
                    acc[1] += jx;
                    acc[2] += jy;
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
                        acc[3] += (pc == 0 ? ux : uy) * pxv * pyv;
                    }
                }
            }
            // no trailing barrier: `red` is next written after this item's barriers
            if (s_obs) block_reduce_obs<T, NT, false>(acc, dp->partials + (long long)local * NOBS, red);
        }
        for (int k0 = 0, gi = 0; k0 < K; k0 += G, ++gi) {
            const int ng = K - k0 < G ? K - k0 : G;
            T* rg = r0 + (gi % Ge::NB) * Ge::n_r0;   // this group's staged f^n
            if (Ge::NB == 2 && k0 + G < K) {
                // copy the next group's tiles into the other buffer (free since
                // the previous group's last barrier), wait for this group's
                stage_group(k0 + G, r0 + ((gi + 1) % 2) * Ge::n_r0);
                cp_async_commit();
                cp_async_wait_prior<1>();
            } else {
                cp_async_wait_prior<0>();
            }
            __syncthreads();
            const GroupC gc = group_consts(k0);
            group_faces(gc, rg, (long long)H0 * W0, W0, 3, 6, W1, H1, ng);
            __syncthreads();
            for (int p = tid; p < N1; p += NT) {
                const int r = p / W1, c = p - r * W1;
                const NodeM m = load_m(p);
#pragma unroll
                for (int pp = 0; pp < G; ++pp) {
                    if (pp < ng) {
                        T uk;
                        const T inc = node_inc(gc, m, rg + pp * H0 * W0, W0, 3, 6, pp, r, c, uk);
                        s1[(k0 + pp) * N1 + p] = uk + inc;
                    }
                }
            }
            __syncthreads();   // before the next group's staging and faces
            if (Ge::NB == 1 && k0 + G < K) {
                stage_group(k0 + G, r0);
                cp_async_commit();
            }
        }

        // ---- stage 2: f^(2) = f^n + 1/4 ((f^(1) - f^n) + dt L(f^(1))) on R2 ----
        for (int p = tid; p < H2 * W2; p += NT) {
            const int r = p / W2, c = p - r * W2;
            T u[K];
#pragma unroll
            for (int k = 0; k < K; ++k) u[k] = s1[k * N1 + (r + 3) * W1 + c + 3];
            T dr, jx, jy, ux, uy;
            node_moments(u, p, dr, jx, jy, ux, uy);
        }
        __syncthreads();
        for (int k0 = 0; k0 < K; k0 += G) {
            const int ng = K - k0 < G ? K - k0 : G;
            const GroupC gc = group_consts(k0);
            group_faces(gc, s1 + k0 * N1, (long long)N1, W1, 3, 3, W2, H2, ng);
            __syncthreads();
            T res[Ge::NR2][G];
#pragma unroll
            for (int i = 0; i < Ge::NR2; ++i) {
                const int p = tid + i * NT;
                if (p < H2 * W2) {
                    const int r = p / W2, c = p - r * W2;
                    const NodeM m = load_m(p);
#pragma unroll
                    for (int pp = 0; pp < G; ++pp) {
                        if (pp < ng) {
                            const int k = k0 + pp;
                            T uk;
                            const T inc = node_inc(gc, m, s1 + k * N1, W1, 3, 3, pp, r, c, uk);
                            const long long off = (long long)k * plane + s_row[r + 6] + s_col[c + 9];
                            const T fn = LBM_BC_NODE(dp, K, off) ? Fn[off] : T(0);
                            res[i][pp] = fn + T(0.25) * ((uk - fn) + inc);
                        }
                    }
                }
            }
            __syncthreads();   // every old value of the group has been read
#pragma unroll
            for (int i = 0; i < Ge::NR2; ++i) {
                const int p = tid + i * NT;
                if (p < H2 * W2) {
                    const int r = p / W2, c = p - r * W2;
#pragma unroll
                    for (int pp = 0; pp < G; ++pp)
                        if (pp < ng) s1[(k0 + pp) * N1 + (r + 3) * W1 + c + 3] = res[i][pp];
                }
            }
        }
        __syncthreads();

        // ---- stage 3: f^(n+1) = f^n + 2/3 ((f^(2) - f^n) + dt L(f^(2))) on the tile ----
        for (int p = tid; p < TY * 32; p += NT) {
            const int r = p / 32, c = p - r * 32;
            T u[K];
#pragma unroll
            for (int k = 0; k < K; ++k) u[k] = s1[k * N1 + (r + 6) * W1 + c + 6];
            T dr, jx, jy, ux, uy;
            node_moments(u, p, dr, jx, jy, ux, uy);
        }
        __syncthreads();
        for (int k0 = 0; k0 < K; k0 += G) {
            const int ng = K - k0 < G ? K - k0 : G;
            const GroupC gc = group_consts(k0);
            group_faces(gc, s1 + k0 * N1, (long long)N1, W1, 6, 6, 32, TY, ng);
            __syncthreads();
            for (int p = tid; p < TY * 32; p += NT) {
                const int r = p / 32, c = p - r * 32;
                const int x = x0 + c, y = y0 + r;
                if (x < nx && y < ny) {
                    const NodeM m = load_m(p);
#pragma unroll
                    for (int pp = 0; pp < G; ++pp) {
                        if (pp < ng) {
                            const int k = k0 + pp;
                            T uk;
                            const T inc = node_inc(gc, m, s1 + k * N1, W1, 6, 6, pp, r, c, uk);
                            const long long off = (long long)k * plane + (long long)y * pitch + x;
                            if (LBM_BC_NODE(dp, K, off)) {
                                const T fn = Fn[off];
                                out[off] = fn + T(2.0 / 3.0) * ((uk - fn) + inc);
                            }
                        }
                    }
                }
            }
            __syncthreads();   // before the next group's faces
        }
    }
}

// Output tile heights of the fused kernel: 16, 8 or 4 rows (FD_T32x16,
// FD_T32x8, FD_T32x4). Taller tiles spend fewer node-stages on the halo
// (per output node: 5.0 for 32 x 16, 6.5 for 32 x 8, 9.6 for 32 x 4) but
// need more shared memory.
static int fused_ty(int tile) {
    return tile == FD_T32x16 ? 16 : (tile == FD_T32x8 ? 8 : (tile == FD_T32x4 ? 4 : 0));
}

template <typename T, int Q1>
static const void* fused_ptr_q(int ty) {
    return ty == 16 ? (const void*)fd_fused_kernel<T, Q1, 16>
                    : (ty == 8 ? (const void*)fd_fused_kernel<T, Q1, 8>
                               : (ty == 4 ? (const void*)fd_fused_kernel<T, Q1, 4> : nullptr));
}
template <typename T>
static const void* fused_ptr(int q1, int ty) {
    return q1 == 3 ? fused_ptr_q<T, 3>(ty) : (q1 == 4 ? fused_ptr_q<T, 4>(ty) : (q1 == 5 ? fused_ptr_q<T, 5>(ty) : nullptr));
}
template <typename T, int Q1>
static size_t fused_bytes_q(int ty) {
    return ty == 16 ? FusedGeo<T, Q1, 16>::bytes
                    : (ty == 8 ? FusedGeo<T, Q1, 8>::bytes : (ty == 4 ? FusedGeo<T, Q1, 4>::bytes : 0));
}
template <typename T>
static size_t fused_bytes_t(int q1, int ty) {
    return q1 == 3 ? fused_bytes_q<T, 3>(ty) : (q1 == 4 ? fused_bytes_q<T, 4>(ty) : (q1 == 5 ? fused_bytes_q<T, 5>(ty) : 0));
}

int fd_fused_threads(int precision) { return precision == LBM_FP64 ? 256 : 512; }

// Opt a variant into the dynamic shared memory it needs; once per process.
// Variants that do not fit the device (or tile shapes without a fused
// kernel) are refused.
static cudaError_t fused_prepare(int precision, int tile, int q1) {
    // 0 unknown, 1 ready, 2 unavailable; atomic: the two lanes of a server
    // may prepare the same variant at once (both then make the same calls)
    static std::atomic<int> state[2][FD_NTILES][3] = {};
    if (tile < 0 || tile >= FD_NTILES || q1 < 3 || q1 > 5) return cudaErrorInvalidValue;
    const int p = precision == LBM_FP64 ? 0 : 1;
    std::atomic<int>& st = state[p][tile][q1 - 3];
    if (st == 1) return cudaSuccess;
    if (st == 2) return cudaErrorInvalidConfiguration;
    const int ty = fused_ty(tile);
    const void* fn = ty ? (precision == LBM_FP64 ? fused_ptr<double>(q1, ty) : fused_ptr<float>(q1, ty)) : nullptr;
    const size_t need = precision == LBM_FP64 ? fused_bytes_t<double>(q1, ty) : fused_bytes_t<float>(q1, ty);
    int dev = 0, optin = 0;
    if (!fn || cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
        cudaGetLastError();
        st = fn ? 0 : 2;
        return cudaErrorInvalidConfiguration;
    }
    if (need > (size_t)optin ||
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need) != cudaSuccess) {
        cudaGetLastError();
        st = 2;
        return cudaErrorInvalidConfiguration;
    }
    st = 1;
    return cudaSuccess;
}

bool fd_fused_fits(int precision, int q1, int tile) { return fused_prepare(precision, tile, q1) == cudaSuccess; }

int fd_fused_blocks_per_sm(int precision, int q1, int tile) {
    if (!fd_fused_fits(precision, q1, tile)) return 1;
    const int ty = fused_ty(tile);
    const void* fn = precision == LBM_FP64 ? fused_ptr<double>(q1, ty) : fused_ptr<float>(q1, ty);
    const size_t bytes = precision == LBM_FP64 ? fused_bytes_t<double>(q1, ty) : fused_bytes_t<float>(q1, ty);
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, fd_fused_threads(precision), bytes) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return n > 0 ? n : 1;
}

cudaError_t launch_fd_fused(int precision, int q1, int tile, int grid, const GroupDev& g, int j, cudaStream_t s) {
    if (grid <= 0) return cudaErrorInvalidValue;
    cudaError_t e = fused_prepare(precision, tile, q1);
    if (e != cudaSuccess) return e;
    const int ty = fused_ty(tile);
    const void* fn = precision == LBM_FP64 ? fused_ptr<double>(q1, ty) : fused_ptr<float>(q1, ty);
    const size_t bytes = precision == LBM_FP64 ? fused_bytes_t<double>(q1, ty) : fused_bytes_t<float>(q1, ty);
    GroupDev gg = g;
    int jj = j;
    void* args[] = {&gg, &jj};
    return cudaLaunchKernel(fn, dim3(grid), dim3(fd_fused_threads(precision)), args, bytes, s);
}

}  // namespace lbm
