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
//
// In-place storage (one buffer, the AA access pattern): steps alternate.
//   even step, state in node order (slot k at x holds f_k(x)): collide at x
//     and write f*_k to slot 8 - k (the opposite velocity, k = ix + 3 iy) at x;
//   odd step, state as the even step left it (f_k(x) is in slot 8 - k at
//     x - c_k): read there, collide, write f*_k to slot k at x + c_k, which
//     leaves the state in node order again.
// In both steps a node reads and writes the same nine locations and no other
// node touches them, so the update needs no second buffer and has no races.
// Which step a lattice takes is its phase bit (LatDesc::cur) flipped every
// step, so lattices of either storage and phase share a launch.
#include "kernels.h"
#include "ptx.cuh"

namespace lbm {

enum { CS_AB = 0, CS_AA_EVEN = 1, CS_AA_ODD = 2 };

__device__ __forceinline__ int cs_mode(const LatDesc& d, int j) {
    const int ph = d.cur ^ (j & 1);
    return d.inplace ? (ph ? CS_AA_ODD : CS_AA_EVEN) : CS_AB;
}

// In-place rows of the plain kernel (see above); buf is the one state buffer.
template <typename T, int RY, int MODE>
__device__ __forceinline__ void cs_plain_aa_rows(const LatDesc* dp, T* buf, int x, int by, T omega, T r0, bool obs,
                                                 int pc, T pxv, T (&acc)[NOBS]) {
    const int nx = dp->nx, ny = dp->ny, pitch = dp->pitch;
    const long long plane = dp->plane;
    const int xm = (x == 0) ? nx - 1 : x - 1;
    const int xp = (x + 1 >= nx) ? x + 1 - nx : x + 1;
#pragma unroll
    for (int r = 0; r < RY; ++r) {
        const int y = by * RY + r;
        if (y >= ny) break;
        const int ym = (y == 0) ? ny - 1 : y - 1;
        const int yp = (y + 1 >= ny) ? y + 1 - ny : y + 1;
        const long long rowm = (long long)ym * pitch, row0 = (long long)y * pitch, rowp = (long long)yp * pitch;
        T s[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const int cx = c3_of(k % 3), cy = c3_of(k / 3);
            long long off;
            if (MODE == CS_AA_EVEN) {
                off = k * plane + row0 + x;
            } else {
                const int sx = cx == 1 ? xm : (cx == -1 ? xp : x);
                const long long sr = cy == 1 ? rowm : (cy == -1 ? rowp : row0);
                off = (8 - k) * plane + sr + sx;
            }
            s[k] = LBM_BC_NODE(dp, 9, off) ? buf[off] : T(0);
        }
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
            const T v = s[k] - omega * (s[k] - geq);
            const int cx = c3_of(k % 3), cy = c3_of(k / 3);
            long long off;
            if (MODE == CS_AA_EVEN) {
                off = (8 - k) * plane + row0 + x;
            } else {
                const int dxx = cx == 1 ? xp : (cx == -1 ? xm : x);
                const long long drw = cy == 1 ? rowp : (cy == -1 ? rowm : row0);
                off = k * plane + drw + dxx;
            }
            if (LBM_BC_NODE(dp, 9, off)) buf[off] = v;
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

template <typename T, int TX, int RY>
__global__ void __launch_bounds__(TX) cs_step_kernel(GroupDev g, int j) {
    __shared__ double red[(TX / 32) * NOBS];
    const int n_lat = g.hdr[0];
    const int total = g.hdr[1];
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
        const int cur = dp->cur ^ (j & 1);   // A/B storage: the buffer holding the state
        const T* __restrict__ in = static_cast<const T*>(dp->buf[cur]);
        T* __restrict__ out = static_cast<T*>(dp->buf[cur ^ 1]);
        const T omega = lat_val<T>(dp->omega, dp->omega_f);
        const T r0 = lat_val<T>(dp->rho0, dp->rho0_f);
        const bool obs = observe_now(*dp, j);
        const int pc = dp->probe_comp;
        T acc[NOBS] = {T(0), T(0), T(0), T(0)};

        const int x = bx * TX + threadIdx.x;
        const int mode = cs_mode(*dp, j);
        if (mode != CS_AB) {
            if (x < nx) {
                T pxv = T(0);
                if (obs && pc >= 0) {
                    if constexpr (sizeof(T) == 4) pxv = dp->probe_pxf[x]; else pxv = (T)dp->probe_px[x];
                }
                T* buf = static_cast<T*>(dp->buf[0]);
                if (mode == CS_AA_EVEN)
                    cs_plain_aa_rows<T, RY, CS_AA_EVEN>(dp, buf, x, by, omega, r0, obs, pc, pxv, acc);
                else
                    cs_plain_aa_rows<T, RY, CS_AA_ODD>(dp, buf, x, by, omega, r0, obs, pc, pxv, acc);
            }
        } else if (x < nx) {
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
                    s[k] = LBM_BC_NODE(dp, 9, k * plane + sr + sx) ? in[k * plane + sr + sx] : T(0);
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
                    if (LBM_BC_NODE(dp, 9, k * plane + row0 + x)) out[k * plane + row0 + x] = s[k] - omega * (s[k] - geq);
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

// ---------------------------------------------------------------------------
// Warp-specialised variant. A work item is W columns x RB rows of one
// lattice. Warp 0 (one lane) streams, for every output row y, the nine
// population row segments it gathers from (rows y - c_ky) into a ring of S
// shared-memory slots with 1D bulk asynchronous copies; each slot's mbarrier
// counts the bytes in. Warps 1..W/32 take one node per thread from the slot,
// collide, store, and release the slot. A segment covers [x0 - 4, x0 + W + 4):
// 16-byte aligned, inside the allocation (4 elements of padding precede x = 0
// and every buffer has a tail pad), and it contains the x-1 / x+1 neighbours;
// only the periodic wrap at x = 0 / nx - 1 is read from global memory.
// All waits are bounded; a timeout sets hdr[2] and the block finishes
// without waiting again. hdr[3] > 0 is a test injection: every wait of the
// launch is limited to hdr[3] microseconds and block 0's producer skips the
// copies of its first row, so that row's consumers wait on a barrier nothing
// completes and run out of time (no fault, no unbounded wait).
template <typename T, int W, int RB, int S>
__host__ __device__ constexpr size_t cs_bulk_smem() {
    return (size_t)S * 9 * (W + 8) * sizeof(T) + 2 * S * sizeof(uint64_t) + (W / 32) * NOBS * sizeof(double);
}

// Producer: issue the row copies of one work item (rows y0 .. y1-1) into the
// ring. Slot row k holds what the consumers gather for population k: two
// buffers, plane k at row y - c_ky; in place, even step: plane k at row y;
// odd step: plane 8 - k at row y - c_ky. Returns false when a wait ran out.
template <typename T, int W, int S, int MODE>
__device__ __forceinline__ bool cs_bulk_issue(const LatDesc* dp, T* ring, uint64_t* full, uint64_t* empty, const T* in,
                                              long long plane, int pitch, int ny, int x0, int y0, int y1, unsigned& it,
                                              bool skip_first, unsigned long long lim) {
    constexpr int SEG = W + 8;
    constexpr unsigned SEG_BYTES = SEG * sizeof(T);
    constexpr unsigned SLOT_BYTES = 9 * SEG_BYTES;
    for (int y = y0; y < y1; ++y, ++it) {
        const int s = it % S;
        if (it >= (unsigned)S && !mbar_wait(&empty[s], ((it / S) - 1) & 1, lim)) return false;
        if (skip_first && it == 0) continue;   // injected: this slot is never filled
        const int ym = (y == 0) ? ny - 1 : y - 1;
        const int yp = (y + 1 >= ny) ? y + 1 - ny : y + 1;
#ifdef LBM_BOUNDS_CHECK
        bool spans_ok = true;
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const int cy = c3_of(k / 3);
            const int sy = MODE == CS_AA_EVEN ? y : (cy == 1 ? ym : (cy == -1 ? yp : y));
            const int sp = MODE == CS_AA_ODD ? 8 - k : k;
            spans_ok = spans_ok && LBM_BC_SPAN(dp, 9, sp * plane + (long long)sy * pitch + x0 - 4, SEG);
        }
        if (!spans_ok) {   // no copy: the slot completes empty (the step is reported invalid)
            mbar_arrive(&full[s]);
            continue;
        }
#endif
        mbar_arrive_expect_tx(&full[s], SLOT_BYTES);
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const int cy = c3_of(k / 3);
            const int sy = MODE == CS_AA_EVEN ? y : (cy == 1 ? ym : (cy == -1 ? yp : y));
            const int sp = MODE == CS_AA_ODD ? 8 - k : k;
            bulk_g2s(ring + ((size_t)s * 9 + k) * SEG, in + sp * plane + (long long)sy * pitch + x0 - 4, SEG_BYTES,
                     &full[s]);
        }
    }
    return true;
}

// Consumers: collide the rows of one work item from the ring and store (two
// buffers: to the other buffer at x; in place, even: to slot 8 - k at x; odd:
// to slot k at x + c_k). `in` and `out` are the same buffer in place: every
// node reads its nine locations (from shared memory, or for the periodic x
// wrap from global memory) before it writes them.
template <typename T, int W, int S, int MODE>
__device__ __forceinline__ void cs_bulk_consume(const T* ring, uint64_t* full, uint64_t* empty, const T* in_, T* out_,
                                                const LatDesc* dp, int x0, int y0, int y1, T omega, T r0, bool obs,
                                                T pxv, unsigned& it, bool& dead, int* err, unsigned long long lim,
                                                T (&acc)[NOBS]) {
    constexpr int SEG = W + 8;
    const T* __restrict__ in = in_;
    T* __restrict__ out = out_;
    const int ctid = threadIdx.x - 32, lane = threadIdx.x & 31;
    const int nx = dp->nx, ny = dp->ny, pitch = dp->pitch;
    const long long plane = dp->plane;
    const int pc = dp->probe_comp;
    const int x = x0 + ctid;
    const bool xin = x < nx;
    for (int y = y0; y < y1; ++y, ++it) {
        const int s = it % S;
        if (!dead && !mbar_wait(&full[s], (it / S) & 1, lim)) {
            dead = true;
            atomicOr(err, ERR_WAIT_TIMEOUT);
        }
        if (!dead && xin) {
            const T* slot = ring + (size_t)s * 9 * SEG;
            const int ym = (y == 0) ? ny - 1 : y - 1;
            const int yp = (y + 1 >= ny) ? y + 1 - ny : y + 1;
            T f[9];
#pragma unroll
            for (int k = 0; k < 9; ++k) {
                const int cx = c3_of(k % 3), cy = c3_of(k / 3);
                if (MODE == CS_AA_EVEN) {
                    f[k] = slot[k * SEG + ctid + 4];
                } else {
                    f[k] = slot[k * SEG + ctid + 4 - cx];
                    if ((cx == 1 && x == 0) || (cx == -1 && x == nx - 1)) {
                        const int sy = cy == 1 ? ym : (cy == -1 ? yp : y);
                        const int sp = MODE == CS_AA_ODD ? 8 - k : k;
                        const long long off = sp * plane + (long long)sy * pitch + (cx == 1 ? nx - 1 : 0);
                        f[k] = LBM_BC_NODE(dp, 9, off) ? in[off] : T(0);
                    }
                }
            }
            T dr = T(0), jx = T(0), jy = T(0);
#pragma unroll
            for (int k = 0; k < 9; ++k) {
                dr += f[k];
                if (vx_of<3>(k) != 0.0) jx += f[k] * (T)vx_of<3>(k);
                if (vy_of<3>(k) != 0.0) jy += f[k] * (T)vy_of<3>(k);
            }
            const T rho = r0 + dr;
            const T inv = T(1) / rho;
            const T ux = jx * inv, uy = jy * inv;
            const T usq = ux * ux + uy * uy;
            const long long row0 = (long long)y * pitch + x;
#pragma unroll
            for (int k = 0; k < 9; ++k) {
                const T xi = (T)vx_of<3>(k) * ux + (T)vy_of<3>(k) * uy;
                const T geq = (T)w_of<3>(k) * (dr + rho * (xi + T(0.5) * (xi * xi - usq)));
                const T v = f[k] - omega * (f[k] - geq);
                long long off;
                if (MODE == CS_AB) {
                    off = k * plane + row0;
                } else if (MODE == CS_AA_EVEN) {
                    off = (8 - k) * plane + row0;
                } else {
                    const int cx = c3_of(k % 3), cy = c3_of(k / 3);
                    const int dxx = cx == 1 ? (x + 1 >= nx ? 0 : x + 1) : (cx == -1 ? (x == 0 ? nx - 1 : x - 1) : x);
                    const int dyy = cy == 1 ? yp : (cy == -1 ? ym : y);
                    off = k * plane + (long long)dyy * pitch + dxx;
                }
                if (LBM_BC_NODE(dp, 9, off)) __stcs(out + off, v);
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
        __syncwarp();
        if (lane == 0 && !dead) mbar_arrive(&empty[s]);
    }
}

// Resident blocks per SM the register allocation is bounded for: the
// blocks the shared-memory ring allows (FP32: 4 of 38 KiB at W = 256, 6 at
// W = 128; FP64: 2 and 3), so that the bytes in flight, not registers, set
// the occupancy (about 56 registers per thread for FP32).
template <typename T, int W>
constexpr int cs_bulk_min_blocks() { return sizeof(T) == 4 ? (W == 256 ? 4 : 6) : (W == 256 ? 2 : 3); }

template <typename T, int W, int RB, int S>
__global__ void __launch_bounds__(32 + W, cs_bulk_min_blocks<T, W>()) cs_bulk_kernel(GroupDev g, int j) {
    constexpr int NCW = W / 32;
    constexpr int SEG = W + 8;
    constexpr unsigned SEG_BYTES = SEG * sizeof(T);
    constexpr unsigned SLOT_BYTES = 9 * SEG_BYTES;
    extern __shared__ __align__(128) unsigned char sm[];
    T* ring = reinterpret_cast<T*>(sm);
    uint64_t* full = reinterpret_cast<uint64_t*>(sm + (size_t)S * SLOT_BYTES);
    uint64_t* empty = full + S;
    double* red = reinterpret_cast<double*>(empty + S);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], NCW);
        }
        fence_mbar_init();
    }
    __syncthreads();
    const int n_lat = g.hdr[0];
    const int total = g.hdr[1];
    const int inject_us = g.hdr[3];
    const unsigned long long lim = inject_us > 0 ? 1000ull * (unsigned long long)inject_us : WAIT_NS;

    if (warp == 0) {
        // ---------------- producer
        if (lane != 0) return;
        unsigned it = 0;
        bool ok = true;
        const bool skip_first = inject_us > 0 && blockIdx.x == 0;
        for (int item = blockIdx.x; item < total && ok; item += gridDim.x) {
            const int li = find_lattice(g.item_begin, n_lat, item);
            const LatDesc* dp = g.desc + li;
            if ((long long)j >= dp->remaining) {
                item = last_item_of(*dp, item);
                continue;
            }
            const int ny = dp->ny, pitch = dp->pitch;
            const long long plane = dp->plane;
            const int local = item - dp->item_begin;
            const int bx = local % dp->tiles_x, by = local / dp->tiles_x;
            const int x0 = bx * W, y0 = by * RB;
            const int y1 = min(y0 + RB, ny);
            const int mode = cs_mode(*dp, j);
            const T* in = static_cast<const T*>(dp->buf[mode == CS_AB ? dp->cur ^ (j & 1) : 0]);
            if (mode == CS_AB)
                ok = cs_bulk_issue<T, W, S, CS_AB>(dp, ring, full, empty, in, plane, pitch, ny, x0, y0, y1, it, skip_first, lim);
            else if (mode == CS_AA_EVEN)
                ok = cs_bulk_issue<T, W, S, CS_AA_EVEN>(dp, ring, full, empty, in, plane, pitch, ny, x0, y0, y1, it,
                                                        skip_first, lim);
            else
                ok = cs_bulk_issue<T, W, S, CS_AA_ODD>(dp, ring, full, empty, in, plane, pitch, ny, x0, y0, y1, it,
                                                       skip_first, lim);
        }
        if (!ok) atomicOr(g.hdr + 2, ERR_WAIT_TIMEOUT);
        // every copy issued lands before the block exits, also when the
        // consumers stopped waiting after a timeout (bounded waits)
        const unsigned first = it > (unsigned)S ? it - S : 0;
        for (unsigned q = first; q < it; ++q)
            if (!(skip_first && q == 0)) mbar_wait(&full[q % S], (q / S) & 1, lim);
        return;
    }

    // ---------------- consumers: one node per thread per row
    const int ctid = threadIdx.x - 32;
    unsigned it = 0;
    bool dead = false;
    for (int item = blockIdx.x; item < total; item += gridDim.x) {
        const int li = find_lattice(g.item_begin, n_lat, item);
        const LatDesc* dp = g.desc + li;
        if ((long long)j >= dp->remaining) {
            item = last_item_of(*dp, item);
            continue;
        }
        const int nx = dp->nx, ny = dp->ny;
        const int local = item - dp->item_begin;
        const int bx = local % dp->tiles_x, by = local / dp->tiles_x;
        const int x0 = bx * W, y0 = by * RB;
        const int y1 = min(y0 + RB, ny);
        const int mode = cs_mode(*dp, j);
        const int cur = dp->cur ^ (j & 1);
        const T* in = static_cast<const T*>(dp->buf[mode == CS_AB ? cur : 0]);
        T* out = static_cast<T*>(dp->buf[mode == CS_AB ? cur ^ 1 : 0]);
        const T omega = lat_val<T>(dp->omega, dp->omega_f);
        const T r0 = lat_val<T>(dp->rho0, dp->rho0_f);
        const bool obs = observe_now(*dp, j);
        const int pc = dp->probe_comp;
        const int x = x0 + ctid;
        T acc[NOBS] = {T(0), T(0), T(0), T(0)};
        T pxv = T(0);
        if (obs && pc >= 0 && x < nx) {
            if constexpr (sizeof(T) == 4) pxv = dp->probe_pxf[x]; else pxv = (T)dp->probe_px[x];
        }
        if (mode == CS_AB)
            cs_bulk_consume<T, W, S, CS_AB>(ring, full, empty, in, out, dp, x0, y0, y1, omega, r0, obs, pxv, it, dead,
                                            g.hdr + 2, lim, acc);
        else if (mode == CS_AA_EVEN)
            cs_bulk_consume<T, W, S, CS_AA_EVEN>(ring, full, empty, in, out, dp, x0, y0, y1, omega, r0, obs, pxv, it,
                                                 dead, g.hdr + 2, lim, acc);
        else
            cs_bulk_consume<T, W, S, CS_AA_ODD>(ring, full, empty, in, out, dp, x0, y0, y1, omega, r0, obs, pxv, it,
                                                dead, g.hdr + 2, lim, acc);
        if (obs) {
            T r[NOBS];
#pragma unroll
            for (int q = 0; q < NOBS; ++q) {
                T v = acc[q];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                r[q] = v;
            }
            if (lane == 0)
#pragma unroll
                for (int q = 0; q < NOBS; ++q) red[(warp - 1) * NOBS + q] = (double)r[q];
            named_sync(1, W);
            if (ctid < NOBS) {
                double t = 0.0;
                for (int w = 0; w < NCW; ++w) t += red[w * NOBS + ctid];
                dp->partials[(long long)local * NOBS + ctid] = t;
            }
            named_sync(1, W);
        }
    }
}

int cs_tile_tx(int v) {
    switch (v) {
        case CS_T128x1: case CS_T128x2: case CS_B128x32: return 128;
        case CS_T256x1: case CS_T256x2: case CS_B256x32: return 256;
        case CS_T64x4: return 64;
    }
    return 0;
}
int cs_tile_ty(int v) {
    switch (v) {
        case CS_T128x1: case CS_T256x1: return 1;
        case CS_T128x2: case CS_T256x2: return 2;
        case CS_T64x4: return 4;
        case CS_B256x32: case CS_B128x32: return 32;
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
        case CS_B256x32: return (const void*)cs_bulk_kernel<T, 256, 32, 4>;
        case CS_B128x32: return (const void*)cs_bulk_kernel<T, 128, 32, 6>;
    }
    return nullptr;
}

template <typename T>
static size_t cs_smem(int tile) {
    switch (tile) {
        case CS_B256x32: return cs_bulk_smem<T, 256, 32, 4>();
        case CS_B128x32: return cs_bulk_smem<T, 128, 32, 6>();
    }
    return 0;
}

static bool cs_is_bulk(int tile) { return tile == CS_B256x32 || tile == CS_B128x32; }

static const void* cs_fn(int precision, int tile) {
    return precision == LBM_FP64 ? cs_kernel_ptr<double>(tile) : cs_kernel_ptr<float>(tile);
}
static size_t cs_bytes(int precision, int tile) {
    return precision == LBM_FP64 ? cs_smem<double>(tile) : cs_smem<float>(tile);
}
static int cs_threads(int tile) { return cs_is_bulk(tile) ? 32 + cs_tile_tx(tile) : cs_tile_tx(tile); }

static cudaError_t cs_prepare(int precision, int tile) {
    static bool done[2][CS_NTILES] = {};
    const int p = precision == LBM_FP64 ? 0 : 1;
    if (done[p][tile]) return cudaSuccess;
    cudaError_t e = cudaSuccess;
    if (cs_bytes(precision, tile) > 0)
        e = cudaFuncSetAttribute(cs_fn(precision, tile), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)cs_bytes(precision, tile));
    if (e == cudaSuccess) done[p][tile] = true;
    return e;
}

cudaError_t launch_cs_step(int precision, int tile, int grid, const GroupDev& g, int j, cudaStream_t s) {
    if (tile < 0 || tile >= CS_NTILES || grid <= 0) return cudaErrorInvalidValue;
    const void* fn = cs_fn(precision, tile);
    cudaError_t e = cs_prepare(precision, tile);
    if (e != cudaSuccess) return e;
    GroupDev gg = g;
    int jj = j;
    void* args[] = {&gg, &jj};
    return cudaLaunchKernel(fn, dim3(grid), dim3(cs_threads(tile)), args, cs_bytes(precision, tile), s);
}

int cs_blocks_per_sm(int precision, int tile) {
    if (tile < 0 || tile >= CS_NTILES || cs_prepare(precision, tile) != cudaSuccess) return 1;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, cs_fn(precision, tile), cs_threads(tile),
                                                      cs_bytes(precision, tile)) != cudaSuccess)
        return 1;
    return n > 0 ? n : 1;
}

}  // namespace lbm
