// Host engine: memory layout, validation, descriptors, step scheduling.
//
// Layout in HBM: each lattice owns one allocation holding its 2 (CS) or 3
// (FD) state buffers; a buffer is K population planes [ny][pitch], x fastest,
// pitch = nx + 8 rounded up to 32 elements (128-byte rows for FP32), plane
// stride = pitch * ny. Element (0, 0) of a buffer sits HEAD = 4 elements into
// its slot and each slot ends with TAIL = 1024 spare elements, so a row
// segment [x0 - 4, x0 + W + 4) read by the bulk-copy kernels (W <= 256) is
// always 16-byte aligned and inside the allocation. Tile partials,
// descriptors and probe tables are small side allocations.
#include "engine.h"

#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <limits>

namespace lbm {

static thread_local char g_last_error[512];

void set_error(const char* msg) {
    size_t i = 0;
    for (; msg && msg[i] && i + 1 < sizeof g_last_error; ++i) g_last_error[i] = msg[i];
    g_last_error[i] = 0;
}
const char* last_error_cstr() { return g_last_error; }

int cuda_fail(cudaError_t e, const char* what) {
    char buf[256];
    snprintf(buf, sizeof buf, "%s: %s (%d)", what, cudaGetErrorString(e), (int)e);
    set_error(buf);
    return e == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA;
}

#define CK(call)                                              \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);   \
    } while (0)

static const double SQRT3 = 1.73205080756887729353;

// NVTX range for the lifetime of the object (tools such as Nsight Compute
// filter launches by range; without a tool attached the calls do nothing).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};
static_assert(Lattice::HEAD == STATE_HEAD && Lattice::TAIL == STATE_TAIL, "state buffer layout");

static double vmax_of(int q1) {
    switch (q1) {
        case 3: return GH<3>::vmax();
        case 4: return GH<4>::vmax();
        case 5: return GH<5>::vmax();
    }
    return NAN;
}

int Engine::validate(const lbm_spec* in, lbm_spec* out) {
    if (!in || !out) { set_error("null spec"); return LBM_EINVAL; }
    lbm_spec s = *in;
    if (s.model != LBM_CS && s.model != LBM_FD) { set_error("model must be LBM_CS or LBM_FD"); return LBM_EINVAL; }
    if (s.model == LBM_CS && s.q_per_axis != 3) { set_error("CS uses the D2Q9 set: q_per_axis = 3"); return LBM_EINVAL; }
    if (s.model == LBM_FD && (s.q_per_axis < 3 || s.q_per_axis > 5)) {
        set_error("FD q_per_axis must be 3, 4 or 5");
        return LBM_EINVAL;
    }
    if (s.precision != LBM_FP64 && s.precision != LBM_FP32_DEV) { set_error("bad precision"); return LBM_EINVAL; }
    if (s.nx < 1 || s.ny < 1 || s.nx > (1 << 24) || s.ny > (1 << 24)) { set_error("nx, ny must be in [1, 2^24]"); return LBM_EINVAL; }
    const int K = s.q_per_axis * s.q_per_axis;
    if ((double)s.nx * s.ny * K >= 1099511627776.0) { set_error("lattice too large"); return LBM_EINVAL; }
    if (!std::isfinite(s.tau) || s.tau <= 0) { set_error("tau must be positive and finite"); return LBM_EINVAL; }
    if (s.rho0 == 0) s.rho0 = 1.0;
    if (!std::isfinite(s.rho0) || s.rho0 <= 0) { set_error("rho0 must be positive"); return LBM_EINVAL; }
    if (s.model == LBM_CS) {
        if (s.dx == 0 && s.dt == 0) { s.dx = 1.0; s.dt = 1.0 / SQRT3; }
        else if (s.dx == 0) s.dx = s.dt * SQRT3;
        else if (s.dt == 0) s.dt = s.dx / SQRT3;
        if (!(s.dx > 0) || !(s.dt > 0) || std::fabs(s.dx / s.dt / SQRT3 - 1.0) > 1e-12) {
            set_error("CS requires dx/dt = sqrt(3) (on-lattice D2Q9, Sec. 2)");
            return LBM_EINVAL;
        }
        if (!(s.tau > 0.5 * s.dt)) { set_error("CS requires tau_LU > dt/2 (nu_LU > 0, Eq. nulu)"); return LBM_EINVAL; }
    } else {
        if (s.dx == 0) s.dx = 1.0 / s.nx;
        if (!(s.dx > 0) || !std::isfinite(s.dx) || !(s.dt > 0) || !std::isfinite(s.dt)) {
            set_error("FD requires dt > 0 and dx > 0");
            return LBM_EINVAL;
        }
        const double cfl = vmax_of(s.q_per_axis) * s.dt / s.dx;
        if (cfl > 1.0 + 1e-12) {
            char b[160];
            snprintf(b, sizeof b, "CFL = max|v| dt/dx = %.6g > 1 (Sec. 4.1)", cfl);
            set_error(b);
            return LBM_ECFL;
        }
        if (s.scheme != LBM_TS_RK3 && s.scheme != LBM_TS_IMEX && s.scheme != LBM_TS_RK3_FUSED) {
            set_error("bad FD scheme");
            return LBM_EINVAL;
        }
        if (s.scheme != LBM_TS_IMEX && s.dt > s.tau * (1.0 + 1e-12)) {
            set_error("FD requires dt <= tau with the RK3 scheme (non-stiff BGK term, Sec. 4.1); "
                      "LBM_TS_IMEX lifts it");
            return LBM_ESTIFF;
        }
    }
    if (s.model == LBM_CS && s.scheme != LBM_TS_RK3) { set_error("the scheme field is for FD lattices"); return LBM_EINVAL; }
    if (s.reserved != 0) { set_error("lbm_spec.reserved must be 0"); return LBM_EINVAL; }
    if (s.storage != LBM_STORE_AB && s.storage != LBM_STORE_INPLACE) { set_error("bad storage"); return LBM_EINVAL; }
    if (s.storage == LBM_STORE_INPLACE && s.model != LBM_CS) {
        set_error("in-place storage is for CS lattices (FD needs its three stage buffers)");
        return LBM_EINVAL;
    }
    *out = s;
    return LBM_OK;
}

Engine::~Engine() {
    if (stream_) cudaStreamSynchronize(stream_);
    invalidate_graph();
    for (auto& L : lat) free_lattice(L);
    for (auto& g : groups) {
        cudaFree(g.d_desc);
        cudaFree(g.d_item_begin);
        cudaFree(g.d_hdr);
        cudaFree(g.d_partials);
        cudaFree(g.d_chunks);
    }
    if (own_stream_ && stream_) cudaStreamDestroy(stream_);
}

void Engine::invalidate_graph() {
    if (graph_) cudaGraphExecDestroy(graph_);
    graph_ = nullptr;
    graph_chunk_ = 0;
}

// Default grid of a group: one block per work item (tile) when the lattices
// are fixed (the hardware scheduler balances the tiles; the tuner picked this
// for every workload measured, e.g. CS D2Q9 8192^2 in place 90 GLUPS against
// 72 with one block set per SM), one block set per SM for a server's engine,
// whose lattices change under a captured graph (the blocks then loop over
// the items), or grid_mult_ block sets, so that each block covers fewer items
// and retires sooner (SMs then free up for another stream's kernels).
int Engine::persistent_grid(const Group& g, int tile) const {
    int bps = g.model == LBM_CS ? cs_blocks_per_sm(g.precision, tile)
                                : fd_blocks_per_sm(g.precision, g.q1, tile, g.scheme);
    return (int)std::max<long long>(1, (long long)sm_count_ * bps);
}

int Engine::default_grid(const Group& g, int tile) const {
    if (!dynamic_ && g.total_items > 0) return g.total_items;
    return persistent_grid(g, tile) * std::max(1, grid_mult_);
}

int Engine::open(void* stream) {
    int dev = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sm_count_, cudaDevAttrMultiProcessorCount, dev));
    if (stream) {
        stream_ = static_cast<cudaStream_t>(stream);
    } else {
        CK(cudaStreamCreateWithFlags(&stream_, cudaStreamNonBlocking));
        own_stream_ = true;
    }
    return LBM_OK;
}

void Engine::free_lattice(Lattice& L) {
    cudaFree(L.mem);
    cudaFree(L.d_px);
    cudaFree(L.d_py);
    cudaFree(L.d_pxf);
    cudaFree(L.d_pyf);
    cudaFree(L.d_series);
    cudaFree(L.d_io);
    cudaFree(L.d_part);
    cudaFree(L.d_snap);
    L.mem = L.d_io = nullptr;
    L.d_px = L.d_py = L.d_part = L.d_snap = nullptr;
    L.d_pxf = L.d_pyf = nullptr;
    L.d_series = nullptr;
    for (auto& b : L.buf) b = nullptr;
    L.io_bytes = 0;
}

size_t Engine::footprint(const lbm_spec& s) {
    const int K = s.q_per_axis * s.q_per_axis;
    const long long pitch = (s.nx + 8 + 31) / 32 * 32;
    const long long plane = pitch * s.ny;
    const int nbuf = state_buffers(s);
    const int elem = s.precision == LBM_FP64 ? 8 : 4;
    return (size_t)nbuf * (K * plane + Lattice::TAIL) * elem + sizeof(double) * NOBS * 1024;
}

int Engine::add_lattice(const lbm_spec* spec, int* index, bool upload) {
    Lattice L;
    const int rc = validate(spec, &L.spec);
    if (rc != LBM_OK) return rc;
    const lbm_spec& s = L.spec;
    L.K = s.q_per_axis * s.q_per_axis;
    L.elem = s.precision == LBM_FP64 ? 8 : 4;
    L.pitch = (s.nx + 8 + 31) / 32 * 32;
    L.plane = (long long)L.pitch * s.ny;
    L.nbuf = state_buffers(s);
    L.rho0s = s.precision == LBM_FP64 ? 0.0 : s.rho0;
    if (s.model == LBM_CS) {
        L.omega = s.dt / s.tau;
    } else {
        L.cdx = s.dt / s.dx;
        L.dt_tau = s.dt / s.tau;
    }
    const size_t bytes = L.state_bytes();
    cudaError_t e = cudaMalloc(&L.mem, bytes);
    if (e != cudaSuccess) {
        L.mem = nullptr;
        return cuda_fail(e, "cudaMalloc(state)");
    }
    // poison: every byte 0xFF, a NaN in float and double, so row padding and
    // slack never read into a result without showing up as non-finite
    e = cudaMemsetAsync(L.mem, 0xFF, bytes, stream_);
    if (e == cudaSuccess) e = cudaMalloc(&L.d_part, sizeof(double) * NOBS * 1024);
    if (e == cudaSuccess) e = cudaMalloc(&L.d_snap, sizeof(double) * NOBS);
    if (e != cudaSuccess) {
        free_lattice(L);
        return cuda_fail(e, "lattice allocation");
    }
    L.part_blocks = 1024;
    for (int b = 0; b < L.nbuf; ++b)
        L.buf[b] = static_cast<char*>(L.mem) + (b * L.buf_stride() + Lattice::HEAD) * L.elem;
    // group membership: one group per (model, velocity set, storage)
    int gi = -1;
    for (size_t g = 0; g < groups.size(); ++g)
        if (groups[g].model == s.model && groups[g].q1 == s.q_per_axis && groups[g].precision == s.precision &&
            groups[g].scheme == s.scheme)
            gi = (int)g;
    if (gi < 0) {
        Group g;
        g.model = s.model;
        g.q1 = s.q_per_axis;
        g.precision = s.precision;
        g.scheme = s.scheme;
        g.tile = s.model == LBM_CS ? (int)CS_B256x32 : (int)FD_T32x8;
        // the fused FD kernel's largest tiles do not fit every set and precision
        if (s.model == LBM_FD && s.scheme == LBM_TS_RK3_FUSED && !fd_variant_fits(s.precision, s.q_per_axis, g.tile, s.scheme))
            g.tile = FD_T32x4;
        groups.push_back(g);
        gi = (int)groups.size() - 1;
        invalidate_graph();
    }
    L.group = gi;
    const int idx = (int)lat.size();
    lat.push_back(L);
    groups[gi].members.push_back(idx);
    if (index) *index = idx;
    return upload ? upload_group(gi) : LBM_OK;
}

int Engine::remove_lattice(int i) {
    if (!valid(i) || !lat[i].alive) { set_error("no such lattice"); return LBM_EINVAL; }
    CK(cudaStreamSynchronize(stream_));
    Lattice& L = lat[i];
    Group& g = groups[L.group];
    g.members.erase(std::remove(g.members.begin(), g.members.end(), i), g.members.end());
    free_lattice(L);
    L.alive = false;
    L.active = false;
    return upload_group(L.group);
}

int Engine::create(const lbm_spec* specs, int n, void* stream) {
    if (n < 1 || !specs) { set_error("need at least one lattice"); return LBM_EINVAL; }
    for (int i = 0; i < n; ++i) {  // all parameters are checked before any CUDA call
        lbm_spec tmp;
        const int rc = validate(&specs[i], &tmp);
        if (rc != LBM_OK) {
            char b[64];
            snprintf(b, sizeof b, " (lattice %d)", i);
            set_error(std::string(lbm_last_error()) + b);
            return rc;
        }
    }
    int rc = open(stream);
    if (rc) return rc;
    lat.reserve(n);
    for (int i = 0; i < n; ++i) {
        rc = add_lattice(&specs[i], nullptr, false);
        if (rc) return rc;
    }
    return upload_all();
}

LatDesc Engine::make_desc(const Lattice& L, const Group& g, int item_begin, double* partials) const {
    LatDesc d;
    memset(&d, 0, sizeof d);
    for (int b = 0; b < 3; ++b) d.buf[b] = L.buf[b];
    d.nx = L.spec.nx;
    d.ny = L.spec.ny;
    d.pitch = L.pitch;
    const int tx = g.model == LBM_CS ? cs_tile_tx(g.tile) : fd_tile_tx(g.tile);
    const int ty = g.model == LBM_CS ? cs_tile_ty(g.tile) : fd_tile_ty(g.tile);
    d.tiles_x = (L.spec.nx + tx - 1) / tx;
    const int tiles_y = (L.spec.ny + ty - 1) / ty;
    d.plane = L.plane;
    d.item_begin = item_begin;
    d.items = d.tiles_x * tiles_y;
    d.cur = L.cur;
    d.inplace = L.inplace() ? 1 : 0;
    d.obs_every = (int)L.obs_every;
    d.obs_base = L.obs_base;
    d.step0 = L.step0;
    d.remaining = L.active ? L.remaining : 0;
    d.omega = L.omega;
    d.cdx = L.cdx;
    d.dt_tau = L.dt_tau;
    d.rho0 = L.rho0s;
    d.eps = L.eps;
    d.omega_f = (float)L.omega;
    d.cdx_f = (float)L.cdx;
    d.dt_tau_f = (float)L.dt_tau;
    d.rho0_f = (float)L.rho0s;
    d.eps_f = (float)L.eps;
    d.err = g.d_hdr + 2;
    d.dt = L.spec.dt;
    d.probe_comp = L.probe_comp;
    d.obs_cap = (int)std::min<long long>(L.obs_cap, std::numeric_limits<int>::max());
    d.probe_norm = L.probe_norm;
    d.probe_px = L.d_px;
    d.probe_py = L.d_py;
    d.probe_pxf = L.d_pxf;
    d.probe_pyf = L.d_pyf;
    d.partials = partials;
    d.series = L.d_series;
    d.snap = L.d_snap;
    return d;
}

int Engine::upload_group(int gi) {
    Group& g = groups[gi];
    const int tx = g.model == LBM_CS ? cs_tile_tx(g.tile) : fd_tile_tx(g.tile);
    const int ty = g.model == LBM_CS ? cs_tile_ty(g.tile) : fd_tile_ty(g.tile);
    std::vector<int> begins;
    long long items = 0;
    const bool had_obs = g.any_obs;
    g.any_obs = false;
    for (int li : g.members) {
        const Lattice& L = lat[li];
        begins.push_back((int)items);
        items += (long long)((L.spec.nx + tx - 1) / tx) * ((L.spec.ny + ty - 1) / ty);
        if (L.obs_every > 0) g.any_obs = true;
    }
    if (items >= (1LL << 31)) { set_error("too many work items"); return LBM_EINVAL; }
    if (g.any_obs != had_obs) invalidate_graph();
    const int nm = (int)g.members.size();
    if (nm > g.cap_lat) {
        cudaFree(g.d_desc);
        cudaFree(g.d_item_begin);
        cudaFree(g.d_hdr);
        g.d_desc = nullptr;
        g.d_item_begin = nullptr;
        g.d_hdr = nullptr;
        const int cap = std::max(std::max(nm, 1), dynamic_ ? 2 * g.cap_lat : 0);  // grow geometrically
        CK(cudaMalloc(&g.d_desc, sizeof(LatDesc) * cap));
        CK(cudaMalloc(&g.d_item_begin, sizeof(int) * cap));
        CK(cudaMalloc(&g.d_hdr, sizeof(int) * 4));
        g.cap_lat = cap;
        invalidate_graph();
    }
    if (items > g.cap_items) {
        cudaFree(g.d_partials);
        g.d_partials = nullptr;
        const long long cap = std::max(std::max<long long>(items, 1), dynamic_ ? 2 * g.cap_items : 0);
        CK(cudaMalloc(&g.d_partials, sizeof(double) * NOBS * cap));
        g.cap_items = cap;
        invalidate_graph();
    }
    g.total_items = (int)items;
    long long max_items = 1;
    for (int li : g.members) {
        const Lattice& L = lat[li];
        max_items = std::max<long long>(max_items, (long long)((L.spec.nx + tx - 1) / tx) * ((L.spec.ny + ty - 1) / ty));
    }
    // chunks of the observables reduction; fixed for dynamic engines so that
    // membership changes do not change the captured launches
    const int nch = dynamic_ ? 128 : (int)std::min<long long>(128, std::max<long long>(1, (max_items + 2047) / 2048));
    if (nch != g.nchunks || (long long)g.cap_lat * nch > g.chunk_cap || !g.d_chunks) {
        cudaFree(g.d_chunks);
        g.d_chunks = nullptr;
        g.nchunks = nch;
        g.chunk_cap = g.cap_lat * nch;
        CK(cudaMalloc(&g.d_chunks, sizeof(double) * NOBS * g.chunk_cap));
        invalidate_graph();
    }
    std::vector<LatDesc> descs;
    for (int m = 0; m < nm; ++m) {
        lat[g.members[m]].slot = m;
        descs.push_back(make_desc(lat[g.members[m]], g, begins[m], g.d_partials + (long long)begins[m] * NOBS));
    }
    const int hdr[4] = {nm, (int)items, 0, inject_us_};
    if (nm) {
        CK(cudaMemcpyAsync(g.d_desc, descs.data(), sizeof(LatDesc) * nm, cudaMemcpyHostToDevice, stream_));
        CK(cudaMemcpyAsync(g.d_item_begin, begins.data(), sizeof(int) * nm, cudaMemcpyHostToDevice, stream_));
    }
    CK(cudaMemcpyAsync(g.d_hdr, hdr, sizeof hdr, cudaMemcpyHostToDevice, stream_));
    CK(cudaStreamSynchronize(stream_));
    if (g.grid <= 0) g.grid = default_grid(g, g.tile);
    return LBM_OK;
}

int Engine::upload_all() {
    for (int g = 0; g < (int)groups.size(); ++g) {
        int rc = upload_group(g);
        if (rc) return rc;
    }
    invalidate_graph();
    return LBM_OK;
}

int Engine::set_group_config(int gi, int tile, int grid) {
    if (gi < 0 || gi >= (int)groups.size()) { set_error("no such group"); return LBM_EINVAL; }
    Group& g = groups[gi];
    if (tile < 0 || tile >= (g.model == LBM_CS ? (int)CS_NTILES : (int)FD_NTILES) || grid < 0) {
        set_error("no such tile variant");
        return LBM_EINVAL;
    }
    if (g.model == LBM_FD && !fd_variant_fits(g.precision, g.q1, tile, g.scheme)) {
        set_error("this FD tile variant needs more shared memory than the device offers for this set/precision");
        return LBM_EINVAL;
    }
    CK(cudaStreamSynchronize(stream_));
    g.tile = tile;
    g.grid = 0;
    int rc = upload_group(gi);
    if (rc) return rc;
    g.grid = grid > 0 ? grid : default_grid(g, tile);
    invalidate_graph();
    return LBM_OK;
}

int Engine::enqueue_chunk(int c) {
    long long n = 0;
    for (int j = 0; j < c; ++j) {
        for (auto& g : groups) {
            if (g.cap_lat == 0) continue;  // empty groups launch too: kernels read the live count
            const GroupDev gd = g.dev();
            cudaError_t e;
            if (g.model == LBM_CS) {
                e = launch_cs_step(g.precision, g.tile, g.grid, gd, j, stream_);
                if (e != cudaSuccess) return cuda_fail(e, "launch_cs_step");
                ++n;
                if (g.any_obs) {
                    if ((e = launch_obs_finalize(gd, g.cap_lat, g.nchunks, g.d_chunks, j, stream_)) != cudaSuccess)
                        return cuda_fail(e, "launch_obs_finalize");
                    n += 2;
                }
            } else {
                for (int st = 1; st <= fd_stages(g.scheme); ++st) {
                    e = launch_fd_stage(g.precision, g.q1, g.scheme, g.tile, g.grid, gd, j, st, stream_);
                    if (e != cudaSuccess) return cuda_fail(e, "launch_fd_stage");
                    ++n;
                    if (st == 1 && g.any_obs) {
                        if ((e = launch_obs_finalize(gd, g.cap_lat, g.nchunks, g.d_chunks, j, stream_)) != cudaSuccess)
                            return cuda_fail(e, "launch_obs_finalize");
                        n += 2;
                    }
                }
            }
        }
    }
    for (auto& g : groups) {
        if (g.cap_lat == 0) continue;  // empty groups launch too: kernels read the live count
        cudaError_t e = launch_advance(g.dev(), g.cap_lat, c, g.flips() ? 1 : 0, stream_);
        if (e != cudaSuccess) return cuda_fail(e, "launch_advance");
        ++n;
    }
    last_chunk_launches_ = n;
    return LBM_OK;
}

void Engine::mirror_advance(int c) {
    for (auto& L : lat) {
        if (!L.alive || !L.active) continue;
        const long long adv = std::min<long long>(L.remaining, c);
        L.step0 += adv;
        L.remaining -= adv;
        if (L.flips() && (adv & 1)) L.cur ^= 1;
    }
}

int Engine::step(long long n) {
    if (n < 0) { set_error("negative step count"); return LBM_EINVAL; }
    NvtxRange range("lbm.step");
    while (n > 0) {
        const int c = (int)std::min<long long>(n, chunk);
        NvtxRange chunk_range(use_graphs && c == chunk && chunk > 1 ? "lbm.chunk.graph" : "lbm.chunk");
        if (use_graphs && c == chunk && chunk > 1) {
            if (!graph_ || graph_chunk_ != c) {
                invalidate_graph();
                cudaGraph_t gr = nullptr;
                CK(cudaStreamBeginCapture(stream_, cudaStreamCaptureModeThreadLocal));
                int rc = enqueue_chunk(c);
                cudaError_t e = cudaStreamEndCapture(stream_, &gr);
                if (rc) {
                    if (gr) cudaGraphDestroy(gr);
                    return rc;
                }
                if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
                e = cudaGraphInstantiate(&graph_, gr, 0);
                cudaGraphDestroy(gr);
                if (e != cudaSuccess) {
                    graph_ = nullptr;
                    return cuda_fail(e, "cudaGraphInstantiate");
                }
                graph_chunk_ = c;
                graph_launches_ = last_chunk_launches_;
            }
            CK(cudaGraphLaunch(graph_, stream_));
            launches_ += graph_launches_;
        } else {
            int rc = enqueue_chunk(c);
            if (rc) return rc;
            launches_ += last_chunk_launches_;
        }
        mirror_advance(c);
        n -= c;
    }
    return LBM_OK;
}

int Engine::step_profiled(long long n, double* ms, int cap, double* total_ms) {
    if (n < 0 || (cap > 0 && !ms)) { set_error("bad arguments"); return LBM_EINVAL; }
    const int G = (int)groups.size();
    for (int i = 0; i < cap; ++i) ms[i] = 0.0;
    if (total_ms) *total_ms = 0.0;
    if (n == 0) return LBM_OK;
    NvtxRange range("lbm.step_profiled");
    // events: per step and group, one before and one after each launch
    struct Mark { int slot; cudaEvent_t a, b; };
    std::vector<Mark> marks;
    std::vector<cudaEvent_t> pool;
    auto ev = [&]() -> cudaEvent_t {
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        pool.push_back(e);
        return e;
    };
    auto cleanup = [&]() { for (auto e : pool) cudaEventDestroy(e); };
    cudaEvent_t t0 = ev(), t1 = ev();
    if (!t0 || !t1) { cleanup(); return cuda_fail(cudaGetLastError(), "cudaEventCreate"); }
    CK(cudaEventRecord(t0, stream_));
    for (long long s = 0; s < n; ++s) {
        for (int gi = 0; gi < G; ++gi) {
            Group& g = groups[gi];
            if (g.cap_lat == 0) continue;  // empty groups launch too: kernels read the live count
            const GroupDev gd = g.dev();
            const int nk = g.model == LBM_CS ? 1 : fd_stages(g.scheme);
            for (int st = 1; st <= nk; ++st) {
                static const char* const kNames[4] = {"lbm.cs_step", "lbm.fd_stage1", "lbm.fd_stage2", "lbm.fd_stage3"};
                NvtxRange kernel_range(kNames[g.model == LBM_CS ? 0 : st]);
                cudaEvent_t a = ev(), b = ev();
                if (!a || !b) { cleanup(); return cuda_fail(cudaGetLastError(), "cudaEventCreate"); }
                cudaEventRecord(a, stream_);
                cudaError_t e = g.model == LBM_CS ? launch_cs_step(g.precision, g.tile, g.grid, gd, 0, stream_)
                                                  : launch_fd_stage(g.precision, g.q1, g.scheme, g.tile, g.grid, gd, 0, st,
                                                                    stream_);
                cudaEventRecord(b, stream_);
                if (e != cudaSuccess) { cleanup(); return cuda_fail(e, "profiled launch"); }
                ++launches_;
                marks.push_back({gi * 4 + (st - 1), a, b});
                if (st == 1 && g.any_obs) {
                    cudaEvent_t c = ev(), d = ev();
                    if (!c || !d) { cleanup(); return cuda_fail(cudaGetLastError(), "cudaEventCreate"); }
                    cudaEventRecord(c, stream_);
                    e = launch_obs_finalize(gd, g.cap_lat, g.nchunks, g.d_chunks, 0, stream_);
                    cudaEventRecord(d, stream_);
                    if (e != cudaSuccess) { cleanup(); return cuda_fail(e, "profiled finalize"); }
                    launches_ += 2;
                    marks.push_back({gi * 4 + 3, c, d});
                }
            }
        }
        for (auto& g : groups) {
            if (g.cap_lat == 0) continue;  // empty groups launch too: kernels read the live count
            cudaError_t e = launch_advance(g.dev(), g.cap_lat, 1, g.flips() ? 1 : 0, stream_);
            if (e != cudaSuccess) { cleanup(); return cuda_fail(e, "launch_advance"); }
            ++launches_;
        }
        mirror_advance(1);
    }
    CK(cudaEventRecord(t1, stream_));
    cudaError_t e = cudaEventSynchronize(t1);
    if (e != cudaSuccess) { cleanup(); return cuda_fail(e, "cudaEventSynchronize"); }
    for (auto& m : marks) {
        float t = 0;
        cudaEventElapsedTime(&t, m.a, m.b);
        if (m.slot < cap) ms[m.slot] += t;
    }
    float tt = 0;
    cudaEventElapsedTime(&tt, t0, t1);
    if (total_ms) *total_ms = tt;
    cleanup();
    return LBM_OK;
}

int Engine::sync() {
    CK(cudaStreamSynchronize(stream_));
    CK(cudaGetLastError());
    return check_device_errors();
}

int Engine::inject_wait_timeout(int us) {
    if (us < 0 || us > 1000000) {
        set_error("wait-timeout injection takes 0 (off) to 1e6 microseconds");
        return LBM_EINVAL;
    }
    inject_us_ = us;
    for (auto& g : groups) {
        if (!g.d_hdr) continue;
        CK(cudaMemcpyAsync(g.d_hdr + 3, &inject_us_, sizeof(int), cudaMemcpyHostToDevice, stream_));
    }
    CK(cudaStreamSynchronize(stream_));
    return LBM_OK;
}

// Error words the kernels raise instead of hanging (bounded waits that ran
// out); read and cleared here.
int Engine::check_device_errors() {
    int bad = 0;
    for (auto& g : groups) {
        if (!g.d_hdr) continue;
        int h[4];
        CK(cudaMemcpy(h, g.d_hdr, sizeof h, cudaMemcpyDeviceToHost));
        if (h[2] != 0) {
            bad |= h[2];
            const int zero = 0;
            CK(cudaMemcpy(g.d_hdr + 2, &zero, sizeof zero, cudaMemcpyHostToDevice));
        }
    }
    if (bad & ERR_BOUNDS) {
        set_error("a kernel reached outside a state buffer (caught by the bounds-checked build)");
        return LBM_ECUDA;
    }
    if (bad) {
        set_error("a device-side wait ran out of time (bulk-copy pipeline); results of that step are invalid");
        return LBM_ETIMEOUT;
    }
    return LBM_OK;
}

int Engine::ensure_io(Lattice& L, size_t bytes) {
    if (L.io_bytes >= bytes) return LBM_OK;
    CK(cudaStreamSynchronize(stream_));
    cudaFree(L.d_io);
    L.d_io = nullptr;
    L.io_bytes = 0;
    cudaError_t e = cudaMalloc(&L.d_io, bytes);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(readout staging)");
    L.io_bytes = bytes;
    return LBM_OK;
}

static bool all_finite(const double* a, size_t n) {
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(a[i])) return false;
    return true;
}

// Input errors the state initialisation kernels flagged in the group's error
// word (the values are checked on the device, where they are read anyway):
// cleared here; true if there were any.
bool Engine::take_input_error(const Group& g) {
    int h = 0;
    if (cudaMemcpy(&h, g.d_hdr + 2, sizeof h, cudaMemcpyDeviceToHost) != cudaSuccess) return false;
    if (!(h & ERR_INPUT)) return false;
    h &= ~ERR_INPUT;
    cudaMemcpy(g.d_hdr + 2, &h, sizeof h, cudaMemcpyHostToDevice);
    return true;
}

int Engine::init(int i, const double* rho, const double* ux, const double* uy) {
    if (!valid(i) || !rho || !ux || !uy) { set_error("bad arguments"); return LBM_EINVAL; }
    Lattice& L = lat[i];
    const size_t n = (size_t)L.spec.nx * L.spec.ny;
    int rc = ensure_io(L, sizeof(double) * 3 * n);
    if (rc) return rc;
    L.step0 = 0;
    L.cur = 0;
    L.obs_base = 0;
    if (L.remaining == 0 || L.remaining == UNLIMITED) L.remaining = UNLIMITED;
    rc = upload_group(L.group);
    if (rc) return rc;
    CK(cudaMemcpyAsync(L.d_io, rho, sizeof(double) * n, cudaMemcpyHostToDevice, stream_));
    CK(cudaMemcpyAsync(L.d_io + n, ux, sizeof(double) * n, cudaMemcpyHostToDevice, stream_));
    CK(cudaMemcpyAsync(L.d_io + 2 * n, uy, sizeof(double) * n, cudaMemcpyHostToDevice, stream_));
    const Group& g = groups[L.group];
    CK(launch_init_equilibrium(L.spec.precision, L.spec.q_per_axis, L.spec.model == LBM_CS, g.d_desc + L.slot,
                               L.spec.nx, L.spec.ny, L.d_io, L.d_io + n, L.d_io + 2 * n, stream_));
    CK(cudaStreamSynchronize(stream_));
    if (take_input_error(g)) {
        set_error("rho must be positive and finite and u finite (the state is not initialised)");
        return LBM_EINVAL;
    }
    return LBM_OK;
}

int Engine::set_populations(int i, const double* f) {
    if (!valid(i) || !f) { set_error("bad arguments"); return LBM_EINVAL; }
    Lattice& L = lat[i];
    const size_t n = (size_t)L.spec.nx * L.spec.ny * L.K;
    int rc = ensure_io(L, sizeof(double) * n);
    if (rc) return rc;
    CK(cudaMemcpyAsync(L.d_io, f, sizeof(double) * n, cudaMemcpyHostToDevice, stream_));
    const Group& g = groups[L.group];
    CK(launch_set_populations(L.spec.precision, L.spec.q_per_axis, L.spec.model == LBM_CS, g.d_desc + L.slot,
                              L.spec.nx, L.spec.ny, L.d_io, stream_));
    CK(cudaStreamSynchronize(stream_));
    if (take_input_error(g)) {
        set_error("populations must be finite (the state is not set)");
        return LBM_EINVAL;
    }
    return LBM_OK;
}

int Engine::readout(int i, double* f, double* rho, double* ux, double* uy, bool obs) {
    Lattice& L = lat[i];
    const size_t n = (size_t)L.spec.nx * L.spec.ny;
    size_t need = 0;
    if (f) need = std::max(need, (size_t)L.K * n);
    if (rho) need = std::max(need, 3 * n);
    if (need) {
        int rc = ensure_io(L, sizeof(double) * need);
        if (rc) return rc;
    }
    const Group& g = groups[L.group];
    double* df = f ? L.d_io : nullptr;
    double* dr = rho ? L.d_io : nullptr;
    if (f && rho) { set_error("internal: one readout target at a time"); return LBM_EINVAL; }
    CK(launch_readout(L.spec.precision, L.spec.q_per_axis, L.spec.model == LBM_CS, g.d_desc + L.slot, L.spec.nx,
                      L.spec.ny, 0, 0, L.spec.nx, L.spec.ny, df, dr, dr ? dr + n : nullptr, dr ? dr + 2 * n : nullptr,
                      obs ? L.d_part : nullptr, L.part_blocks, stream_));
    if (f) CK(cudaMemcpyAsync(f, L.d_io, sizeof(double) * L.K * n, cudaMemcpyDeviceToHost, stream_));
    if (rho) {
        CK(cudaMemcpyAsync(rho, L.d_io, sizeof(double) * n, cudaMemcpyDeviceToHost, stream_));
        CK(cudaMemcpyAsync(ux, L.d_io + n, sizeof(double) * n, cudaMemcpyDeviceToHost, stream_));
        CK(cudaMemcpyAsync(uy, L.d_io + 2 * n, sizeof(double) * n, cudaMemcpyDeviceToHost, stream_));
    }
    CK(cudaStreamSynchronize(stream_));
    return LBM_OK;
}

int Engine::moments(int i, double* rho, double* ux, double* uy) {
    if (!valid(i) || !rho || !ux || !uy) { set_error("bad arguments"); return LBM_EINVAL; }
    return readout(i, nullptr, rho, ux, uy, false);
}

int Engine::populations(int i, double* f) {
    if (!valid(i) || !f) { set_error("bad arguments"); return LBM_EINVAL; }
    return readout(i, f, nullptr, nullptr, nullptr, false);
}

int Engine::populations_region(int i, int x0, int y0, int wx, int wy, double* f) {
    if (!valid(i) || !f) { set_error("bad arguments"); return LBM_EINVAL; }
    Lattice& L = lat[i];
    if (x0 < 0 || y0 < 0 || x0 >= L.spec.nx || y0 >= L.spec.ny || wx < 1 || wy < 1 || wx > L.spec.nx ||
        wy > L.spec.ny) {
        set_error("window out of range");
        return LBM_EINVAL;
    }
    const size_t n = (size_t)wx * wy;
    int rc = ensure_io(L, sizeof(double) * L.K * n);
    if (rc) return rc;
    const Group& g = groups[L.group];
    CK(launch_readout(L.spec.precision, L.spec.q_per_axis, L.spec.model == LBM_CS, g.d_desc + L.slot, L.spec.nx,
                      L.spec.ny, x0, y0, wx, wy, L.d_io, nullptr, nullptr, nullptr, nullptr, 0, stream_));
    CK(cudaMemcpyAsync(f, L.d_io, sizeof(double) * L.K * n, cudaMemcpyDeviceToHost, stream_));
    CK(cudaStreamSynchronize(stream_));
    return LBM_OK;
}

int Engine::observables(int i, lbm_obs* out) {
    if (!valid(i) || !out) { set_error("bad arguments"); return LBM_EINVAL; }
    int rc = readout(i, nullptr, nullptr, nullptr, nullptr, true);
    if (rc) return rc;
    Lattice& L = lat[i];
    double s[NOBS];
    CK(cudaMemcpy(s, L.d_snap, sizeof s, cudaMemcpyDeviceToHost));
    const double n = (double)L.spec.nx * L.spec.ny;
    out->step = L.step0;
    out->time = (double)L.step0 * L.spec.dt;
    out->mass = n * L.rho0s + s[0];
    out->mom_x = s[1];
    out->mom_y = s[2];
    out->amp = L.probe_comp >= 0 ? L.probe_norm * s[3] : 0.0;
    out->nonfinite = (std::isfinite(out->mass) && std::isfinite(out->amp) && std::isfinite(out->mom_x) &&
                      std::isfinite(out->mom_y)) ? 0 : 1;
    out->reserved = 0;
    return LBM_OK;
}

int Engine::set_probe(int i, int comp, const double* px, const double* py, double norm) {
    if (!valid(i) || (comp != 0 && comp != 1) || !px || !py || !std::isfinite(norm)) {
        set_error("bad probe arguments");
        return LBM_EINVAL;
    }
    Lattice& L = lat[i];
    const int nx = L.spec.nx, ny = L.spec.ny;
    if (!all_finite(px, nx) || !all_finite(py, ny)) { set_error("probe tables must be finite"); return LBM_EINVAL; }
    CK(cudaStreamSynchronize(stream_));
    if (!L.d_px) {
        CK(cudaMalloc(&L.d_px, sizeof(double) * nx));
        CK(cudaMalloc(&L.d_py, sizeof(double) * ny));
        CK(cudaMalloc(&L.d_pxf, sizeof(float) * nx));
        CK(cudaMalloc(&L.d_pyf, sizeof(float) * ny));
    }
    std::vector<float> fx(px, px + nx), fy(py, py + ny);
    CK(cudaMemcpy(L.d_px, px, sizeof(double) * nx, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(L.d_py, py, sizeof(double) * ny, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(L.d_pxf, fx.data(), sizeof(float) * nx, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(L.d_pyf, fy.data(), sizeof(float) * ny, cudaMemcpyHostToDevice));
    L.probe_comp = comp;
    L.probe_norm = norm;
    return upload_group(L.group);
}

int Engine::record(int i, long long every, long long cap) {
    if (!valid(i) || every < 0 || (every > 0 && cap < 1) || cap > (1LL << 30)) {
        set_error("bad record arguments");
        return LBM_EINVAL;
    }
    Lattice& L = lat[i];
    CK(cudaStreamSynchronize(stream_));
    cudaFree(L.d_series);
    L.d_series = nullptr;
    L.obs_every = 0;
    L.obs_cap = 0;
    if (every > 0) {
        CK(cudaMalloc(&L.d_series, sizeof(lbm_obs) * cap));
        CK(cudaMemset(L.d_series, 0, sizeof(lbm_obs) * cap));
        L.obs_every = every;
        L.obs_cap = cap;
    }
    L.obs_base = L.step0;
    invalidate_graph();
    return upload_group(L.group);
}

int Engine::series(int i, lbm_obs* out, long long cap, long long* count) {
    if (!valid(i) || cap < 0 || (cap > 0 && !out)) { set_error("bad arguments"); return LBM_EINVAL; }
    Lattice& L = lat[i];
    CK(cudaStreamSynchronize(stream_));
    long long n = 0;
    if (L.obs_every > 0 && L.step0 > L.obs_base) n = (L.step0 - L.obs_base + L.obs_every - 1) / L.obs_every;
    n = std::min(n, L.obs_cap);
    if (count) *count = n;
    const long long m = std::min(n, cap);
    if (m > 0) CK(cudaMemcpy(out, L.d_series, sizeof(lbm_obs) * m, cudaMemcpyDeviceToHost));
    return LBM_OK;
}

int Engine::set_budget(int i, long long steps) {
    if (!valid(i) || steps < 0) { set_error("bad budget"); return LBM_EINVAL; }
    CK(cudaStreamSynchronize(stream_));
    lat[i].remaining = steps;
    return upload_group(lat[i].group);
}

int Engine::set_budgets(const std::vector<std::pair<int, long long>>& budgets) {
    for (const auto& b : budgets)
        if (!valid(b.first) || b.second < 0) { set_error("bad budget"); return LBM_EINVAL; }
    CK(cudaStreamSynchronize(stream_));
    std::vector<char> touched(groups.size(), 0);
    for (const auto& b : budgets) {
        lat[b.first].remaining = b.second;
        touched[lat[b.first].group] = 1;
    }
    for (int gi = 0; gi < (int)groups.size(); ++gi)
        if (touched[gi]) {
            const int rc = upload_group(gi);
            if (rc) return rc;
        }
    return LBM_OK;
}

int Engine::release_io(int i) {
    if (!valid(i)) { set_error("bad arguments"); return LBM_EINVAL; }
    CK(cudaStreamSynchronize(stream_));
    cudaFree(lat[i].d_io);
    lat[i].d_io = nullptr;
    lat[i].io_bytes = 0;
    return LBM_OK;
}

int Engine::set_eps(int i, double eps) {
    Lattice& L = lat[i];
    if (L.spec.model != LBM_FD) { set_error("WENO epsilon applies to FD lattices"); return LBM_EINVAL; }
    const bool ok = L.spec.precision == LBM_FP64 ? (eps >= 1e-60 && eps <= 1e60) : (eps >= 1e-8 && eps <= 1e9);
    if (!ok || !std::isfinite(eps)) { set_error("epsilon out of range for this precision"); return LBM_EINVAL; }
    CK(cudaStreamSynchronize(stream_));
    L.eps = eps;
    return upload_group(L.group);
}

// ---- checkpoint ---------------------------------------------------------
struct CkptHeader {
    char magic[8];
    lbm_spec spec;
    int64_t step0;
    int64_t eps_bits;
    int64_t state_bytes;
    int64_t phase;   // in-place CS: phase of the stored state
};

size_t Engine::checkpoint_size(int i) const {
    const Lattice& L = lat[i];
    return sizeof(CkptHeader) + (size_t)L.K * L.plane * L.elem;
}

int Engine::save(int i, void* buf, size_t size) {
    if (!valid(i) || !buf || size < checkpoint_size(i)) { set_error("checkpoint buffer too small"); return LBM_EINVAL; }
    Lattice& L = lat[i];
    CkptHeader h;
    memset(&h, 0, sizeof h);
    memcpy(h.magic, "LBMCKPT2", 8);
    h.spec = L.spec;
    h.step0 = L.step0;
    memcpy(&h.eps_bits, &L.eps, 8);
    h.state_bytes = (int64_t)L.K * L.plane * L.elem;
    h.phase = L.inplace() ? L.cur : 0;
    memcpy(buf, &h, sizeof h);
    CK(cudaMemcpyAsync(static_cast<char*>(buf) + sizeof h, L.buf[L.state_buf()], h.state_bytes, cudaMemcpyDeviceToHost,
                       stream_));
    CK(cudaStreamSynchronize(stream_));
    return LBM_OK;
}

int Engine::load(int i, const void* buf, size_t size) {
    if (!valid(i) || !buf || size < sizeof(CkptHeader)) { set_error("bad checkpoint"); return LBM_EINVAL; }
    Lattice& L = lat[i];
    CkptHeader h;
    memcpy(&h, buf, sizeof h);
    if (memcmp(h.magic, "LBMCKPT2", 8) != 0 || memcmp(&h.spec, &L.spec, sizeof(lbm_spec)) != 0 ||
        h.state_bytes != (int64_t)L.K * L.plane * L.elem || size < checkpoint_size(i)) {
        set_error("checkpoint does not match this lattice");
        return LBM_EINVAL;
    }
    CK(cudaStreamSynchronize(stream_));
    CK(cudaMemcpyAsync(L.buf[0], static_cast<const char*>(buf) + sizeof h, h.state_bytes, cudaMemcpyHostToDevice, stream_));
    L.cur = L.inplace() ? (int)(h.phase & 1) : 0;
    L.step0 = h.step0;
    memcpy(&L.eps, &h.eps_bits, 8);
    L.obs_base = L.step0;
    return upload_group(L.group);
}

}  // namespace lbm
