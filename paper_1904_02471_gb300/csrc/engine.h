// Host engine behind the C ABI: owns the device memory of a set of lattices,
// groups them by (model, velocity set, storage type), keeps the device
// descriptors in sync and enqueues steps (directly or by replaying a captured
// CUDA graph of a fixed chunk of steps).
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <utility>
#include <vector>

#include "kernels.h"

namespace lbm {

constexpr long long UNLIMITED = (1LL << 62);

// Thread-local detail of the last error, returned by lbm_last_error(); kept
// in a fixed buffer, so recording an error never allocates.
void set_error(const char* msg);
inline void set_error(const std::string& msg) { set_error(msg.c_str()); }
int cuda_fail(cudaError_t e, const char* what);

// State buffers of a lattice: two-buffer CS 2, in-place CS 1, FD 3 (f^n and
// the two stage buffers; IMEX: f^n, Z, P), temporally blocked FD 2 (f^n and
// f^(n+1), alternating).
inline int state_buffers(const lbm_spec& s) {
    if (s.model == LBM_CS) return s.storage == LBM_STORE_INPLACE ? 1 : 2;
    return s.scheme == LBM_TS_RK3_FUSED ? 2 : 3;
}

struct Lattice {
    lbm_spec spec{};
    int K = 0;
    int pitch = 0;
    long long plane = 0;
    int elem = 0;            // bytes per stored value
    int nbuf = 0;            // state buffers: state_buffers(spec)
    void* mem = nullptr;     // one allocation for all state buffers
    void* buf[3] = {nullptr, nullptr, nullptr};
    double omega = 0, cdx = 0, dt_tau = 0, rho0s = 0, eps = 1e-6;
    // host mirror of the device-side dynamic state
    long long step0 = 0;
    long long remaining = UNLIMITED;
    int cur = 0;             // buffer holding the state (two-buffer CS, fused FD; 0 for
                             // RK3 / IMEX FD) or phase (in-place CS)
    bool inplace() const { return spec.model == LBM_CS && spec.storage == LBM_STORE_INPLACE; }
    // cur flips with every step
    bool flips() const { return spec.model == LBM_CS || spec.scheme == LBM_TS_RK3_FUSED; }
    // buffer that holds the current state
    int state_buf() const { return inplace() ? 0 : cur; }
    // lbm_view::cs_pull_phase of the current state
    int phase_code() const { return spec.model != LBM_CS ? 0 : (!inplace() ? 1 : (cur ? 2 : 0)); }
    // observables
    int probe_comp = -1;
    double probe_norm = 0;
    double* d_px = nullptr;
    double* d_py = nullptr;
    float* d_pxf = nullptr;
    float* d_pyf = nullptr;
    long long obs_every = 0, obs_cap = 0, obs_base = 0;
    lbm_obs* d_series = nullptr;
    // scratch: staging for init/readout (lazy), snapshot partials
    double* d_io = nullptr;
    size_t io_bytes = 0;
    double* d_part = nullptr;
    int part_blocks = 0;
    double* d_snap = nullptr;
    int group = -1;
    int slot = -1;
    bool active = true;      // member of its group's work list
    bool alive = true;       // false once removed (memory freed, index retired)
    // buffer b starts HEAD elements into its slot of the allocation; slots are
    // K * plane + TAIL elements (see engine.cu for why)
    static constexpr long long HEAD = 4, TAIL = 1024;
    long long buf_stride() const { return (long long)K * plane + TAIL; }
    size_t state_bytes() const { return (size_t)nbuf * buf_stride() * elem; }
};

struct Group {
    int model = 0, q1 = 0, precision = 0;
    int scheme = LBM_TS_RK3;   // FD time integration
    // the lattices' cur flips with every step (CS, fused FD)
    bool flips() const { return model == LBM_CS || scheme == LBM_TS_RK3_FUSED; }
    int tile = 0;
    int grid = 0;
    std::vector<int> members;
    LatDesc* d_desc = nullptr;
    int* d_item_begin = nullptr;
    int* d_hdr = nullptr;
    double* d_partials = nullptr;
    int cap_lat = 0;
    long long cap_items = 0;
    int total_items = 0;
    bool any_obs = false;
    int nchunks = 1;            // observables reduction chunks per lattice
    double* d_chunks = nullptr; // [cap_lat][nchunks][NOBS]
    int chunk_cap = 0;
    GroupDev dev() const { return GroupDev{d_desc, d_item_begin, d_hdr}; }
};

class Engine {
  public:
    Engine() = default;
    ~Engine();
    Engine(const Engine&) = delete;
    Engine& operator=(const Engine&) = delete;

    int create(const lbm_spec* specs, int n, void* stream);
    // dynamic membership (continuous batching): a lattice index stays valid
    // until remove_lattice; removed indices are never reused
    int open(void* stream);
    int add_lattice(const lbm_spec* spec, int* index, bool upload = true);
    int remove_lattice(int i);
    static size_t footprint(const lbm_spec& s);  // device bytes of one lattice
    bool dynamic_ = false;   // persistent grids sized for the machine, not the current work
    int grid_mult_ = 1;      // dynamic engines: blocks per resident block slot (1: one block set per SM)
    int inject_us_ = 0;      // group header word 3 (wait-timeout injection)
    static int validate(const lbm_spec* in, lbm_spec* out);

    int n_lattices() const { return (int)lat.size(); }
    bool valid(int i) const { return i >= 0 && i < (int)lat.size() && lat[i].alive; }
    Lattice& L(int i) { return lat[i]; }
    cudaStream_t stream() const { return stream_; }

    int init(int i, const double* rho, const double* ux, const double* uy);
    int set_populations(int i, const double* f);
    int step(long long n);
    // n steps launched one by one with CUDA events around every kernel;
    // ms[g * 4 + kind] accumulates the device time of group g's kernels of
    // kind 0..2 (CS step, or FD stages 1..3) and 3 (observables finalise);
    // *total_ms spans the whole sequence.
    int step_profiled(long long n, double* ms, int cap, double* total_ms);
    long long kernel_launches() const { return launches_; }
    int sync();
    int check_device_errors();
    bool take_input_error(const Group& g);
    // Test injection of a device-side wait that runs out (see lbm.h,
    // lbm_inject_wait_timeout): 0 = off, else the wait limit in microseconds.
    int inject_wait_timeout(int microseconds);
    int moments(int i, double* rho, double* ux, double* uy);
    int populations(int i, double* f);
    int populations_region(int i, int x0, int y0, int wx, int wy, double* f);
    int observables(int i, lbm_obs* out);
    int set_probe(int i, int comp, const double* px, const double* py, double norm);
    int record(int i, long long every, long long cap);
    int series(int i, lbm_obs* out, long long cap, long long* count);
    int set_budget(int i, long long steps);
    // Several budgets at once: one upload per group touched.
    int set_budgets(const std::vector<std::pair<int, long long>>& budgets);
    int release_io(int i);   // free the staging buffer of init / readout
    int set_eps(int i, double eps);
    size_t checkpoint_size(int i) const;
    int save(int i, void* buf, size_t size);
    int load(int i, const void* buf, size_t size);

    // Tile / grid selection for a group (autotuner hooks).
    int set_group_config(int g, int tile, int grid);
    int n_groups() const { return (int)groups.size(); }
    Group& G(int g) { return groups[g]; }
    int sm_count() const { return sm_count_; }
    int default_grid(const Group& g, int tile) const;
    int persistent_grid(const Group& g, int tile) const;
    int tune(int trial_steps, std::string* report);

    int chunk = 32;          // steps per captured graph
    bool use_graphs = true;

  protected:
    int upload_group(int g);
    int upload_all();
    int enqueue_chunk(int c);
    void mirror_advance(int c);
    int ensure_io(Lattice& L, size_t bytes);
    int readout(int i, double* f, double* rho, double* ux, double* uy, bool obs);
    LatDesc make_desc(const Lattice& L, const Group& g, int item_begin, double* partials) const;
    void invalidate_graph();
    void free_lattice(Lattice& L);

    std::vector<Lattice> lat;
    std::vector<Group> groups;
    cudaStream_t stream_ = nullptr;
    bool own_stream_ = false;
    int sm_count_ = 0;
    cudaGraphExec_t graph_ = nullptr;
    int graph_chunk_ = 0;
    long long graph_launches_ = 0;   // kernel nodes in the captured chunk
    long long launches_ = 0;         // kernels enqueued so far (graph nodes included)
    long long last_chunk_launches_ = 0;
};

}  // namespace lbm
