// Autotuner: picks the tile shape and grid size of every group by
// timing each candidate on the group's own lattices (state saved and
// restored around the trials). Results are cached per (model, q, precision,
// storage, work-size class) for the life of the process.
#include <algorithm>
#include <cstdio>
#include <map>
#include <mutex>
#include <tuple>

#include "engine.h"

namespace lbm {

namespace {
using Key = std::tuple<int, int, int, int, int>;
std::map<Key, std::pair<int, int>>& cache() {
    static std::map<Key, std::pair<int, int>> m;
    return m;
}
std::mutex& cache_mutex() {
    static std::mutex m;
    return m;
}
int size_class(long long cells) {
    int c = 0;
    while (cells > 1) {
        cells >>= 1;
        ++c;
    }
    return c;
}
}  // namespace

int Engine::tune(int trial_steps, std::string* report) {
    if (trial_steps < 1) trial_steps = 1;
    std::string rep;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return cuda_fail(cudaGetLastError(), "cudaEventCreate");
    for (int gi = 0; gi < (int)groups.size(); ++gi) {
        Group& g = groups[gi];
        if (g.members.empty()) continue;
        long long cells = 0;
        for (int li : g.members) cells += (long long)lat[li].spec.nx * lat[li].spec.ny;
        const Key key{g.model, g.q1, g.precision, g.scheme, size_class(cells)};
        {
            std::lock_guard<std::mutex> lk(cache_mutex());
            auto it = cache().find(key);
            if (it != cache().end()) {
                int rc = set_group_config(gi, it->second.first, 0);
                if (rc) return rc;
                g.grid = std::min(g.grid, std::max(1, it->second.second));
                char b[160];
                snprintf(b, sizeof b, "[g%d %s q%d %s cached tile=%d grid=%d] ", gi, g.model == LBM_CS ? "CS" : "FD", g.q1,
                         g.precision == LBM_FP64 ? "fp64" : "fp32", g.tile, g.grid);
                rep += b;
                continue;
            }
        }
        // save the state of the group's lattices
        std::vector<void*> saved;
        for (int li : g.members) {
            void* p = nullptr;
            cudaError_t e = cudaMalloc(&p, lat[li].state_bytes());
            if (e != cudaSuccess) {
                for (void* q : saved) cudaFree(q);
                return cuda_fail(e, "cudaMalloc(tune save)");
            }
            e = cudaMemcpyAsync(p, lat[li].mem, lat[li].state_bytes(), cudaMemcpyDeviceToDevice, stream_);
            if (e != cudaSuccess) return cuda_fail(e, "tune save copy");
            saved.push_back(p);
        }
        const int ntiles = g.model == LBM_CS ? (int)CS_NTILES : (int)FD_NTILES;
        float best = 1e30f;
        int best_tile = g.tile, best_grid = g.grid;
        const int orig_any_obs = g.any_obs;
        g.any_obs = false;
        for (int t = 0; t < ntiles; ++t) {
            if (g.model == LBM_FD && !fd_variant_fits(g.precision, g.q1, t, g.scheme)) continue;
            int rc = set_group_config(gi, t, 0);
            if (rc) return rc;
            g.any_obs = false;
            const int full = g.total_items;
            const int pers = std::min(full, persistent_grid(g, t));
            const int cands[3] = {pers, std::min(full, 2 * pers), full};
            for (int ci = 0; ci < 3; ++ci) {
                const int grid = std::max(1, cands[ci]);
                if (ci > 0 && grid == cands[ci - 1]) continue;
                g.grid = grid;
                const GroupDev gd = g.dev();
                auto run = [&](int steps) -> cudaError_t {
                    for (int j = 0; j < steps; ++j) {
                        cudaError_t e;
                        if (g.model == LBM_CS) e = launch_cs_step(g.precision, g.tile, g.grid, gd, j, stream_);
                        else {
                            e = cudaSuccess;
                            for (int st = 1; st <= fd_stages(g.scheme) && e == cudaSuccess; ++st)
                                e = launch_fd_stage(g.precision, g.q1, g.scheme, g.tile, g.grid, gd, j, st, stream_);
                        }
                        if (e != cudaSuccess) return e;
                    }
                    return cudaSuccess;
                };
                cudaError_t e = run(1);
                if (e == cudaSuccess) e = cudaEventRecord(e0, stream_);
                if (e == cudaSuccess) e = run(trial_steps);
                if (e == cudaSuccess) e = cudaEventRecord(e1, stream_);
                if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                if (e != cudaSuccess) return cuda_fail(e, "tune trial");
                float ms = 0;
                cudaEventElapsedTime(&ms, e0, e1);
                if (ms < best) {
                    best = ms;
                    best_tile = t;
                    best_grid = grid;
                }
            }
        }
        // restore state and apply the winner
        for (size_t m = 0; m < g.members.size(); ++m) {
            const Lattice& L = lat[g.members[m]];
            cudaError_t e = cudaMemcpyAsync(L.mem, saved[m], L.state_bytes(), cudaMemcpyDeviceToDevice, stream_);
            if (e != cudaSuccess) return cuda_fail(e, "tune restore copy");
        }
        cudaStreamSynchronize(stream_);
        for (void* p : saved) cudaFree(p);
        g.any_obs = orig_any_obs;
        int rc = set_group_config(gi, best_tile, best_grid);
        if (rc) return rc;
        {
            std::lock_guard<std::mutex> lk(cache_mutex());
            cache()[key] = {best_tile, best_grid};
        }
        char b[200];
        snprintf(b, sizeof b, "[g%d %s q%d %s tile=%dx%d grid=%d %.4f ms/step] ", gi, g.model == LBM_CS ? "CS" : "FD",
                 g.q1, g.precision == LBM_FP64 ? "fp64" : "fp32",
                 g.model == LBM_CS ? cs_tile_tx(best_tile) : fd_tile_tx(best_tile),
                 g.model == LBM_CS ? cs_tile_ty(best_tile) : fd_tile_ty(best_tile), best_grid, best / trial_steps);
        rep += b;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    invalidate_graph();
    if (report) *report = rep;
    return LBM_OK;
}

}  // namespace lbm
