// Host-side launch interface of the kernels (no templates cross this header).
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"

namespace lbm {

// Device view of a group: descriptors, first item of each lattice, and a
// two-int header {number of lattices, total work items} read by the kernels
// at run time (so a captured graph stays valid when the membership changes).
struct GroupDev {
    LatDesc* desc;
    const int* item_begin;
    int* hdr;   // {lattices, items, error bits, unused}
};

// Tile variants. CS: TX threads along x, RY rows per thread; the B
// variants are the warp-specialised bulk-copy kernel (W columns x RB rows).
// FD: TX x TY cells per tile, one cell per thread.
enum CsTile { CS_T128x1 = 0, CS_T128x2, CS_T256x1, CS_T256x2, CS_T64x4, CS_B256x32, CS_B128x32, CS_NTILES };
enum FdTile { FD_T32x8 = 0, FD_T32x4, FD_T32x16, FD_T32x2, FD_NTILES };

int cs_tile_tx(int v);
int cs_tile_ty(int v);
int fd_tile_tx(int v);
int fd_tile_ty(int v);

// One CS step (Eq. sc_evolution) for every lattice of the group at sub-step j.
cudaError_t launch_cs_step(int precision, int tile, int grid, const GroupDev& g, int j, cudaStream_t s);
// One stage of the FD update for every lattice of the group: scheme
// LBM_TS_RK3, SSP-RK3 stages 1..3; LBM_TS_IMEX, IMEX-SSP2(2,2,2) stages 1..2;
// LBM_TS_RK3_FUSED, stage 1 = the whole SSP-RK3 step (launch_fd_fused).
cudaError_t launch_fd_stage(int precision, int q1, int scheme, int tile, int grid, const GroupDev& g, int j,
                            int stage, cudaStream_t s);
// Launches per FD step of a scheme.
inline int fd_stages(int scheme) { return scheme == LBM_TS_IMEX ? 2 : (scheme == LBM_TS_RK3_FUSED ? 1 : 3); }
// Temporally blocked SSP-RK3 step (kernels_fd_fused.cu): the three stages of
// a step for every lattice of the group in one launch, buf[cur] -> buf[cur ^ 1]
// (tile FD_T32x16, FD_T32x8 or FD_T32x4: output tiles of 32 x 16, 32 x 8 or
// 32 x 4 nodes, where they fit the device's shared memory).
cudaError_t launch_fd_fused(int precision, int q1, int tile, int grid, const GroupDev& g, int j, cudaStream_t s);
bool fd_fused_fits(int precision, int q1, int tile);
int fd_fused_blocks_per_sm(int precision, int q1, int tile);
// Occupancy-based resident CTAs per SM of a variant (for persistent grids).
int cs_blocks_per_sm(int precision, int tile);
int fd_blocks_per_sm(int precision, int q1, int tile, int scheme);
// Whether an FD variant of a scheme fits this device (shared memory); unfit
// variants are refused by set_group_config and skipped by the autotuner.
bool fd_variant_fits(int precision, int q1, int tile, int scheme);

// Fused-observables finalisation: lattices observing at sub-step j reduce
// their tile partials (in nchunks chunks, scratch chunks[max_lat][nchunks][NOBS])
// into their series. Two launches.
cudaError_t launch_obs_finalize(const GroupDev& g, int max_lat, int nchunks, double* chunks, int j, cudaStream_t s);
// Advance steps/phase of every lattice by min(remaining, c).
cudaError_t launch_advance(const GroupDev& g, int max_lat, int c, int flip_phase, cudaStream_t s);

// Per-lattice state I/O (d points at the lattice's device descriptor).
// pull: 1 for CS (stored phase shifted by the lattice vectors), 0 for FD.
cudaError_t launch_init_equilibrium(int precision, int q1, int pull, const LatDesc* d, int nx, int ny,
                                    const double* rho, const double* ux, const double* uy, cudaStream_t s);
cudaError_t launch_set_populations(int precision, int q1, int pull, const LatDesc* d, int nx, int ny,
                                   const double* f, cudaStream_t s);
// Readout of the canonical state over the window [x0, x0+wx) x [y0, y0+wy)
// (periodic; the whole lattice is x0 = y0 = 0, wx = nx, wy = ny): any of
// f [K][wy][wx], rho/ux/uy [wy][wx] may be null; if part != null, block
// partial sums of the observables are written to part[nblocks][NOBS] and
// reduced into d->snap.
cudaError_t launch_readout(int precision, int q1, int pull, const LatDesc* d, int nx, int ny, int x0, int y0, int wx,
                           int wy, double* f, double* rho, double* ux, double* uy, double* part, int nblocks,
                           cudaStream_t s);

}  // namespace lbm
