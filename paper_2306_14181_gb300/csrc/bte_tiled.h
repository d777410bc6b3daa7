// Shared-memory tiled forward kernel of the explicit DOM step: plan and launch interface.
#pragma once

#include <string>
#include <vector>

#include "bte_internal.h"

namespace bte {

// Device-side view of the plan, passed by value to the kernels.
struct TiledArgs {
    const int *unit_seg0;  // [U] first segment (row of P / PW) of each unit
    const int *tile_seg0;  // [ntiles + 1] segments of tile t are rows tile_seg0[t] .. tile_seg0[t+1]-1
    int U, J, np, ntiles;  // units, parts per tile, planes (nb*nd), tiles
    float *PW;             // diffuse-wall partials [G][nwd][tw]
    const float *hdr;      // per-plane constants [nb*nd][16] (see tiled_build_headers)
    const void *isorow;    // thermalizing-wall emission rows [6][nb][nx] (FP32 storage)
    int *err;              // bounded-wait failure flags (1: consumer, 2: producer)
    int tw;                // wall slots per wall per segment
    int nwd;               // number of diffuse walls
    int wslot[6];          // compact index of each diffuse wall, -1 for the others
    int nty, ntz;          // tiles along y and z
    int ns;                // shared-memory stages
    int stage0, stage_bytes, side_off, hdr_off, wall_off, bt_off, acc_off, rho_off;  // shared-memory layout (bytes)
    int ty, tz;            // tile extents (rows, slices)
    int tcells;            // cells of a full tile (row length of P)
    int chunk;             // rows per bulk copy of a box slice
    unsigned long long wait_ns;  // limit of a bounded mbarrier wait (ns)
    int stall;                   // failure-detection test: 1 the consumers', 2 the producer's first wait never completes
    int nxt;                     // row capacity of the kernel instance (tile arrays' row length, >= nx)
};

// Plane-synchronous schedule of the tiled forward kernel.  The plane list (k*nd + d) of every
// spatial tile is cut into J parts; unit u covers part u / ntiles of tile u % ntiles.  CTA c
// processes units c, c + nctas, c + 2 nctas, ... so in each round neighbouring tiles are
// worked on by neighbouring CTAs over the same planes, and the halo rows one CTA loads are
// still in L2 when its neighbour needs them.  J = nctas / gcd(ntiles, nctas) makes the unit
// count a multiple of the CTA count.  A segment is the run of one unit within one band; it
// writes one row of moment partials P[seg][tile cells] and one row of diffuse-wall partials.
// Segments are numbered tile by tile (parts in order, bands in order within a part), so a
// tile's partials are one contiguous run of rows, summed in that order by the finalize.
struct TiledPlan {
    int valid = 0;
    int dim = 0, vx = 0;
    int G = 0, nctas = 0;
    int nty = 0, ntz = 0, ntiles = 0, tcells = 0, tw = 0;
    int ns = 0, stage0 = 0, stage_bytes = 0, side_off = 0, hdr_off = 0, wall_off = 0, bt_off = 0, acc_off = 0;
    int rho_off = 0, smem = 0;
    int ty = 0, tz = 0, threads = 0;
    int nwd = 0, wslot[6] = {-1, -1, -1, -1, -1, -1};
    void *kernel = nullptr;
    int U = 0, J = 0, np = 0;
    std::vector<int> h_unit_seg0;
    int *unit_seg0 = nullptr;
    int *seg_band = nullptr;  // [G] band of each segment row
    float *PW = nullptr;
    float *hdr = nullptr;
    void *isorow = nullptr;
    int storage = 0, nx = 0, chunk = 4;  // nx: the instance's row capacity NX (>= the grid's nx)
    int *err = nullptr;
    unsigned long long wait_ns = 2000000000ull;  // bounded-wait limit (bte_set_wait_limit)
    int stall = 0;                               // one-shot stall test of the next launch (bte_set_wait_limit)
};

// Shape check, tile geometry and the schedule (queries the current device for its SM count
// and the kernel's occupancy).  false + reason if the grid cannot be tiled.
bool tiled_plan(int dim, const int n[3], int nb, int nd, int storage, int limiter, bool sr, const int bc[6],
                TiledPlan &plan, std::string &why);
// Device copies of the schedule tables, the wall partials and the error flag, and the per-plane
// constant records the producer copies into each stage (built from the step tables in a).
bool tiled_setup(TiledPlan &plan, const StepArgs &a, std::string &why);
void tiled_free(TiledPlan &plan);
TiledArgs tiled_device_args(const TiledPlan &plan);
cudaError_t launch_step_tiled(const StepArgs &a, const TiledPlan &plan, cudaStream_t s);
cudaError_t launch_finalize_tiled(const StepArgs &a, const TiledPlan &plan, int storage, float *TL_out,
                                  cudaStream_t s);

}  // namespace bte
