// Shared-memory tiled forward kernel of the explicit DOM step: plan and launch interface.
#pragma once

#include <string>

#include "bte_internal.h"

namespace bte {

// Static, balanced schedule of the tiled forward kernel.  Work is the ordered list of
// (spatial tile, band, direction) plane-tiles, tile-major; CTA b processes the contiguous
// range [begin[b], begin[b+1]).  A "segment" is a run of one CTA's range with one tile and one
// band; each segment writes one moment partial row P[seg][tile cells] and, for diffuse walls,
// one wall partial row.  The finalize pass sums, per tile, its segments in order.
struct TiledPlan {
    int valid = 0;
    int G = 0;                  // number of segments (rows of P)
    int nctas = 0;
    int tx = 0, ty = 0, tz = 0; // tile extents (cells)
    int ntiles = 0;
    // device arrays
    int *cta_begin = nullptr;   // [nctas + 1] first plane-tile of each CTA
    int *tile_seg0 = nullptr;   // [ntiles + 1] first segment of each tile
    int *seg_band = nullptr;    // [G] band of each segment
    float *PW = nullptr;        // diffuse-wall partials [G][wall slots of the tile]
    void *maps = nullptr;       // TMA descriptors (two state buffers)
};

bool tiled_plan(int dim, const int n[3], int nb, int nd, int storage, const int bc[6], TiledPlan &plan,
                std::string &why);
bool tiled_setup(TiledPlan &plan, void *e0, void *e1, size_t elem_bytes, std::string &why);
void tiled_free(TiledPlan &plan);
cudaError_t launch_step_tiled(const StepArgs &a, const TiledPlan &plan, int cur, int storage, int limiter,
                              cudaStream_t s);
cudaError_t launch_finalize_tiled(const StepArgs &a, const TiledPlan &plan, float *TL_out, cudaStream_t s);

}  // namespace bte
