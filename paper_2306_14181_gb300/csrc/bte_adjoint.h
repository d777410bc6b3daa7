// Adjoint-step interface (kernels in bte_adjoint.cu, driver in bte_api.cu).
#pragma once

#include "bte_internal.h"
#include "bte_tiled.h"

namespace bte {

struct AdjArgs {
    const float *lam_in;  // lambda^{n+1} [nb*nd][ncell]
    float *lam_out;       // lambda^n
    const float *mu_in;   // mu^{n+1} [ncell]: sum_{k,d} lambda^{n+1} dt C_k / (W tau_k)
    float *pmu;           // [nb][ncell] per-band parts of mu^n
    float *pq;            // [nb][ncell] sum_d lambda^{n+1} (source gradient)
    float *pt;            // [nb][ncell] log-tau gradient terms of this step
    const float *w;       // [nd] direction weights
    float W;              // sum_d w_d
};

// The transposed step (reads a.e_in = e^n with its reference a.R, a.TL = T_L^n, a.ediff_in).
cudaError_t launch_adj_step(const StepArgs &a, const AdjArgs &g, int storage, int limiter, cudaStream_t s);
// lambda^N and the final state's log-tau terms (a.e_in = e^N, a.TL = T_L^N).
cudaError_t launch_adj_init(const StepArgs &a, const AdjArgs &g, int storage, const float *probe, cudaStream_t s);
// mu_out = sum_k pmu; gQ += amp sum_k dt C_k/(sum C W) pq; gtau[k] += sum_i pt[k][i] (FP64,
// fixed order; tau_part holds nb * adj_tau_blocks(ncell) doubles).
cudaError_t launch_adj_reduce(const StepArgs &a, const AdjArgs &g, float amp, float *mu_out, double *gQ,
                              double *tau_part, double *gtau, cudaStream_t s);
int adj_tau_blocks(long long ncell);

// Tiled adjoint (bte_adjoint_tiled*.cu): segment partials and their finalize.
struct AdjTFinal {
    const int *tile_seg0;  // [ntiles + 1] the tile's segment rows
    const int *seg_band;   // [G] band of each segment
    const float *Pm, *Pq;  // [G][tcells]
    const float *Ps;       // [G][2]
    const float *mu_in;    // mu^{n+1}
    const float *corr[3];  // wall corrections per axis [nb][4][lines]
    int G, tcells, ty, tz, nty;
};
// Wall pass along every non-periodic axis (two launches per axis; corr[ax]: nb * 4 * lines
// floats; scratch: adj_walls_scratch_floats(a) floats).
cudaError_t launch_adj_walls(const StepArgs &a, const AdjArgs &g, int storage, int limiter, float *lam_out,
                             float *const corr[3], float *scratch, cudaStream_t s);
long long adj_walls_scratch_floats(const StepArgs &a);
int adj_walls_max_dirs();  // directions the wall pass's combine phase holds in shared memory
// mu^n, dJ/dQ += amp q^n, dJ/dlog tau from the segment scalars (mt_part: ceil(ncell/256) doubles).
// The tiled adjoint step on the forward plan's tiles and schedule: lambda^n (interior and
// periodic faces), segment rows Pm, Pq ([G][tcells]) and Ps ([G][2]).
cudaError_t launch_adj_tiled(const StepArgs &a, const TiledPlan &plan, const float *lam_in, float *lam_out,
                             const float *mu_in, float *Pm, float *Pq, float *Ps, const float *w, int storage,
                             int limiter, cudaStream_t s);
cudaError_t launch_adj_tfinal(const StepArgs &a, const AdjTFinal &f, float amp, float *mu_out, double *gQ,
                              double *mt_part, double W, double *gtau, cudaStream_t s);

}  // namespace bte
