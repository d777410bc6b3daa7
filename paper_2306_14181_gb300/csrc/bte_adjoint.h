// Adjoint-step interface (kernels in bte_adjoint.cu, driver in bte_api.cu).
#pragma once

#include "bte_internal.h"

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

}  // namespace bte
