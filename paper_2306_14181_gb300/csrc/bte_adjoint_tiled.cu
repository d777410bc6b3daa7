// Launch of the tiled adjoint kernel (device code in bte_adjoint_tiled.cuh).
#include "bte_adjoint_tiled.cuh"

namespace bte {

using namespace tiled;

cudaError_t launch_adj_tiled(const StepArgs &a, const TiledPlan &plan, const float *lam_in, float *lam_out,
                             const float *mu_in, float *Pm, float *Pq, float *Ps, const float *w, int storage,
                             int limiter, cudaStream_t s) {
    AdjKernel k = storage == kStoreF32 ? adj_pick_f32(limiter, plan.nx, plan.dim)
                  : storage == kStoreF16 ? adj_pick_f16(limiter, plan.nx, plan.dim)
                                         : adj_pick_bf16(limiter, plan.nx, plan.dim);
    if (!k) return cudaErrorInvalidConfiguration;
    const int ncw = plan.dim == 2 ? Geo<2, 1>::NCW : Geo<3, 1>::NCW;
    // accumulators of mu and of the source gradient, the block reduction, and in 3-D the z-face
    // terms passed between slices (two plane-tile parities of A and C)
    const size_t smem = (size_t)(plan.dim == 3 ? 6 : 2) * plan.tcells * sizeof(float) + 2 * ncw * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    AdjTiledArgs g;
    g.lam_in = lam_in;
    g.lam_out = lam_out;
    g.mu_in = mu_in;
    g.Pm = Pm;
    g.Pq = Pq;
    g.Ps = Ps;
    g.w = w;
    k<<<plan.nctas, ncw * 32, smem, s>>>(a, tiled_device_args(plan), g);
    return cudaGetLastError();
}

}  // namespace bte
