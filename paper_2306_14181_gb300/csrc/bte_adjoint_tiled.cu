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
    // accumulators of mu and of the source gradient and the block reduction; in 3-D the z-face
    // terms passed between slices and the plane-tile's box of e and lambda; with 16-bit storage
    // the unit's reference box, and mu and T_L of the tile, each where it still fits
    const size_t box = (size_t)(plan.ty + 4) * (plan.dim == 3 ? plan.tz + 4 : 1) * plan.nx;
    const size_t limit = (size_t)227 * 1024 / sizeof(float);
    size_t nf = (size_t)2 * plan.tcells + 2 * ncw + (plan.dim == 3 ? (size_t)2 * plan.tcells + 2 * box : 0);
    const bool cache_r = storage != kStoreF32 && (plan.dim == 2 || nf + box <= limit);
    if (cache_r) nf += box;
    const bool cache_mt = nf + (size_t)2 * plan.tcells <= limit;
    if (cache_mt) nf += (size_t)2 * plan.tcells;
    const size_t smem = nf * sizeof(float);
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
    g.cache_r = cache_r ? 1 : 0;
    g.cache_mt = cache_mt ? 1 : 0;
    k<<<plan.nctas, ncw * 32, smem, s>>>(a, tiled_device_args(plan), g);
    return cudaGetLastError();
}

}  // namespace bte
