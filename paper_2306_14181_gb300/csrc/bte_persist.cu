// Persistent forward step for small 1-D problems (the cross-plane film of Sec. 3.6): the whole
// FP32 state lives in the shared memory of one thread-block cluster for all the steps of one
// bte_step call, so a step costs block barriers and one cluster barrier instead of launches.  Each step follows
// Eq. (disretized_transientBTE) with the limited face value of Sec. 4.1 and the wall ghosts of
// Sec. 2.2 (periodic wrap, thermalizing emission, diffuse value Eq. diff_bound, specular
// mirror), then forms T_L of Eq. (BTE_get_e0) from the new state.  At the end the state, T_L
// and the diffuse-wall values are written back, so the context continues as after bte_step.
#include <cooperative_groups.h>

#include "bte_device.cuh"

namespace bte {

// Value of plane (band lb of this CTA, global band kg, direction d) at position p of the 1-D
// line (p in [-2, n+1]); eps: the CTA's state [nbl*nd][n]; ed: its diffuse-wall values [2][nbl].
__device__ __forceinline__ float p1_ext(const StepArgs &a, const float *eps, const float *ed, int lb, int kg, int d,
                                       int p, float nu, int nbl) {
    const int n = a.n[0];
    const float *row = eps + (lb * a.nd + d) * n;
    if (p >= 0 && p < n) return row[p];
    const int side = p < 0 ? 0 : 1;
    const int bc = a.bc[side];
    if (bc == kBcPeriodic) return row[side ? p - n : p + n];
    if (bc == kBcSpecular) {
        const int layer = side ? p - n + 1 : -p;
        return eps[(lb * a.nd + a.mirror[d]) * n + (side ? n - layer : layer - 1)];
    }
    const bool incoming = side == 0 ? nu > 0.f : nu < 0.f;
    if (!incoming) return row[side ? n - 1 : 0];
    if (bc == kBcIsothermal) return a.iso[side * a.nb + kg];
    return ed[side * nbl + lb];
}

// Persistent kernel: a thread-block cluster of C CTAs, CTA r owning bands r, r + C, ...; each
// holds its bands' state in shared memory for all the steps.  Per step a CTA updates its planes,
// forms its bands' share of the T_L numerator per cell (fixed plane order) in a double-buffered
// shared array, the cluster synchronises once, and every CTA adds the C shares in rank order
// from distributed shared memory.  C = 1 is the single-CTA case.
template <int LIM>
__global__ void __launch_bounds__(1024, 1) k_persist_1d(const StepArgs a, int nsteps, const float *amps, float *e_io,
                                                        float *tl_out, float *ediff_out) {
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    const int C = (int)cl.num_blocks(), rank = (int)cl.block_rank();
    extern __shared__ __align__(16) float sm[];
    const int n = a.n[0], nd = a.nd;
    const int nbl = (a.nb - rank + C - 1) / C;  // bands of this CTA: rank, rank + C, ...
    const int npl = nbl * nd, nel = npl * n;
    float *e0 = sm, *e1 = sm + nel, *tl = e1 + nel;
    float *part = tl + n;  // [2][n] this CTA's share of the T_L numerator, read by the cluster
    float *ed = part + 2 * n;  // [2][nbl] diffuse-wall values of this CTA's bands
    float *pnu = ed + 2 * nbl, *pwm = pnu + npl, *pdt = pwm + npl, *pck = pdt + npl, *psr = pck + npl;
    // local plane lp = lb * nd + d is global plane (rank + lb C) nd + d
    auto gplane = [&](int lp) { return (rank + (lp / nd) * C) * nd + lp % nd; };
    for (int j = threadIdx.x; j < nel; j += blockDim.x) e0[j] = e_io[(long long)gplane(j / n) * n + j % n];
    for (int lp = threadIdx.x; lp < npl; lp += blockDim.x) {
        const int pl = gplane(lp);
        const BandConst b = a.band[pl / nd];
        pnu[lp] = a.nu[3 * pl];
        pwm[lp] = a.wmom[pl];
        pdt[lp] = b.dtinv;
        pck[lp] = b.ck;
        psr[lp] = b.srck;
    }
    __syncthreads();
    // this CTA's diffuse-wall values and share of the T_L numerator, from the state es
    auto walls_and_share = [&](const float *es, float *pt) {
        for (int j = threadIdx.x; j < 2 * nbl; j += blockDim.x) {
            const int side = j / nbl, lb = j % nbl;
            float v = 0.f;
            if (a.bc[side] == kBcDiffuse) {
                const int x = side ? n - 1 : 0;
                for (int d = 0; d < nd; ++d) v = fmaf(a.wdiff[side * nd + d], es[(lb * nd + d) * n + x], v);
                v *= a.inv_den[side];
            }
            ed[j] = v;
        }
        for (int x = threadIdx.x; x < n; x += blockDim.x) {
            float v = 0.f;
            for (int lp = 0; lp < npl; ++lp) v = fmaf(pwm[lp], es[lp * n + x], v);
            pt[x] = v;
        }
    };
    auto gather_tl = [&](int buf) {
        for (int x = threadIdx.x; x < n; x += blockDim.x) {
            float v = 0.f;
            for (int r = 0; r < C; ++r) v += cl.map_shared_rank(part + buf * n, r)[x];
            tl[x] = v * a.invD;
        }
    };
    int buf = 0;
    walls_and_share(e0, part + buf * n);
    cl.sync();
    gather_tl(buf);
    __syncthreads();
    const int bx = blockDim.x % n, bp = blockDim.x / n;
    const int x00 = threadIdx.x % n, p00 = threadIdx.x / n;
    for (int s = 0; s < nsteps; ++s) {
        const float amp = amps[s];
        int x = x00, lp = p00;
        for (int j = threadIdx.x; j < nel; j += blockDim.x) {
            const int lb = lp / nd, d = lp - lb * nd;
            const float nu = pnu[lp];
            const float u0 = e0[j];
            float div = 0.f;
            if (nu != 0.f) {
                const int sg = nu > 0.f ? 1 : -1;
                // interior cells read the row directly; the two cells next to each wall use the
                // ghost rules (the mirrored direction is in the same band, so in this CTA)
                float um2, um1, up1;
                if (x >= 2 && x + 2 < n) {
                    um2 = e0[j - 2 * sg];
                    um1 = e0[j - sg];
                    up1 = e0[j + sg];
                } else {
                    const int kg = rank + lb * C;
                    um2 = p1_ext(a, e0, ed, lb, kg, d, x - 2 * sg, nu, nbl);
                    um1 = p1_ext(a, e0, ed, lb, kg, d, x - sg, nu, nbl);
                    up1 = p1_ext(a, e0, ed, lb, kg, d, x + sg, nu, nbl);
                }
                const float fo = u0 + 0.5f * limit<LIM>(u0 - um1, up1 - u0);
                const float fi = um1 + 0.5f * limit<LIM>(um1 - um2, u0 - um1);
                div = fabsf(nu) * (fo - fi);
            }
            const float src = a.Q ? psr[lp] * (amp * a.Q[x]) : 0.f;
            e1[j] = u0 - div + pdt[lp] * (pck[lp] * tl[x] - u0) + src;
            x += bx;
            lp += bp;
            if (x >= n) {
                x -= n;
                ++lp;
            }
        }
        __syncthreads();
        buf ^= 1;
        walls_and_share(e1, part + buf * n);
        cl.sync();  // every CTA's share of this step is written; the previous buffer is free
        gather_tl(buf);
        __syncthreads();
        float *t = e0;
        e0 = e1;
        e1 = t;
    }
    for (int j = threadIdx.x; j < nel; j += blockDim.x) e_io[(long long)gplane(j / n) * n + j % n] = e0[j];
    if (rank == 0)
        for (int x = threadIdx.x; x < n; x += blockDim.x) tl_out[x] = tl[x];
    // the diffuse-wall values in the layout the other kernels read: [wall][k][wall cell 0]
    for (int j = threadIdx.x; j < 2 * nbl; j += blockDim.x) {
        const int side = j / nbl, lb = j % nbl;
        ediff_out[(long long)(side * a.nb + rank + lb * C) * a.wc_max] = ed[j];
    }
    cl.sync();  // no CTA leaves while another may still read its shared memory
}

static size_t persist_smem(const StepArgs &a, int C) {
    const size_t nbl = (a.nb + C - 1) / C, npl = nbl * a.nd;
    return (2 * npl * a.n[0] + 3 * (size_t)a.n[0] + 2 * nbl + 5 * npl) * sizeof(float);
}

size_t persist_1d_smem(const StepArgs &a) { return persist_smem(a, 1); }

cudaError_t launch_persist_1d(const StepArgs &a, int limiter, int nsteps, const float *amps, float *e_io,
                              float *tl_out, float *ediff_out, cudaStream_t s) {
    void (*k)(const StepArgs, int, const float *, float *, float *, float *) =
        limiter == kLimFirst ? k_persist_1d<kLimFirst> : limiter == kLimMinmod ? k_persist_1d<kLimMinmod>
                                                                                : k_persist_1d<kLimVanAlbada>;
    // the largest cluster (<= 16, <= nb) the device can place; one CTA if none
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) cudaGetLastError();
    for (int C = a.nb < 16 ? a.nb : 16; C >= 1; --C) {
        const size_t smem = persist_smem(a, C);
        if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)C);
        cfg.blockDim = dim3(1024);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = s;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = (unsigned)C;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int ncl = 0;
        if (cudaOccupancyMaxActiveClusters(&ncl, k, &cfg) != cudaSuccess || ncl < 1) {
            cudaGetLastError();
            continue;
        }
        return cudaLaunchKernelEx(&cfg, k, a, nsteps, amps, e_io, tl_out, ediff_out);
    }
    return cudaErrorInvalidConfiguration;
}

}  // namespace bte
