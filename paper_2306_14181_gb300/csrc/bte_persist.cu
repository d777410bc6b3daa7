// Persistent single-CTA forward step for small 1-D problems (the cross-plane film of Sec. 3.6):
// the whole FP32 state lives in shared memory for all the steps of one bte_step call, so a
// step costs two block barriers instead of two kernel launches.  Each step follows
// Eq. (disretized_transientBTE) with the limited face value of Sec. 4.1 and the wall ghosts of
// Sec. 2.2 (periodic wrap, thermalizing emission, diffuse value Eq. diff_bound, specular
// mirror), then forms T_L of Eq. (BTE_get_e0) from the new state.  At the end the state, T_L
// and the diffuse-wall values are written back, so the context continues as after bte_step.
#include "bte_device.cuh"

namespace bte {

// Value of plane (k, d) at position p of the 1-D line (p in [-2, n+1]); eps: the state in
// shared memory [nb*nd][n]; ed: the diffuse-wall values [2][nb] of the same state.
__device__ __forceinline__ float p1_ext(const StepArgs &a, const float *eps, const float *ed, int k, int d, int p,
                                       float nu) {
    const int n = a.n[0];
    const float *row = eps + (long long)(k * a.nd + d) * n;
    if (p >= 0 && p < n) return row[p];
    const int side = p < 0 ? 0 : 1;
    const int bc = a.bc[side];
    if (bc == kBcPeriodic) return row[side ? p - n : p + n];
    if (bc == kBcSpecular) {
        const int layer = side ? p - n + 1 : -p;
        return eps[(long long)(k * a.nd + a.mirror[d]) * n + (side ? n - layer : layer - 1)];
    }
    const bool incoming = side == 0 ? nu > 0.f : nu < 0.f;
    if (!incoming) return row[side ? n - 1 : 0];
    if (bc == kBcIsothermal) return a.iso[side * a.nb + k];
    return ed[side * a.nb + k];
}

// Diffuse-wall values of the state eps: e_diff[wall][k] = sum_{leaving} w (s.n) e / sum_in w|s.n|.
__device__ __forceinline__ void p1_ediff(const StepArgs &a, const float *eps, float *ed) {
    const int n = a.n[0];
    for (int j = threadIdx.x; j < 2 * a.nb; j += blockDim.x) {
        const int side = j / a.nb, k = j % a.nb;
        float s = 0.f;
        if (a.bc[side] == kBcDiffuse) {
            const int x = side ? n - 1 : 0;
            for (int d = 0; d < a.nd; ++d) s = fmaf(a.wdiff[side * a.nd + d], eps[(long long)(k * a.nd + d) * n + x], s);
            s *= a.inv_den[side];
        }
        ed[j] = s;
    }
}

// T_L of every cell from the state eps: kTlParts threads per cell sum every kTlParts-th plane
// (w_d / tau_k from shared memory), then the parts are added in order.
constexpr int kTlParts = 8;
__device__ __forceinline__ void p1_tl(const StepArgs &a, const float *eps, const float *wm, float *part, float *tl) {
    const int n = a.n[0], np = a.nb * a.nd;
    for (int t = threadIdx.x; t < n * kTlParts; t += blockDim.x) {
        const int x = t / kTlParts, r = t - x * kTlParts;
        float s = 0.f;
        for (int pl = r; pl < np; pl += kTlParts) s = fmaf(wm[pl], eps[pl * n + x], s);
        part[t] = s;
    }
    __syncthreads();
    for (int x = threadIdx.x; x < n; x += blockDim.x) {
        float s = 0.f;
        #pragma unroll
        for (int r = 0; r < kTlParts; ++r) s += part[x * kTlParts + r];
        tl[x] = s * a.invD;
    }
}

template <int LIM>
__global__ void __launch_bounds__(1024, 1) k_persist_1d(const StepArgs a, int nsteps, const float *amps, float *e_io,
                                                        float *tl_out, float *ediff_out) {
    extern __shared__ __align__(16) float sm[];
    const int n = a.n[0], np = a.nb * a.nd;
    const int nel = np * n;
    float *e0 = sm, *e1 = sm + nel, *tl = e1 + nel, *ed = tl + n;
    // per-plane constants: nu, w/tau, dt/tau, C/W, dt C/(sum C W); T_L parts
    float *pnu = ed + 2 * a.nb, *pwm = pnu + np, *pdt = pwm + np, *pck = pdt + np, *psr = pck + np;
    float *part = psr + np;
    for (int j = threadIdx.x; j < nel; j += blockDim.x) e0[j] = e_io[j];
    for (int pl = threadIdx.x; pl < np; pl += blockDim.x) {
        const BandConst b = a.band[pl / a.nd];
        pnu[pl] = a.nu[3 * pl];
        pwm[pl] = a.wmom[pl];
        pdt[pl] = b.dtinv;
        pck[pl] = b.ck;
        psr[pl] = b.srck;
    }
    __syncthreads();
    p1_tl(a, e0, pwm, part, tl);
    p1_ediff(a, e0, ed);
    __syncthreads();
    // this thread's first element (x, plane) and the stride in both
    const int bx = blockDim.x % n, bp = blockDim.x / n;
    const int x00 = threadIdx.x % n, p00 = threadIdx.x / n;
    for (int s = 0; s < nsteps; ++s) {
        const float amp = amps[s];
        int x = x00, plane = p00;
        for (int j = threadIdx.x; j < nel; j += blockDim.x) {
            const int k = plane / a.nd, d = plane - k * a.nd;
            const float nu = pnu[plane];
            const float u0 = e0[j];
            float div = 0.f;
            if (nu != 0.f) {
                const int sg = nu > 0.f ? 1 : -1;
                // interior cells read the row directly; the two cells next to each wall use the
                // ghost rules
                float um2, um1, up1;
                if (x >= 2 && x + 2 < n) {
                    um2 = e0[j - 2 * sg];
                    um1 = e0[j - sg];
                    up1 = e0[j + sg];
                } else {
                    um2 = p1_ext(a, e0, ed, k, d, x - 2 * sg, nu);
                    um1 = p1_ext(a, e0, ed, k, d, x - sg, nu);
                    up1 = p1_ext(a, e0, ed, k, d, x + sg, nu);
                }
                const float fo = u0 + 0.5f * limit<LIM>(u0 - um1, up1 - u0);
                const float fi = um1 + 0.5f * limit<LIM>(um1 - um2, u0 - um1);
                div = fabsf(nu) * (fo - fi);
            }
            const float src = a.Q ? psr[plane] * (amp * a.Q[x]) : 0.f;
            e1[j] = u0 - div + pdt[plane] * (pck[plane] * tl[x] - u0) + src;
            x += bx;
            plane += bp;
            if (x >= n) {
                x -= n;
                ++plane;
            }
        }
        __syncthreads();
        p1_tl(a, e1, pwm, part, tl);
        p1_ediff(a, e1, ed);
        __syncthreads();
        float *t = e0;
        e0 = e1;
        e1 = t;
    }
    for (int j = threadIdx.x; j < nel; j += blockDim.x) e_io[j] = e0[j];
    for (int x = threadIdx.x; x < n; x += blockDim.x) tl_out[x] = tl[x];
    // the diffuse-wall values in the layout the other kernels read: [wall][k][wall cell 0]
    for (int j = threadIdx.x; j < 2 * a.nb; j += blockDim.x) ediff_out[(long long)j * a.wc_max] = ed[j];
}

size_t persist_1d_smem(const StepArgs &a) {
    const size_t np = (size_t)a.nb * a.nd;
    return (2 * np * a.n[0] + a.n[0] + 2 * a.nb + 5 * np + (size_t)kTlParts * a.n[0]) * sizeof(float);
}

cudaError_t launch_persist_1d(const StepArgs &a, int limiter, int nsteps, const float *amps, float *e_io,
                              float *tl_out, float *ediff_out, cudaStream_t s) {
    const size_t smem = persist_1d_smem(a);
    void (*k)(const StepArgs, int, const float *, float *, float *, float *) =
        limiter == kLimFirst ? k_persist_1d<kLimFirst> : limiter == kLimMinmod ? k_persist_1d<kLimMinmod>
                                                                                : k_persist_1d<kLimVanAlbada>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<1, 1024, smem, s>>>(a, nsteps, amps, e_io, tl_out, ediff_out);
    return cudaGetLastError();
}

}  // namespace bte
