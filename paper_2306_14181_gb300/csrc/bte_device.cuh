// Device helpers shared by the generic forward kernels (bte_kernels.cu) and the adjoint
// kernels (bte_adjoint.cu): storage codecs, limiters, ghost values of Sec. 2.2.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "bte_internal.h"

namespace bte {

// ------------------------------------------------------------------------------------------
// Storage codecs.  FP32 storage keeps e itself.  16-bit storage keeps, per (k, d, cell i),
//   h = round(e / s_k - rho_i),   s_k = C_k T_scale / W,   rho_i = R_i / T_scale,
// where R is the reference temperature field of the state (the T_L the step that wrote it
// relaxed towards).  s_k rho_i = C_k R_i / W is band k's equilibrium at R_i, so h holds only
// the departure from the local equilibrium and the 16-bit rounding error scales with that
// departure instead of with e: e = s_k (h + rho_i).  All arithmetic is FP32.
// st() stores the rounded code and returns the value it represents, so that the moment and
// the diffuse-wall sums use the stored state.
// ------------------------------------------------------------------------------------------
template <int S> struct Codec;
template <> struct Codec<kStoreF32> {
    using T = float;
    static constexpr bool kRef = false;
    static __device__ __forceinline__ float ld(const T *p, long long i, const BandConst &, float) { return p[i]; }
    static __device__ __forceinline__ double ld64(const T *p, long long i, const BandConst &, float) {
        return (double)p[i];
    }
    static __device__ __forceinline__ float st(T *p, long long i, float v, const BandConst &, float) {
        p[i] = v;
        return v;
    }
    static __device__ __forceinline__ float st_sr(T *p, long long i, float v, const BandConst &, float, uint32_t) {
        p[i] = v;
        return v;
    }
};
template <> struct Codec<kStoreF16> {
    using T = __half;
    static constexpr bool kRef = true;
    static __device__ __forceinline__ float ld(const T *p, long long i, const BandConst &b, float rho) {
        return b.scale * (__half2float(p[i]) + rho);
    }
    static __device__ __forceinline__ double ld64(const T *p, long long i, const BandConst &b, float rho) {
        return (double)b.scale * ((double)__half2float(p[i]) + (double)rho);
    }
    static __device__ __forceinline__ float st(T *p, long long i, float v, const BandConst &b, float rho) {
        const __half h = __float2half_rn(fmaf(v, b.inv_scale, -rho));
        p[i] = h;
        return b.scale * (__half2float(h) + rho);
    }
    // stochastic rounding: 13 random bits added below binary16's 10 fraction bits, then
    // truncated (exact for normal binary16 values; round to nearest in the subnormal range)
    static __device__ __forceinline__ float st_sr(T *p, long long i, float v, const BandConst &b, float rho,
                                                  uint32_t bits) {
        const uint32_t u = __float_as_uint(fmaf(v, b.inv_scale, -rho)) + (bits >> 19);
        const __half h = __float2half_rn(__uint_as_float(u & 0xffffe000u));
        p[i] = h;
        return b.scale * (__half2float(h) + rho);
    }
};
template <> struct Codec<kStoreBF16> {
    using T = __nv_bfloat16;
    static constexpr bool kRef = true;
    static __device__ __forceinline__ float ld(const T *p, long long i, const BandConst &b, float rho) {
        return b.scale * (__bfloat162float(p[i]) + rho);
    }
    static __device__ __forceinline__ double ld64(const T *p, long long i, const BandConst &b, float rho) {
        return (double)b.scale * ((double)__bfloat162float(p[i]) + (double)rho);
    }
    static __device__ __forceinline__ float st(T *p, long long i, float v, const BandConst &b, float rho) {
        const __nv_bfloat16 h = __float2bfloat16_rn(fmaf(v, b.inv_scale, -rho));
        p[i] = h;
        return b.scale * (__bfloat162float(h) + rho);
    }
    // stochastic rounding: 16 random bits added below bfloat16's 7 fraction bits, then truncated
    static __device__ __forceinline__ float st_sr(T *p, long long i, float v, const BandConst &b, float rho,
                                                  uint32_t bits) {
        const uint32_t u = __float_as_uint(fmaf(v, b.inv_scale, -rho)) + (bits >> 16);
        const __nv_bfloat16 h = __ushort_as_bfloat16((unsigned short)(u >> 16));
        p[i] = h;
        return b.scale * (__bfloat162float(h) + rho);
    }
};

// Scaled code reference rho_j = R_j / T_scale of cell j (0 for FP32 storage, R untouched).
template <class Cd>
__device__ __forceinline__ float rho_at(const float *R, float invTs, long long j) {
    if constexpr (Cd::kRef) return R[j] * invTs;
    else return 0.f;
}

// Slope limiter of the one-sided differences a (upwind) and b (downwind); e_face = e_m + L/2.
template <int LIM> __device__ __forceinline__ float limit(float a, float b);
template <> __device__ __forceinline__ float limit<kLimFirst>(float, float) { return 0.f; }
template <> __device__ __forceinline__ float limit<kLimMinmod>(float a, float b) {
    return (a * b > 0.f) ? (fabsf(a) < fabsf(b) ? a : b) : 0.f;
}
template <> __device__ __forceinline__ float limit<kLimVanAlbada>(float a, float b) {
    const float ab = a * b;
    return ab > 0.f ? ab * (a + b) / (a * a + b * b) : 0.f;
}

__device__ __forceinline__ double limit64(int lim, double a, double b) {
    if (lim == kLimFirst || a * b <= 0.0) return 0.0;
    if (lim == kLimMinmod) return fabs(a) < fabs(b) ? a : b;
    return a * b * (a + b) / (a * a + b * b);
}

// Index of a wall-adjacent cell within its wall (the two coordinates along the wall).
__device__ __forceinline__ int wall_cell(const StepArgs &a, int ax, const int c[3]) {
    return ax == 0 ? c[2] * a.n[1] + c[1] : (ax == 1 ? c[2] * a.n[0] + c[0] : c[1] * a.n[0] + c[0]);
}

__device__ __forceinline__ void cell_coords(const StepArgs &a, long long i, int c[3]) {
    c[0] = (int)(i % a.n[0]);
    c[1] = (int)((i / a.n[0]) % a.n[1]);
    c[2] = (int)(i / ((long long)a.n[0] * a.n[1]));
}

// Value of plane (k,d) at position pos along axis ax through cell i (coords c), where pos may
// be a ghost (-2, -1, n, n+1).  Ghosts follow Sec. 2.2: periodic wrap; thermalizing wall
// emission C_k T_w / W for incoming directions; diffuse wall value e_diff for incoming
// directions; the wall cell itself for directions leaving through a thermalizing or diffuse
// wall; the mirrored direction at the mirrored cell for a specular wall; periodic ghosts carry
// the pair's temperature jump (+C_k dT / W on the -a side, minus it on the +a side).
template <class Cd>
__device__ __forceinline__ float ext_value(const StepArgs &a, const typename Cd::T *e, const BandConst &b, int k,
                                           int d, long long base, long long i, const int c[3], int ax, int pos,
                                           float nu) {
    const int n = a.n[ax];
    const long long st = a.stride[ax];
    if (pos >= 0 && pos < n) {
        const long long j = i + (long long)(pos - c[ax]) * st;
        return Cd::ld(e, base + j, b, rho_at<Cd>(a.R, a.invTs, j));
    }
    const int side = pos < 0 ? 0 : 1;
    const int wall = 2 * ax + side;
    const int bc = a.bc[wall];
    if (bc == kBcPeriodic) {
        // Sec. 2.2 (iv): the wrapped value, shifted by the pair's temperature difference
        const long long j = i + (long long)((side ? pos - n : pos + n) - c[ax]) * st;
        const float off = a.jmp[ax * a.nb + k];
        return Cd::ld(e, base + j, b, rho_at<Cd>(a.R, a.invTs, j)) + (side ? -off : off);
    }
    if (bc == kBcSpecular) {
        const int layer = side ? pos - n + 1 : -pos;
        const long long j = i + (long long)((side ? n - layer : layer - 1) - c[ax]) * st;
        const long long mbase = ((long long)k * a.nd + a.mirror[ax * a.nd + d]) * a.ncell;
        return Cd::ld(e, mbase + j, b, rho_at<Cd>(a.R, a.invTs, j));
    }
    const bool incoming = side == 0 ? (nu > 0.f) : (nu < 0.f);
    const long long jw = i + (long long)((side ? n - 1 : 0) - c[ax]) * st;  // the wall cell
    if (!incoming) return Cd::ld(e, base + jw, b, rho_at<Cd>(a.R, a.invTs, jw));
    if (bc == kBcIsothermal) return a.iso[wall * a.nb + k];
    return Cd::ld(static_cast<const typename Cd::T *>(a.ediff_in),
                  ((long long)wall * a.nb + k) * a.wc_max + wall_cell(a, ax, c), b, rho_at<Cd>(a.R, a.invTs, jw));
}

// Diffuse walls touched by cell c: their indices into wl[], count returned.
__device__ __forceinline__ int diffuse_walls_of(const StepArgs &a, const int c[3], int wl[6]) {
    int nw = 0;
    for (int w = 0; w < 2 * a.dim; ++w) {
        const int ax = w >> 1;
        if (a.bc[w] == kBcDiffuse && c[ax] == ((w & 1) ? a.n[ax] - 1 : 0)) wl[nw++] = w;
    }
    return nw;
}

}  // namespace bte
