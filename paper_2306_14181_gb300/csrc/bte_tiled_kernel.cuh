// Device code of the tiled forward kernel (the design is described in bte_tiled.cu); included
// by the instantiation units bte_tiled_<storage>_<dim>d.cu so the instances compile in parallel.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "bte_tiled.h"

namespace bte {
namespace tiled {

constexpr unsigned long long kWaitLimitNs = 2000000000ull;  // 2 s: the drain limit, and the default of TiledArgs::wait_ns
constexpr int kStallOff = 96;   // byte offset of an mbarrier nothing arrives on (failure-detection test)
constexpr int kAbortOff = 112;  // byte offset of the CTA's abort word in shared memory (after <= 6 + 6 mbarriers)
constexpr int kHdrFloats = 16;                        // per-plane constants written by the producer

// Tile geometry: a lane holds VL consecutive cells of a row, WPR warps cover a row of
// nx = 32 VL WPR cells; NCW consumer warps stream KR rows each; 2-D tiles are TY rows, 3-D
// tiles TY rows by TZ slices.  2-D CTAs run 16 consumer warps of 4 rows (104 registers a
// thread after the split below), 3-D ones 12 warps of 4 rows (152; the z-stencil needs more
// live values).  Fewer, wider warps on 256-cell rows measured slower: 8 warps of 8 rows at 4
// cells a lane (224 registers) by 35%, and 8 warps of 4 rows at 8 cells a lane (142 registers;
// 40 instead of 50 instructions per update, but issue slots 40% busy instead of 61%, and twice
// the shared-memory bank conflicts from the 32-byte lane stride) by 23%: 9 resident warps
// cannot hide latency.
template <int DIM, int WPR> struct Geo;
// The producer is a warpgroup of its own (one working warp, three idle) so that registers can
// move between the two roles: at launch every thread gets 65536 / threads (rounded down to a
// multiple of 8); the producer warpgroup then gives back all but RP a thread and the consumer
// warpgroups take RC.  2-D: 640 threads x 96 = 61440 at launch, 16 x 32 x 104 + 4 x 32 x 56 =
// 60416 after; 3-D: 512 x 128 = 65536 at launch, 12 x 32 x 152 + 4 x 32 x 56 = 65536 after.
// Per SM sub-partition (warps w, w + 4, ...): 2-D 4 x 32 x 104 + 32 x 56 = 15104, 3-D 3 x 32 x
// 152 + 32 x 56 = 16384, within its 16384 registers.  (A 17th warp alone would cap every
// thread at 96 registers: five warps share one sub-partition.)
template <int WPR> struct Geo<2, WPR> {
    static constexpr int NCW = 16, KR = 4, TZ = 1, TY = NCW / WPR * KR;
    static constexpr int RC = 104, RP = 56;
};
template <> struct Geo<3, 1> {
    static constexpr int NCW = 12, KR = 4, TZ = 6, TY = NCW / TZ * KR;
    static constexpr int RC = 152, RP = 56;
};
constexpr int kProducerWarps = 4;  // one warpgroup
// Where a consumer keeps the moment partials of its cells for a segment: in registers in 3-D
// (152 a thread leave room for KR x VL more; measured 3 % faster on the laser block), in shared
// memory in 2-D (at 104 registers the 16 more live values cost 2 %).
template <int DIM> constexpr bool kAccRegs = DIM == 3;
template <int DIM, int WPR> constexpr int launch_regs() {
    return 65536 / ((Geo<DIM, WPR>::NCW + kProducerWarps) * 32) / 8 * 8;
}
static_assert(Geo<2, 2>::NCW % 4 == 0 && Geo<3, 1>::NCW % 4 == 0, "consumers fill whole warpgroups");
static_assert(Geo<2, 2>::NCW * 32 * Geo<2, 2>::RC + kProducerWarps * 32 * Geo<2, 2>::RP <=
                  (Geo<2, 2>::NCW + kProducerWarps) * 32 * launch_regs<2, 2>(), "2-D register split");
static_assert(Geo<3, 1>::NCW * 32 * Geo<3, 1>::RC + kProducerWarps * 32 * Geo<3, 1>::RP <=
                  (Geo<3, 1>::NCW + kProducerWarps) * 32 * launch_regs<3, 1>(), "3-D register split");
static_assert((Geo<2, 2>::NCW / 4) * 32 * Geo<2, 2>::RC + 32 * Geo<2, 2>::RP <= 16384 &&
                  (Geo<3, 1>::NCW / 4) * 32 * Geo<3, 1>::RC + 32 * Geo<3, 1>::RP <= 16384, "per sub-partition");

// Storage codecs.  FP32 storage keeps e.  16-bit storage keeps h = round(e / s_k - rho_i) with
// rho_i = R_i / T_scale the cell's code reference (the departure from band k's equilibrium at
// the reference temperature R_i, in units of s_k = C_k T_scale / W).  The 16-bit instances work
// in these scaled units throughout a plane: decoding is e / s_k = h + rho_i, and the updated
// value leaves the arithmetic already as the departure from the new reference, so encoding is
// the rounding alone.
template <int S> struct St;
template <> struct St<kStoreF32> {
    using T = float;
    using C = float;  // a code held in a register
    static constexpr bool kRef = false;
    static __device__ __forceinline__ float dec(T h, float) { return h; }
    static __device__ __forceinline__ float val(C c) { return c; }
    static __device__ __forceinline__ C bits(T h) { return h; }
    static __device__ __forceinline__ C enc(float v) { return v; }
    static __device__ __forceinline__ C enc_sr(float v, uint32_t) { return v; }
};
template <> struct St<kStoreF16> {
    using T = __half;
    using C = uint32_t;  // the code's 16 bits in the low half
    static constexpr bool kRef = true;
    static __device__ __forceinline__ float dec(T h, float rho) { return __half2float(h) + rho; }
    static __device__ __forceinline__ float val(C c) { return __half2float(__ushort_as_half((unsigned short)c)); }
    static __device__ __forceinline__ C bits(T h) { return __half_as_ushort(h); }
    static __device__ __forceinline__ C enc(float v) { return __half_as_ushort(__float2half_rn(v)); }
    // stochastic rounding: 13 random bits below binary16's 10 fraction bits, then truncation
    // (exact for normal binary16 values; round to nearest in the subnormal range)
    static __device__ __forceinline__ C enc_sr(float v, uint32_t bits) {
        return __half_as_ushort(__float2half_rn(__uint_as_float((__float_as_uint(v) + (bits >> 19)) & 0xffffe000u)));
    }
};
template <> struct St<kStoreBF16> {
    using T = __nv_bfloat16;
    using C = uint32_t;
    static constexpr bool kRef = true;
    static __device__ __forceinline__ float dec(T h, float rho) { return __bfloat162float(h) + rho; }
    static __device__ __forceinline__ float val(C c) { return __uint_as_float(c << 16); }
    static __device__ __forceinline__ C bits(T h) { return __bfloat16_as_ushort(h); }
    static __device__ __forceinline__ C enc(float v) { return __bfloat16_as_ushort(__float2bfloat16_rn(v)); }
    // stochastic rounding: 16 random bits below bfloat16's 7 fraction bits, then truncation
    static __device__ __forceinline__ C enc_sr(float v, uint32_t bits) { return (__float_as_uint(v) + (bits >> 16)) >> 16; }
};

// PTX approximate reciprocal (one MUFU operation, no special-case branches).
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Limiter.  Van Albada, L = max(ab, 0) (a + b) / (a^2 + b^2 + 1e-30): the approximate
// reciprocal of a denominator that is always a normal number, and no compare or select (pairs
// with ab <= 0 give a zero numerator; the 1e-30 changes L by a relative 1e-30 / (a^2 + b^2)).
// max(ab, 0) is taken as (ab + |ab|) / 2, an add on the FMA pipe instead of a min/max on the
// busier ALU pipe; the factors of 2 are exact, so the result is the same.
constexpr float kVaTiny = 1e-30f;
template <int LIM> __device__ __forceinline__ float lim(float a, float b);
template <> __device__ __forceinline__ float lim<kLimFirst>(float, float) { return 0.f; }
template <> __device__ __forceinline__ float lim<kLimMinmod>(float a, float b) {
    const float m = fabsf(a) < fabsf(b) ? a : b;
    return a * b > 0.f ? m : 0.f;
}
template <> __device__ __forceinline__ float lim<kLimVanAlbada>(float a, float b) {
    const float ab = a * b;
    return 0.5f * ((ab + fabsf(ab)) * (a + b)) * rcp_approx(fmaf(a, a, fmaf(b, b, kVaTiny)));
}
// face value e_m + L(e_m - e_l, e_r - e_m) / 2 at the upwind cell m
template <int LIM> __device__ __forceinline__ float face(float ul, float um, float ur) {
    return fmaf(0.5f, lim<LIM>(um - ul, ur - um), um);
}

// The same for two independent faces with the packed FP32x2 instructions of sm_100+ (each
// lane-pair operation rounds exactly like the scalar one).  a - b as one fused a + (-1) b,
// which rounds once, like a subtraction.
__device__ __forceinline__ float2 f2(float x) { return make_float2(x, x); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, f2(-1.f), a); }

template <int LIM> __device__ __forceinline__ float2 face2(float2 ul, float2 um, float2 ur);
template <> __device__ __forceinline__ float2 face2<kLimFirst>(float2, float2 um, float2) { return um; }
template <> __device__ __forceinline__ float2 face2<kLimMinmod>(float2 ul, float2 um, float2 ur) {
    const float2 a = sub2(um, ul), b = sub2(ur, um);
    const float2 L = make_float2(lim<kLimMinmod>(a.x, b.x), lim<kLimMinmod>(a.y, b.y));
    return __ffma2_rn(f2(0.5f), L, um);
}
template <> __device__ __forceinline__ float2 face2<kLimVanAlbada>(float2 ul, float2 um, float2 ur) {
    const float2 a = sub2(um, ul), b = sub2(ur, um);
    const float2 ab = __fmul2_rn(a, b);
    // (ab + |ab|) = 2 max(ab, 0), the 2 taken out by the final 1/4
    const float2 num = __fmul2_rn(make_float2(ab.x + fabsf(ab.x), ab.y + fabsf(ab.y)), __fadd2_rn(a, b));
    const float2 den = __ffma2_rn(a, a, __ffma2_rn(b, b, f2(kVaTiny)));
    const float2 L = __fmul2_rn(num, make_float2(rcp_approx(den.x), rcp_approx(den.y)));
    return __ffma2_rn(f2(0.25f), L, um);
}

// out[i] = face(ul[i], um[i], ur[i]) for i < N, two at a time
template <int LIM, int N>
__device__ __forceinline__ void faces(const float *ul, const float *um, const float *ur, float *out) {
    #pragma unroll
    for (int i = 0; i + 1 < N; i += 2) {
        const float2 f = face2<LIM>(make_float2(ul[i], ul[i + 1]), make_float2(um[i], um[i + 1]),
                                    make_float2(ur[i], ur[i + 1]));
        out[i] = f.x;
        out[i + 1] = f.y;
    }
    if constexpr (N & 1) out[N - 1] = face<LIM>(ul[N - 1], um[N - 1], ur[N - 1]);
}

// ---- PTX wrappers: mbarrier, bulk copy, timers ---------------------------------------------
__device__ __forceinline__ uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(su32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(su32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(su32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Wait for phase `parity` of the barrier, giving up after limit_ns nanoseconds: the error word
// gets `code` and false is returned.  The callers never leave the CTA's schedule on a false
// return (see the abort word below), so a give-up cannot strand another warp at a barrier.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, int *err, int code,
                                          unsigned long long limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = gtimer();
    while (!mbar_try_wait(bar, parity)) {
        if (gtimer() - t0 > limit_ns) {
            atomicOr(err, code);
            return false;
        }
    }
    return true;
}
// The CTA's abort word (shared memory): set once any warp's bounded wait gave up.  From then on
// the producer issues no more copies and the consumers skip their waits and their arithmetic
// but still walk the whole schedule, so every warp reaches each named barrier and each stage
// release the same number of times and the kernel ends.  The step's output is invalid and the
// host reports BTE_ETIMEOUT.
__device__ __forceinline__ bool cta_aborted(const char *smem) {
    return __any_sync(0xffffffffu, *reinterpret_cast<const volatile int *>(smem + kAbortOff) != 0);
}
__device__ __forceinline__ void cta_abort(char *smem) { *reinterpret_cast<volatile int *>(smem + kAbortOff) = 1; }
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     su32(dst)),
                 "l"(src), "r"(bytes), "r"(su32(bar))
                 : "memory");
}
__device__ __forceinline__ void bulk_prefetch_l2(const void *src, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
template <int NCW>
__device__ __forceinline__ void consumer_sync() { asm volatile("bar.sync 1, %0;" ::"n"(NCW * 32) : "memory"); }

// ---- VL-wide loads and stores ---------------------------------------------------------------
// VL decoded values of a box row: p points at the codes, r at the same cells' references in the
// shared reference box (read by the 16-bit instances only).  Codes are taken from 32-bit words
// in registers (no local arrays).
template <int S, int VL>
__device__ __forceinline__ void ld_row(float (&v)[VL], const typename St<S>::T *p, const float *r) {
    using Q = St<S>;
    if constexpr (!Q::kRef) {
        if constexpr (VL == 4) {
            const float4 f = *reinterpret_cast<const float4 *>(p);
            v[0] = f.x; v[1] = f.y; v[2] = f.z; v[3] = f.w;
        } else {
            #pragma unroll
            for (int j = 0; j < VL; ++j) v[j] = p[j];
        }
    } else {
        float f[VL], rr[VL];
        if constexpr (VL == 4) {
            const uint2 q = *reinterpret_cast<const uint2 *>(p);
            f[0] = Q::val(q.x & 0xffffu); f[1] = Q::val(q.x >> 16);
            f[2] = Q::val(q.y & 0xffffu); f[3] = Q::val(q.y >> 16);
            const float4 g = *reinterpret_cast<const float4 *>(r);
            rr[0] = g.x; rr[1] = g.y; rr[2] = g.z; rr[3] = g.w;
        } else {
            #pragma unroll
            for (int j = 0; j < VL; ++j) {
                f[j] = Q::val(Q::bits(p[j]));
                rr[j] = r[j];
            }
        }
        // h + rho, two at a time
        #pragma unroll
        for (int j = 0; j + 1 < VL; j += 2) {
            const float2 d = __fadd2_rn(make_float2(f[j], f[j + 1]), make_float2(rr[j], rr[j + 1]));
            v[j] = d.x;
            v[j + 1] = d.y;
        }
        if constexpr (VL & 1) v[VL - 1] = f[VL - 1] + rr[VL - 1];
    }
}

template <int S, int VL>
__device__ __forceinline__ void st_row(typename St<S>::T *p, const typename St<S>::C (&c)[VL]) {
    using Q = St<S>;
    if constexpr (!Q::kRef) {
        if constexpr (VL == 4) *reinterpret_cast<float4 *>(p) = make_float4(c[0], c[1], c[2], c[3]);
        else {
            #pragma unroll
            for (int j = 0; j < VL; ++j) p[j] = c[j];
        }
    } else {
        if constexpr (VL == 4) {
            *reinterpret_cast<uint2 *>(p) = make_uint2(c[0] | (c[1] << 16), c[2] | (c[3] << 16));
        } else {
            unsigned short *ps = reinterpret_cast<unsigned short *>(p);
            #pragma unroll
            for (int j = 0; j < VL; ++j) ps[j] = (unsigned short)c[j];
        }
    }
}

// ---- plane-tile decoding ---------------------------------------------------------------------
struct PT {
    int tile, k, d, plane, y0, z0, nyt, nzt;
};

template <int DIM, int WPR>
__device__ __forceinline__ PT decode(const StepArgs &a, const TiledArgs &p, int tile, int plane) {
    PT r;
    r.tile = tile;
    r.plane = plane;
    r.k = plane / a.nd;
    r.d = plane - r.k * a.nd;
    const int ty = tile % p.nty, tz = tile / p.nty;
    r.y0 = ty * Geo<DIM, WPR>::TY;
    r.z0 = tz * Geo<DIM, WPR>::TZ;
    r.nyt = min(Geo<DIM, WPR>::TY, a.n[1] - r.y0);
    r.nzt = DIM == 3 ? min(Geo<DIM, WPR>::TZ, a.n[2] - r.z0) : 1;
    return r;
}

// first plane of part j of a tile's plane list
__device__ __forceinline__ int part_begin(const TiledArgs &p, int j) { return (int)((long long)j * p.np / p.J); }

// Walks this CTA's plane-tiles: units blockIdx.x, blockIdx.x + gridDim.x, ...; within a unit its
// planes in order.  q is kept current without divisions inside a unit.
template <int DIM, int WPR>
struct Cursor {
    int u, p0, p1;
    PT q;
    __device__ __forceinline__ bool enter(const StepArgs &a, const TiledArgs &p) {
        for (; u < p.U; u += gridDim.x) {
            const int j = u / p.ntiles;
            p0 = part_begin(p, j);
            p1 = part_begin(p, j + 1);
            if (p0 < p1) {
                q = decode<DIM, WPR>(a, p, u - j * p.ntiles, p0);
                return true;
            }
        }
        return false;
    }
    __device__ __forceinline__ bool start(const StepArgs &a, const TiledArgs &p) {
        u = blockIdx.x;
        return enter(a, p);
    }
    __device__ __forceinline__ bool next(const StepArgs &a, const TiledArgs &p) {
        if (++q.plane < p1) {
            if (++q.d == a.nd) {
                q.d = 0;
                ++q.k;
            }
            return true;
        }
        u += gridDim.x;
        return enter(a, p);
    }
};

// ---- producer warp ----------------------------------------------------------------------------
enum { kSkip = 0, kCopy = 1, kConst = 2 };

// Source row of a ghost row of the box: position pos (< 0 or >= n) along axis ax (1: y, 2: z)
// at the other coordinate `other` (z for a y-ghost, y for a z-ghost).  Sec. 2.2: the wrapped
// row (periodic), the mirrored direction's row (specular), the wall row itself for directions
// leaving through the wall, the diffuse-wall value row, or the thermalizing wall's emission row.
template <int S, int NX>
__device__ __forceinline__ const typename St<S>::T *ghost_row_src(const StepArgs &a, const TiledArgs &p, const PT &q,
                                                                  int ax, int pos, int other, float nu) {
    using T = typename St<S>::T;
    const int gx = a.n[0], ny = a.n[1];
    const int n = a.n[ax];
    const int side = pos < 0 ? 0 : 1;
    const int wall = 2 * ax + side;
    const int bc = a.bc[wall];
    const T *e = static_cast<const T *>(a.e_in);
    auto row_at = [&](int plane, int along) {
        const int yy = ax == 1 ? along : other, zz = ax == 1 ? other : along;
        return e + (long long)plane * a.ncell + ((long long)zz * ny + yy) * gx;
    };
    if (bc == kBcPeriodic) return row_at(q.plane, side ? pos - n : pos + n);
    if (bc == kBcSpecular) {
        const int layer = side ? pos - n + 1 : -pos;
        return row_at(q.k * a.nd + a.mirror[ax * a.nd + q.d], side ? n - layer : layer - 1);
    }
    const bool incoming = side == 0 ? (nu > 0.f) : (nu < 0.f);
    if (!incoming) return row_at(q.plane, side ? n - 1 : 0);
    if constexpr (!St<S>::kRef) {
        if (bc == kBcIsothermal) return static_cast<const T *>(p.isorow) + ((long long)wall * a.nb + q.k) * NX;
    }
    // diffuse wall (and with 16-bit storage the thermalizing wall, whose emission is coded
    // against each wall cell's reference): wall cells of a y-wall are indexed z*nx + x, those
    // of a z-wall y*nx + x
    return static_cast<const T *>(a.ediff_in) + ((long long)wall * a.nb + q.k) * a.wc_max + (long long)other * gx;
}

// Shared-memory side arrays of a stage for the x-wall ghosts (storage format, bulk-copied):
//   spec[wall][TZ][TY][V]   16 bytes of the mirrored direction's row at the wall (specular)
//   dcol[wall][TZ][TY + V]  the diffuse-wall values of the tile's rows (from a 16-byte aligned start)
// with V = 16 / sizeof(T) elements.
template <int S, int WPR, int DIM> struct Side {
    using T = typename St<S>::T;
    static constexpr int V = 16 / (int)sizeof(T);
    static constexpr int TY = Geo<DIM, WPR>::TY, TZ = Geo<DIM, WPR>::TZ, TYP = TY + V;
    static constexpr int spec_elems = 2 * TZ * TY * V;
    static constexpr int bytes = (spec_elems + 2 * TZ * TYP) * (int)sizeof(T);
    static __device__ __forceinline__ T *spec(char *side, int sd, int zl, int yl) {
        return reinterpret_cast<T *>(side) + ((sd * TZ + zl) * TY + yl) * V;
    }
    static __device__ __forceinline__ T *dcol(char *side, int sd, int zl) {
        return reinterpret_cast<T *>(side) + spec_elems + (sd * TZ + zl) * TYP;
    }
};

// element index of the first diffuse value of the tile's rows at slice z, and its offset from
// the 16-byte aligned start the copy uses
__device__ __forceinline__ long long dcol_src(const StepArgs &a, int sd, int k, int z, int y0) {
    return ((long long)sd * a.nb + k) * a.wc_max + (long long)z * a.n[1] + y0;
}

template <int S, int VL, int WPR, int DIM>
__device__ void producer(const StepArgs &a, const TiledArgs &p, char *smem, uint64_t *full, uint64_t *empty) {
    using T = typename St<S>::T;
    using SD = Side<S, WPR, DIM>;
    constexpr int NX = 32 * VL * WPR, TY = Geo<DIM, WPR>::TY;
    constexpr int V = SD::V;
    const int lane = threadIdx.x & 31;
    const int gx = a.n[0], ny = a.n[1], nz = a.n[2];
    // a row of the grid is gx <= NX cells (a multiple of 16 bytes); box rows keep the stride NX
    const uint32_t rowb = (uint32_t)gx * sizeof(T);
    const T *e = static_cast<const T *>(a.e_in);
    const T *ed = static_cast<const T *>(a.ediff_in);
    const int bx[2] = {a.bc[0], a.bc[1]};
    Cursor<DIM, WPR> cur, ahead;
    bool more = cur.start(a, p);
    bool ahead_ok = ahead.start(a, p);
    for (int j = 0; j < p.ns && ahead_ok; ++j) ahead_ok = ahead.next(a, p);  // the plane-tile ns later
    int s = 0;         // stage of plane-tile i = i mod ns
    uint32_t ph = 0u;  // its use count parity = (i / ns) mod 2
    // failure-detection test: a first wait on a barrier that nothing completes
    if ((p.stall & 2) &&
        !__all_sync(0xffffffffu, mbar_wait(reinterpret_cast<uint64_t *>(smem + kStallOff), 0u, p.err, 2, p.wait_ns)))
        cta_abort(smem);
    int i = 0;         // plane-tiles whose copies were issued
    for (; more; ++i, more = cur.next(a, p)) {
        if (i >= p.ns && !__all_sync(0xffffffffu, mbar_wait(&empty[s], ph ^ 1u, p.err, 2, p.wait_ns))) cta_abort(smem);
        if (cta_aborted(smem)) break;
        fence_proxy_async();
        __syncwarp();
        const PT &q = cur.q;
        const float nux = a.nu[3 * q.plane], nuy = a.nu[3 * q.plane + 1];
        const float nuz = DIM == 3 ? a.nu[3 * q.plane + 2] : 0.f;
        const int ybox0 = q.y0 - (nuy > 0.f ? 2 : 1);
        const int zbox0 = DIM == 3 ? q.z0 - (nuz > 0.f ? 2 : 1) : 0;
        const int nry = q.nyt + 3, nrz = DIM == 3 ? q.nzt + 3 : 1;
        char *stage = smem + p.stage0 + (size_t)s * p.stage_bytes;
        char *side = stage + p.side_off;
        const long long pbase = (long long)q.plane * a.ncell;
        const int ncore = q.nyt * q.nzt;
        const bool spec[2] = {bx[0] == kBcSpecular, bx[1] == kBcSpecular};
        const bool dif[2] = {bx[0] == kBcDiffuse && nux > 0.f, bx[1] == kBcDiffuse && nux < 0.f};
        // Every box row the stencil reads is filled by exactly one bulk copy, so the byte count is
        // closed-form: core slices need all nry rows, the z-halo slices the nyt core rows.  x-wall
        // side copies have fixed sizes.
        const int nneed = DIM == 3 ? q.nzt * nry + (nrz - q.nzt) * q.nyt : nry;
        const int ndcol = (q.nyt + V - 1) / V + 1;  // 16-byte units of a diffuse column copy
        if (lane == 0) {
            const uint32_t bytes = (uint32_t)nneed * rowb + (spec[0] + spec[1]) * (uint32_t)ncore * 16u +
                                   (dif[0] + dif[1]) * (uint32_t)q.nzt * ndcol * 16u + 64u;
            mbar_expect_tx(&full[s], bytes);
            // per-plane constants (64 bytes, prepared once on the device)
            bulk_g2s(stage + p.hdr_off, p.hdr + (size_t)q.plane * kHdrFloats, 64, &full[s]);
        }
        __syncwarp();
        // Work items: per box slice, nch chunks of its in-domain rows (one contiguous run in global
        // and in shared memory) and 4 ghost-row slots (two below, two above the domain in y); a
        // slice outside the domain (a z-wall) uses its first nyt items for the core rows' ghosts.
        const int nch = (nry + p.chunk - 1) / p.chunk;
        const int per = max(nch + 4, DIM == 3 ? q.nyt : 0);
        for (int w = lane; w < nrz * per; w += 32) {
            const int rz = w / per, it = w - rz * per;
            const int z = zbox0 + rz;
            T *slice = reinterpret_cast<T *>(stage) + (size_t)rz * (TY + 3) * NX;
            if (DIM == 3 && (z < 0 || z >= nz)) {
                if (it < q.nyt) {
                    const int y = q.y0 + it;
                    bulk_g2s(slice + (size_t)(y - ybox0) * NX, ghost_row_src<S, NX>(a, p, q, 2, z, y, nuz), rowb, &full[s]);
                }
                continue;
            }
            const bool coreZ = DIM == 2 || (z >= q.z0 && z < q.z0 + q.nzt);
            const int ylo = coreZ ? ybox0 : q.y0, yhi = coreZ ? ybox0 + nry : q.y0 + q.nyt;
            const int ya = max(ylo, 0), yb = min(yhi, ny);
            if (it < nch) {
                const int y = ya + it * p.chunk;
                if (y < yb)
                    bulk_g2s(slice + (size_t)(y - ybox0) * NX, e + pbase + ((long long)z * ny + y) * gx,
                             (uint32_t)min(p.chunk, yb - y) * rowb, &full[s]);
            } else if (it < nch + 4) {
                const int g = it - nch;  // 0, 1: below the domain; 2, 3: above it
                const int y = g < 2 ? ylo + g : yb + (g - 2);
                if (g < 2 ? y < ya : y < yhi)
                    bulk_g2s(slice + (size_t)(y - ybox0) * NX, ghost_row_src<S, NX>(a, p, q, 1, y, z, nuy), rowb, &full[s]);
            }
        }
        // x-wall ghosts outside the tile: 16 bytes of the mirrored direction's row (specular), or
        // the diffuse values of the tile's rows (incoming directions only)
        for (int sd = 0; sd < 2; ++sd) {
            if (spec[sd]) {
                const long long mb = ((long long)q.k * a.nd + a.mirror[q.d]) * a.ncell + (sd ? gx - V : 0);
                for (int j = lane; j < ncore; j += 32) {
                    const int yl = j % q.nyt, zl = j / q.nyt;
                    bulk_g2s(SD::spec(side, sd, zl, yl), e + mb + ((long long)(q.z0 + zl) * ny + q.y0 + yl) * gx, 16, &full[s]);
                }
            }
            if (dif[sd])
                for (int zl = lane; zl < q.nzt; zl += 32) {
                    const long long s0 = dcol_src(a, sd, q.k, q.z0 + zl, q.y0);
                    bulk_g2s(SD::dcol(side, sd, zl), ed + (s0 - (s0 & (V - 1))), (uint32_t)ndcol * 16u, &full[s]);
                }
        }
        mbar_arrive(&full[s]);
        // pull the rows of a later plane-tile towards L2 (no shared memory involved)
        if (ahead_ok) {
            const PT &qp = ahead.q;
            const float pnuy = a.nu[3 * qp.plane + 1];
            const float pnuz = DIM == 3 ? a.nu[3 * qp.plane + 2] : 0.f;
            const int ylo = max(qp.y0 - (pnuy > 0.f ? 2 : 1), 0), yhi = min(qp.y0 + qp.nyt + (pnuy > 0.f ? 1 : 2), ny);
            const int zlo = DIM == 3 ? max(qp.z0 - (pnuz > 0.f ? 2 : 1), 0) : 0;
            const int zhi = DIM == 3 ? min(qp.z0 + qp.nzt + (pnuz > 0.f ? 1 : 2), nz) : 1;
            for (int z = zlo + lane; z < zhi; z += 32)
                bulk_prefetch_l2(e + (long long)qp.plane * a.ncell + ((long long)z * ny + ylo) * gx, (uint32_t)(yhi - ylo) * rowb);
            ahead_ok = ahead.next(a, p);
        }
        if (++s == p.ns) {
            s = 0;
            ph ^= 1u;
        }
    }
    // Before the CTA exits, every bulk copy it issued has landed: the last use of each stage
    // (bounded; a copy that never lands leaves the error flag set).  A stage is reused only after
    // the empty wait, and that is followed by the abort check, so no copy is issued into a stage
    // whose previous copies may still be in flight.
    for (int j = max(i - p.ns, 0); j < i; ++j) mbar_wait(&full[j % p.ns], (uint32_t)(j / p.ns) & 1u, p.err, 2, kWaitLimitNs);
}

// ---- consumer warps -----------------------------------------------------------------------
// Where an end lane of a warp takes its two x-neighbours from (besides the plain shuffle).
enum { kGhShfl = 0, kGhSmem = 1, kGhSpec = 2, kGhDiff = 3, kGhConst = 4, kGhOwn = 5 };

// SY, SX: signs of the direction's y and x components (+1 when positive, else -1), fixed per
// instance so that row steps are constants and the x faces need no orientation branch.  FULL:
// the warp's KR rows all lie in the tile (every tile but a ragged last one), so the row loop
// carries no exit test.
template <int S, int LIM, int VL, int WPR, int DIM, bool SR, int SY, int SX, bool FULL>
__device__ __forceinline__ void rows_of_warp(const StepArgs &a, const TiledArgs &p, const PT &q, const char *stage,
                                             int zl, int rb, int half, float *accsm,
                                             float (&acc)[Geo<DIM, WPR>::KR][VL], const float *btsm, float *wsm,
                                             const float *rbox) {
    using T = typename St<S>::T;
    constexpr bool REF = St<S>::kRef;
    constexpr int NX = 32 * VL * WPR, TY = Geo<DIM, WPR>::TY, RY = TY + 4;
    const int lane = threadIdx.x & 31, x0 = (half * 32 + lane) * VL;
    const int rowlen = a.n[0], ny = a.n[1], nz = a.n[2];
    // The grid's rows hold rowlen <= NX cells (a multiple of VL): lanes past the row's end compute
    // on unused box columns and store nothing.  The right end lane of this warp's part of the row
    // holds its last cell (lane 31 unless the row ends inside this warp's part).
    const bool active = x0 < rowlen;
    const int rend = min(31, (rowlen - half * 32 * VL) / VL - 1);
    const float *hd = reinterpret_cast<const float *>(stage + p.hdr_off);  // per-plane constants
    const float4 h0 = reinterpret_cast<const float4 *>(hd)[0];
    const float nux = h0.x, nuy = h0.y, nuz = h0.z, wm = h0.w;
    const float dtinv = hd[4], sc = hd[5];
    const float any = fabsf(nuy), anz = fabsf(nuz);
    constexpr int sy = SY;
    const int sz = nuz > 0.f ? 1 : -1;
    constexpr int kR = Geo<DIM, WPR>::KR;
    const int nrows = FULL ? kR : min(kR, q.nyt - rb);
    const int yl0 = sy > 0 ? rb : rb + nrows - 1;  // first row in streaming (upwind-to-downwind) order
    const int ybox0 = q.y0 - (sy > 0 ? 2 : 1);
    const int zbox0 = DIM == 3 ? q.z0 - (sz > 0 ? 2 : 1) : 0;
    const int z = q.z0 + zl;
    const T *box = reinterpret_cast<const T *>(stage);
    const int dy = sy * NX;                    // next row in streaming order (elements)
    const int dz = sz * (TY + 3) * NX;         // next slice downwind (elements)
    int o = ((z - zbox0) * (TY + 3) + (q.y0 + yl0 - ybox0)) * NX;  // row start in the box
    int c = (zl * TY + yl0) * NX + x0;         // this lane's cells in the tile arrays
    // the same row in the reference box (rows y0-2.., slices z0-2..), and its upwind steps; a
    // second ghost layer of a thermalizing or diffuse wall holds the wall value coded against
    // the wall cell's reference, as the first layer does
    const int dyR = sy * NX, dzR = sz * RY * NX;
    const uint32_t pkey = SR ? plane_key(a.srkey, q.plane) : 0u;
    int ro = ((DIM == 3 ? zl + 2 : 0) * RY + yl0 + 2) * NX;
    int ry2 = 2 * dyR, rz2 = 2 * dzR;
    if constexpr (REF) {
        const int yg = q.y0 + yl0 - 2 * sy;
        if (yg < 0 || yg >= ny) {
            const int bcy = a.bc[yg < 0 ? 2 : 3];
            if (bcy == kBcIsothermal || bcy == kBcDiffuse) ry2 = dyR;
        }
        if constexpr (DIM == 3) {
            const int zg = z - 2 * sz;
            if (zg < 0 || zg >= nz) {
                const int bcz = a.bc[zg < 0 ? 4 : 5];
                if (bcz == kBcIsothermal || bcz == kBcDiffuse) rz2 = dzR;
            }
        }
    }
    T *eo = static_cast<T *>(a.e_out) + (long long)q.plane * a.ncell + ((long long)z * ny + q.y0 + yl0) * rowlen + x0;
    const int dyg = sy * rowlen;                   // next row in streaming order (global elements)
    using SD = Side<S, WPR, DIM>;
    char *side = const_cast<char *>(stage) + p.side_off;
    // x ghosts of the two end lanes, decided once per plane-tile
    const bool xlo = lane == 0 && half == 0, xhi = x0 + VL == rowlen;
    // Ghost sources of the two end lanes, decided once per plane-tile.  Every lane then reads two
    // values g0 (next to its end) and g1 (second ghost) per row from gptr + j * gstep at gi0 / gi1
    // (other lanes read their own cells), and the mode picks between them, a constant and the
    // lane's own end cell -- no divergent code in the row loop.
    int gmode = kGhShfl;
    const T *gptr = box + o + x0;
    int gstep = dy, gi0 = 0, gi1 = 0;
    int rx0 = x0, rx1 = x0;  // the two ghosts' cells in the reference box row
    float gc = 0.f;
    if (lane == 0 || lane == rend) {
        const int sd = lane == 0 ? 0 : 1;
        const int bc = a.bc[sd];
        const bool wall_lane = sd == 0 ? xlo : xhi;
        const bool leaving = sd == 0 ? nux <= 0.f : nux >= 0.f;
        gmode = kGhSmem;
        if (wall_lane && bc == kBcPeriodic && WPR == 1 && rowlen == NX) {
            // one warp holds the whole row: the plain shuffle wraps around it, which is the
            // periodic image
            gmode = kGhShfl;
        } else if (!wall_lane || bc == kBcPeriodic) {
            const int gi = !wall_lane ? (sd == 0 ? x0 - 2 : x0 + VL) : (sd == 0 ? rowlen - 2 : 0);
            gptr = box + o + gi;
            gi0 = sd == 0 ? 1 : 0;
            gi1 = sd == 0 ? 0 : 1;
            rx0 = gi + gi0;
            rx1 = gi + gi1;
        } else if (bc == kBcSpecular) {
            gptr = SD::spec(side, sd, zl, yl0);
            gstep = sy * SD::V;
            gi0 = sd == 0 ? 0 : SD::V - 1;
            gi1 = sd == 0 ? 1 : SD::V - 2;
            rx0 = (sd == 0 ? 0 : rowlen - SD::V) + gi0;
            rx1 = (sd == 0 ? 0 : rowlen - SD::V) + gi1;
        } else if (leaving) {
            gmode = kGhOwn;
            // FP32: read the lane's own end cell from the box row (same value, no select)
            if constexpr (!REF) gi0 = gi1 = sd == 0 ? 0 : VL - 1;
        } else if (bc == kBcIsothermal) {
            gmode = kGhConst;
            gc = hd[7 + sd];
            // FP32: read the emission value from the plane's constants (no select)
            if constexpr (!REF) {
                gptr = reinterpret_cast<const T *>(hd + 7 + sd);
                gstep = 0;
            }
        } else {
            gptr = SD::dcol(side, sd, zl) + (int)(dcol_src(a, sd, q.k, z, q.y0) & (SD::V - 1)) + yl0;
            gstep = sy;
            rx0 = rx1 = sd == 0 ? 0 : rowlen - 1;
        }
    }
    // whether any end lane of the warp takes its ghosts other than by the plain shuffle (always,
    // when two warps share a row: each has an inner end)
    const bool need_gh = WPR == 2 || __any_sync(0xffffffffu, gmode != kGhShfl);
    // diffuse-wall sums of Eq. (diff_bound) for the next step: cells next to a diffuse wall add
    // w_d (s_d.n) e for the directions leaving through it (weight 0 otherwise)
    const float wx = xlo ? hd[9] : (xhi ? hd[10] : 0.f);
    float *wxp = wsm + (xlo ? max(p.wslot[0], 0) : max(p.wslot[1], 0)) * p.tw + zl * TY + yl0;
    const float wz = DIM == 3 ? (z == 0 ? hd[13] : (z == nz - 1 ? hd[14] : 0.f)) : 0.f;
    float *wzp = wsm + (z == 0 ? max(p.wslot[4], 0) : max(p.wslot[5], 0)) * p.tw + yl0 * NX + x0;
    const float wy0 = hd[11], wy1 = hd[12];
    // the rows of this warp on the y walls, as loop indices in streaming order (-1: none)
    const int ys0 = q.y0 + yl0;
    const int jw0 = wy0 != 0.f ? -ys0 * sy : -1, jw1 = wy1 != 0.f ? (ny - 1 - ys0) * sy : -1;
    float *wy0p = wsm + max(p.wslot[2], 0) * p.tw + zl * NX + x0;
    float *wy1p = wsm + max(p.wslot[3], 0) * p.tw + zl * NX + x0;

    float wm2[VL], wm1[VL], w0[VL], wp1[VL], fin[VL];
    ld_row<S, VL>(wm2, box + o - 2 * dy + x0, rbox + ro - ry2 + x0);
    ld_row<S, VL>(wm1, box + o - dy + x0, rbox + ro - dyR + x0);
    ld_row<S, VL>(w0, box + o + x0, rbox + ro + x0);
    faces<LIM, VL>(wm2, wm1, w0, fin);
    #pragma unroll
    for (int jj = 0; jj < kR; ++jj) {
        // r: the row's place in the warp's stretch (its accumulators); j: its place in the stream
        const int r = SY > 0 ? jj : kR - 1 - jj;
        if (!FULL && r >= nrows) continue;
        const int j = SY > 0 ? r : nrows - 1 - r;
        const int y = q.y0 + yl0 + j * sy;
        ld_row<S, VL>(wp1, box + o + dy + x0, rbox + ro + dyR + x0);
        float fout[VL];
        // y: out face between y and y + sy (upwind y); the in face is the previous row's out face
        faces<LIM, VL>(wm1, w0, wp1, fout);
        // x: neighbours from the adjacent lanes, the end lanes as decided above
        float ex[VL + 4];
        #pragma unroll
        for (int v = 0; v < VL; ++v) ex[v + 2] = w0[v];
        ex[0] = __shfl_sync(0xffffffffu, w0[VL - 2], (lane + 31) & 31);
        ex[1] = __shfl_sync(0xffffffffu, w0[VL - 1], (lane + 31) & 31);
        ex[VL + 2] = __shfl_sync(0xffffffffu, w0[0], (lane + 1) & 31);
        ex[VL + 3] = __shfl_sync(0xffffffffu, w0[1], (lane + 1) & 31);
        if (need_gh) {
            const T *gp = gptr + j * gstep;
            float r0 = 0.f, r1 = 0.f;
            if constexpr (REF) {
                r0 = rbox[ro + rx0];
                r1 = rbox[ro + rx1];
            }
            float g0 = St<S>::dec(gp[gi0], r0), g1 = St<S>::dec(gp[gi1], r1);
            if constexpr (REF) {
                const float own = lane == 0 ? w0[0] : w0[VL - 1];
                g0 = gmode == kGhConst ? gc : (gmode == kGhOwn ? own : g0);
                g1 = gmode == kGhConst ? gc : (gmode == kGhOwn ? own : g1);
            }
            const bool l0 = gmode != kGhShfl && lane == 0, l31 = gmode != kGhShfl && lane == rend;
            ex[1] = l0 ? g0 : ex[1];
            ex[0] = l0 ? g1 : ex[0];
            ex[VL + 2] = l31 ? g0 : ex[VL + 2];
            ex[VL + 3] = l31 ? g1 : ex[VL + 3];
        }
        // faces F_j between x0+j and x0+j+1, j = -1..VL-1 (index j+1); flux in signed form
        float F[VL + 1];
        if constexpr (SX > 0) faces<LIM, VL + 1>(ex, ex + 1, ex + 2, F);  // upwind cell x0+j
        else faces<LIM, VL + 1>(ex + 3, ex + 2, ex + 1, F);             // upwind cell x0+j+1
        float gx[VL];
        #pragma unroll
        for (int v = 0; v < VL; ++v) gx[v] = F[v + 1] - F[v];
        float zo[VL], zi[VL];
        if constexpr (DIM == 3) {
            float zm1[VL], zm2[VL], zp1[VL];
            ld_row<S, VL>(zm1, box + o - dz + x0, rbox + ro - dzR + x0);
            ld_row<S, VL>(zm2, box + o - 2 * dz + x0, rbox + ro - rz2 + x0);
            ld_row<S, VL>(zp1, box + o + dz + x0, rbox + ro + dzR + x0);
            faces<LIM, VL>(zm1, w0, zp1, zo);
            faces<LIM, VL>(zm2, zm1, w0, zi);
        }
        // update, store, moment and diffuse-wall partials
        float bt[VL], ac[VL];
        if constexpr (VL == 4) {
            const float4 f = *reinterpret_cast<const float4 *>(btsm + c);
            bt[0] = f.x; bt[1] = f.y; bt[2] = f.z; bt[3] = f.w;
        } else {
            #pragma unroll
            for (int v = 0; v < VL; ++v) bt[v] = btsm[c + v];
        }
        if constexpr (kAccRegs<DIM>) {
            #pragma unroll
            for (int v = 0; v < VL; ++v) ac[v] = acc[r][v];
        } else if constexpr (VL == 4) {
            const float4 g = *reinterpret_cast<const float4 *>(accsm + c);
            ac[0] = g.x; ac[1] = g.y; ac[2] = g.z; ac[3] = g.w;
        } else {
            #pragma unroll
            for (int v = 0; v < VL; ++v) ac[v] = accsm[c + v];
        }
        typename St<S>::C h[VL];
        float en[VL], es[VL];
        const long long grow = ((long long)z * ny + y) * rowlen;  // global index of the row's first cell
        // FP32: e^{n+1} = e - dt/tau e + bt - |nu_y| (F_out - F_in) - nu_x (F_{v+1} - F_v)
        // [- |nu_z| (F_zout - F_zin)].  16-bit: bt carries -rho_new, so en is already the new code's
        // value.  Two cells at a time.
        #pragma unroll
        for (int v = 0; v + 1 < VL; v += 2) {
            const float2 u = make_float2(w0[v], w0[v + 1]);
            float2 t = __fadd2_rn(__ffma2_rn(f2(-dtinv), u, u), make_float2(bt[v], bt[v + 1]));
            t = __ffma2_rn(f2(-any), sub2(make_float2(fout[v], fout[v + 1]), make_float2(fin[v], fin[v + 1])), t);
            t = __ffma2_rn(f2(-nux), make_float2(gx[v], gx[v + 1]), t);
            if constexpr (DIM == 3)
                t = __ffma2_rn(f2(-anz), sub2(make_float2(zo[v], zo[v + 1]), make_float2(zi[v], zi[v + 1])), t);
            en[v] = t.x;
            en[v + 1] = t.y;
        }
        if constexpr (VL & 1) {
            constexpr int v = VL - 1;
            float t = fmaf(-dtinv, w0[v], w0[v]) + bt[v];
            t = fmaf(-any, fout[v] - fin[v], t);
            t = fmaf(-nux, gx[v], t);
            if constexpr (DIM == 3) t = fmaf(-anz, zo[v] - zi[v], t);
            en[v] = t;
        }
        #pragma unroll
        for (int v = 0; v < VL; ++v) {
            if constexpr (SR) h[v] = St<S>::enc_sr(en[v], mix32(pkey ^ (uint32_t)(grow + x0 + v)));
            else h[v] = St<S>::enc(en[v]);
            es[v] = St<S>::val(h[v]);
        }
        // moment partials, two cells at a time
        #pragma unroll
        for (int v = 0; v + 1 < VL; v += 2) {
            const float2 m = __ffma2_rn(f2(wm), make_float2(es[v], es[v + 1]), make_float2(ac[v], ac[v + 1]));
            ac[v] = m.x;
            ac[v + 1] = m.y;
        }
        if constexpr (VL & 1) ac[VL - 1] = fmaf(wm, es[VL - 1], ac[VL - 1]);
        if constexpr (kAccRegs<DIM>) {
            #pragma unroll
            for (int v = 0; v < VL; ++v) acc[r][v] = ac[v];
        } else if constexpr (VL == 4) {
            *reinterpret_cast<float4 *>(accsm + c) = make_float4(ac[0], ac[1], ac[2], ac[3]);
        } else {
            #pragma unroll
            for (int v = 0; v < VL; ++v) accsm[c + v] = ac[v];
        }
        if (active) st_row<S, VL>(eo, h);
        // the stored values at the walls: 16-bit codes are decoded against the new reference
        // (T_L^n of the cell, read from global memory for wall cells only)
        // x walls: only the two end lanes have a non-zero weight (a predicated update)
        if (wx != 0.f) {
            const int xe = lane == 0 ? 0 : VL - 1;
            float ev = es[xe];
            if constexpr (REF) ev = sc * (ev + a.TL[grow + x0 + xe] * a.invTs);
            wxp[j * sy] += wx * ev;
        }
        if (active && (j == jw0 || j == jw1)) {
            const float wy = j == jw0 ? wy0 : wy1;
            float *w = j == jw0 ? wy0p : wy1p;
            #pragma unroll
            for (int v = 0; v < VL; ++v) {
                float ev = es[v];
                if constexpr (REF) ev = sc * (ev + a.TL[grow + x0 + v] * a.invTs);
                w[v] += wy * ev;
            }
        }
        if (DIM == 3 && wz != 0.f && active) {
            #pragma unroll
            for (int v = 0; v < VL; ++v) {
                float ev = es[v];
                if constexpr (REF) ev = sc * (ev + a.TL[grow + x0 + v] * a.invTs);
                wzp[j * sy * NX + v] += wz * ev;
            }
        }
        #pragma unroll
        for (int v = 0; v < VL; ++v) {
            wm2[v] = wm1[v];
            wm1[v] = w0[v];
            w0[v] = wp1[v];
            fin[v] = fout[v];
        }
        o += dy;
        c += dy;
        eo += dyg;
        ro += dyR;
    }
}

template <int VL, int WPR, int DIM>
__device__ __forceinline__ void warp_place(int &zl, int &rb, int &half) {
    const int warp = threadIdx.x >> 5;
    half = warp % WPR;
    const int u = warp / WPR;
    zl = u % Geo<DIM, WPR>::TZ;
    rb = (u / Geo<DIM, WPR>::TZ) * Geo<DIM, WPR>::KR;
}

// End of a segment: this thread's moment partials to P[seg], the diffuse-wall partials of
// the tile to PW[seg]; both shared arrays are cleared for the next segment.  With 16-bit
// storage the accumulated sum is sum_d w_d/tau h_d over the segment's planes; the stored
// values are s_k (h_d + rho_new), so P = s_k * sum + (sum_d w_d/tau) C_k T_L^n / W.
template <bool REF, int VL, int WPR, int DIM>
__device__ __forceinline__ void flush_segment(const StepArgs &a, const TiledArgs &p, int seg, const PT &q,
                                              float *accsm, float (&acc)[Geo<DIM, WPR>::KR][VL], float *wsm,
                                              float wsum) {
    constexpr int NX = 32 * VL * WPR, TY = Geo<DIM, WPR>::TY, NCW = Geo<DIM, WPR>::NCW;
    int zl, rb, half;
    warp_place<VL, WPR, DIM>(zl, rb, half);
    const int x0 = (half * 32 + (threadIdx.x & 31)) * VL;
    const int gx = a.n[0];
    float *P = a.P + (size_t)seg * p.tcells;
    float sc = 1.f, wck = 0.f;
    if constexpr (REF) {
        const BandConst b = a.band[q.k];
        sc = b.scale;
        wck = wsum * b.ck;
    }
    #pragma unroll
    for (int r = 0; r < Geo<DIM, WPR>::KR; ++r) {
        const int yl = rb + r;
        const int c = (zl * TY + yl) * NX + x0;
        if (yl < q.nyt && zl < q.nzt && x0 < gx) {
            const long long g = ((long long)(q.z0 + zl) * a.n[1] + q.y0 + yl) * gx + x0;
            #pragma unroll
            for (int v = 0; v < VL; ++v) {
                const float m = kAccRegs<DIM> ? acc[r][v] : accsm[c + v];
                if constexpr (REF) P[c + v] = fmaf(sc, m, wck * a.TL[g + v]);
                else P[c + v] = m;
            }
        }
        #pragma unroll
        for (int v = 0; v < VL; ++v) {
            if constexpr (kAccRegs<DIM>) acc[r][v] = 0.f;
            else accsm[c + v] = 0.f;
        }
    }
    consumer_sync<NCW>();
    for (int idx = threadIdx.x; idx < p.nwd * p.tw; idx += NCW * 32) {
        p.PW[(size_t)seg * p.nwd * p.tw + idx] = wsm[idx];
        wsm[idx] = 0.f;
    }
    consumer_sync<NCW>();
}

// Row of the reference box for position pos along an axis of n cells: the cell itself inside,
// the wrapped cell at a periodic wall, else the mirror image (ghost layer L -> cell L-1 from
// the wall), which is the cell a specular or outgoing ghost is copied from; clamped for rows
// the stencil never reads.
__device__ __forceinline__ int ref_row(int pos, int n, int bclo, int bchi) {
    if (pos < 0) pos = bclo == kBcPeriodic ? pos + n : -pos - 1;
    else if (pos >= n) pos = bchi == kBcPeriodic ? pos - n : 2 * n - pos - 1;
    return min(max(pos, 0), n - 1);
}

// Reference box of a unit's tile: rho = R / T_scale at rows y0-2 .. y0+TY+1 (and slices
// z0-2 .. z0+TZ+1 in 3-D) of every x, ghost rows mapped by ref_row.
template <int VL, int WPR, int DIM>
__device__ __forceinline__ void fill_ref_box(const StepArgs &a, const PT &q, float *rbox) {
    constexpr int NX = 32 * VL * WPR, TY = Geo<DIM, WPR>::TY, TZ = Geo<DIM, WPR>::TZ, NCW = Geo<DIM, WPR>::NCW;
    constexpr int RY = TY + 4, RZ = DIM == 3 ? TZ + 4 : 1;
    const int gx = a.n[0], ny = a.n[1], nz = a.n[2];
    for (int idx = threadIdx.x; idx < RZ * RY * NX; idx += NCW * 32) {
        const int x = idx % NX, ry = (idx / NX) % RY, rz = idx / (NX * RY);
        const int y = ref_row(q.y0 - 2 + ry, ny, a.bc[2], a.bc[3]);
        const int z = DIM == 3 ? ref_row(q.z0 - 2 + rz, nz, a.bc[4], a.bc[5]) : 0;
        rbox[idx] = x < gx ? a.R[((long long)z * ny + y) * gx + x] * a.invTs : 0.f;
    }
}

template <int S, int LIM, int VL, int WPR, int DIM, bool SR>
__device__ void consumer(const StepArgs &a, const TiledArgs &p, char *smem, uint64_t *full, uint64_t *empty) {
    constexpr bool REF = St<S>::kRef;
    constexpr int NX = 32 * VL * WPR, TY = Geo<DIM, WPR>::TY, NCW = Geo<DIM, WPR>::NCW;
    const int lane = threadIdx.x & 31;
    int zl, rb, half;
    warp_place<VL, WPR, DIM>(zl, rb, half);
    const int x0 = (half * 32 + lane) * VL;
    const int gx = a.n[0], ny = a.n[1];
    float *wsm = reinterpret_cast<float *>(smem + p.wall_off);
    float *btsm = reinterpret_cast<float *>(smem + p.bt_off);
    float *accsm = reinterpret_cast<float *>(smem + p.acc_off);
    float acc[Geo<DIM, WPR>::KR][VL];  // 3-D: this thread's moment partials of the current segment
    #pragma unroll
    for (int r = 0; r < Geo<DIM, WPR>::KR; ++r)
        #pragma unroll
        for (int v = 0; v < VL; ++v) acc[r][v] = 0.f;
    float *rbox = reinterpret_cast<float *>(smem + p.rho_off);
    int seg = -1, cur_unit = -1, cur_band = -1;
    int s = 0;         // stage of plane-tile i = i mod ns
    uint32_t ph = 0u;  // its use count parity = (i / ns) mod 2
    float wsum = 0.f;  // sum of w_d / tau_k over the segment's planes (16-bit storage)
    PT cur{};
    // failure-detection test: a first wait on a barrier that nothing completes (the CTA then gives
    // up at its first wait for data that does not come)
    if ((p.stall & 1) &&
        !__all_sync(0xffffffffu, mbar_wait(reinterpret_cast<uint64_t *>(smem + kStallOff), 0u, p.err, 1, p.wait_ns)) &&
        lane == 0)
        cta_abort(smem);
    Cursor<DIM, WPR> c;
    bool more = c.start(a, p);
    for (int i = 0; more; ++i, more = c.next(a, p)) {
        const PT q = c.q;
        if (c.u != cur_unit || q.k != cur_band) {
            if (seg >= 0) flush_segment<REF, VL, WPR, DIM>(a, p, seg, cur, accsm, acc, wsm, wsum);
            if constexpr (REF) {
                // after the flush's barriers no warp reads the previous unit's references
                if (c.u != cur_unit) {
                    fill_ref_box<VL, WPR, DIM>(a, q, rbox);
                    consumer_sync<NCW>();
                }
            }
            seg = p.unit_seg0[c.u] + q.k - c.p0 / a.nd;
            cur_unit = c.u;
            cur_band = q.k;
            cur = q;
            wsum = 0.f;
            // per-cell relaxation target and source of this band: dt/tau C T_L / W + a dt C Q/(sum C W)
            // (16-bit: in units of s_k, less the new code reference rho_new = T_L^n / T_scale)
            const BandConst b = a.band[q.k];
            #pragma unroll
            for (int r = 0; r < Geo<DIM, WPR>::KR; ++r) {
                const int yl = rb + r;
                if (yl < q.nyt && zl < q.nzt && x0 < gx) {
                    const long long i0 = ((long long)(q.z0 + zl) * ny + (q.y0 + yl)) * gx + x0;
                    float *bp = btsm + (zl * TY + yl) * NX + x0;
                    #pragma unroll
                    for (int v = 0; v < VL; ++v) {
                        const float src = a.Q ? b.srck * (a.amp * a.Q[i0 + v]) : 0.f;
                        if constexpr (REF)
                            bp[v] = fmaf(b.dtinv - 1.f, a.TL[i0 + v] * a.invTs, src * b.inv_scale);
                        else
                            bp[v] = fmaf(b.dtinv, b.ck * a.TL[i0 + v], src);
                    }
                }
            }
        }
        // warp-uniform: the stage's copies landed, else a bounded wait unless a warp gave up
        bool ok = __all_sync(0xffffffffu, mbar_try_wait(&full[s], ph));
        if (!ok) {
            ok = !cta_aborted(smem);
            if (ok) ok = __all_sync(0xffffffffu, mbar_wait(&full[s], ph, p.err, 1, p.wait_ns));
        }
        if (!ok) {
            // release the stage unread and walk on through the schedule
            if (lane == 0) {
                cta_abort(smem);
                mbar_arrive(&empty[s]);
            }
            if (++s == p.ns) {
                s = 0;
                ph ^= 1u;
            }
            continue;
        }
        const char *stage = smem + p.stage0 + (size_t)s * p.stage_bytes;
        if constexpr (REF) wsum += reinterpret_cast<const float *>(stage + p.hdr_off)[3];
        if (zl < q.nzt && rb < q.nyt) {
            const float *hd = reinterpret_cast<const float *>(stage + p.hdr_off);
            const bool px = hd[0] > 0.f, py = hd[1] > 0.f;  // the signs rows_of_warp takes
            const bool full = rb + Geo<DIM, WPR>::KR <= q.nyt;
#define BTE_ROWS(SY_, SX_, F_) rows_of_warp<S, LIM, VL, WPR, DIM, SR, SY_, SX_, F_>(a, p, q, stage, zl, rb, half, accsm, acc, btsm, wsm, rbox)
            if (full) {
                if (py) { if (px) BTE_ROWS(1, 1, true); else BTE_ROWS(1, -1, true); }
                else { if (px) BTE_ROWS(-1, 1, true); else BTE_ROWS(-1, -1, true); }
            } else {
                if (py) { if (px) BTE_ROWS(1, 1, false); else BTE_ROWS(1, -1, false); }
                else { if (px) BTE_ROWS(-1, 1, false); else BTE_ROWS(-1, -1, false); }
            }
#undef BTE_ROWS
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
        if (++s == p.ns) {
            s = 0;
            ph ^= 1u;
        }
    }
    if (seg >= 0) flush_segment<REF, VL, WPR, DIM>(a, p, seg, cur, accsm, acc, wsm, wsum);
}

// SR: 16-bit codes rounded stochastically (a separate instance, so the round-to-nearest one
// carries none of the hashing)
template <int S, int LIM, int VL, int WPR, int DIM, bool SR>
__global__ void __launch_bounds__((Geo<DIM, WPR>::NCW + kProducerWarps) * 32, 1) k_step_tiled(const StepArgs a, const TiledArgs p) {
    extern __shared__ __align__(128) char smem[];
    uint64_t *full = reinterpret_cast<uint64_t *>(smem);
    uint64_t *empty = full + p.ns;
    if (threadIdx.x == 0) {
        for (int s = 0; s < p.ns; ++s) {
            mbar_init(&full[s], 32);
            mbar_init(&empty[s], Geo<DIM, WPR>::NCW);
        }
        *reinterpret_cast<int *>(smem + kAbortOff) = 0;
        mbar_init(reinterpret_cast<uint64_t *>(smem + kStallOff), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    float *wsm = reinterpret_cast<float *>(smem + p.wall_off);
    for (int j = threadIdx.x; j < p.nwd * p.tw; j += blockDim.x) wsm[j] = 0.f;
    if constexpr (!kAccRegs<DIM>) {
        float *accsm = reinterpret_cast<float *>(smem + p.acc_off);
        for (int j = threadIdx.x; j < p.tcells; j += blockDim.x) accsm[j] = 0.f;
    }
    __syncthreads();
    const int warp = (int)(threadIdx.x >> 5);
    if (warp >= Geo<DIM, WPR>::NCW) {
        asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(Geo<DIM, WPR>::RP));
        if (warp == Geo<DIM, WPR>::NCW) producer<S, VL, WPR, DIM>(a, p, smem, full, empty);
    } else {
        asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(Geo<DIM, WPR>::RC));
        consumer<S, LIM, VL, WPR, DIM, SR>(a, p, smem, full, empty);
    }
}

typedef void (*StepKernel)(const StepArgs, const TiledArgs);

// row capacity 64: VL 2, one warp per row; 96: VL 3, one warp; 128: VL 4, one warp; 256 (2-D
// only): VL 4, two warps
template <int S, int LIM, int DIM, bool SR>
StepKernel pick_nx(int nx) {
    if (nx == 64) return k_step_tiled<S, LIM, 2, 1, DIM, SR>;
    if (nx == 96) return k_step_tiled<S, LIM, 3, 1, DIM, SR>;
    if (nx == 128) return k_step_tiled<S, LIM, 4, 1, DIM, SR>;
    if constexpr (DIM == 2) {
        if (nx == 256) return k_step_tiled<S, LIM, 4, 2, DIM, SR>;
    }
    return nullptr;
}

template <int S, int DIM, bool SR>
StepKernel pick_instance(int lim, int nx) {
    if (lim == kLimFirst) return pick_nx<S, kLimFirst, DIM, SR>(nx);
    if (lim == kLimMinmod) return pick_nx<S, kLimMinmod, DIM, SR>(nx);
    return pick_nx<S, kLimVanAlbada, DIM, SR>(nx);
}

// one definition per instantiation unit (sr: stochastic rounding of 16-bit codes)
StepKernel pick_f32_2d(int lim, int nx);
StepKernel pick_f32_3d(int lim, int nx);
StepKernel pick_f16_2d(int lim, int nx, bool sr);
StepKernel pick_f16_3d(int lim, int nx, bool sr);
StepKernel pick_bf16_2d(int lim, int nx, bool sr);
StepKernel pick_bf16_3d(int lim, int nx, bool sr);
StepKernel pick_f16sr_2d(int lim, int nx);
StepKernel pick_f16sr_3d(int lim, int nx);
StepKernel pick_bf16sr_2d(int lim, int nx);
StepKernel pick_bf16sr_3d(int lim, int nx);

}  // namespace tiled
}  // namespace bte
