// Device code of the tiled forward kernel (the design is described in bte_tiled.cu); included
// by the instantiation units bte_tiled_<storage>_<dim>d.cu so the instances compile in parallel.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "bte_tiled.h"

namespace bte {
namespace tiled {

constexpr int kR = 4;                                 // rows streamed by one warp
constexpr unsigned long long kWaitLimitNs = 2000000000ull;  // 2 s
constexpr int kHdrFloats = 16;                        // per-plane constants written by the producer

// Tile geometry: a lane holds VL consecutive cells of a row, WPR warps cover a row of
// nx = 32 VL WPR cells; NCW consumer warps stream kR rows each; 2-D tiles are TY rows, 3-D
// tiles TY rows by TZ slices.  2-D CTAs run 16 consumer warps (96 registers a thread), 3-D
// ones 12 (128 registers; the z-stencil needs more live values).
template <int DIM, int WPR> struct Geo;
template <int WPR> struct Geo<2, WPR> {
    static constexpr int NCW = 16, TZ = 1, TY = NCW / WPR * kR;
};
template <> struct Geo<3, 1> {
    static constexpr int NCW = 12, TZ = 6, TY = NCW / TZ * kR;
};

template <int S> struct St;
template <> struct St<kStoreF32> {
    using T = float;
    static __device__ __forceinline__ float dec(T h, float) { return h; }
    static __device__ __forceinline__ T enc(float v, float) { return v; }
};
template <> struct St<kStoreF16> {
    using T = __half;
    static __device__ __forceinline__ float dec(T h, float sc) { return sc * __half2float(h); }
    static __device__ __forceinline__ T enc(float v, float inv) { return __float2half_rn(v * inv); }
};
template <> struct St<kStoreBF16> {
    using T = __nv_bfloat16;
    static __device__ __forceinline__ float dec(T h, float sc) { return sc * __bfloat162float(h); }
    static __device__ __forceinline__ T enc(float v, float inv) { return __float2bfloat16_rn(v * inv); }
};

// Limiter with an approximate division; pairs with ab below 1e-30 get a zero slope, which
// keeps the denominator a normal number.
template <int LIM> __device__ __forceinline__ float lim(float a, float b);
template <> __device__ __forceinline__ float lim<kLimFirst>(float, float) { return 0.f; }
template <> __device__ __forceinline__ float lim<kLimMinmod>(float a, float b) {
    return (a * b > 0.f) ? (fabsf(a) < fabsf(b) ? a : b) : 0.f;
}
template <> __device__ __forceinline__ float lim<kLimVanAlbada>(float a, float b) {
    const float ab = a * b;
    return ab > 1e-30f ? __fdividef(ab * (a + b), fmaf(a, a, b * b)) : 0.f;
}
// face value e_m + L(e_m - e_l, e_r - e_m) / 2 at the upwind cell m
template <int LIM> __device__ __forceinline__ float face(float ul, float um, float ur) {
    return fmaf(0.5f, lim<LIM>(um - ul, ur - um), um);
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
// Wait for phase `parity` of the barrier, giving up after kWaitLimitNs: the error word gets
// `code` and the caller stops its work.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, int *err, int code) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = gtimer();
    while (!mbar_try_wait(bar, parity)) {
        if (gtimer() - t0 > kWaitLimitNs) {
            atomicOr(err, code);
            return false;
        }
    }
    return true;
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     su32(dst)),
                 "l"(src), "r"(bytes), "r"(su32(bar))
                 : "memory");
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
template <int NCW>
__device__ __forceinline__ void consumer_sync() { asm volatile("bar.sync 1, %0;" ::"n"(NCW * 32) : "memory"); }

// ---- VL-wide loads and stores ---------------------------------------------------------------
template <int S, int VL>
__device__ __forceinline__ void ld_row(float (&v)[VL], const typename St<S>::T *p, float sc) {
    using T = typename St<S>::T;
    constexpr int B = VL * (int)sizeof(T);
    if constexpr (B == 16) {
        const uint4 q = *reinterpret_cast<const uint4 *>(p);
        const T *h = reinterpret_cast<const T *>(&q);
        #pragma unroll
        for (int j = 0; j < VL; ++j) v[j] = St<S>::dec(h[j], sc);
    } else if constexpr (B == 8) {
        const uint2 q = *reinterpret_cast<const uint2 *>(p);
        const T *h = reinterpret_cast<const T *>(&q);
        #pragma unroll
        for (int j = 0; j < VL; ++j) v[j] = St<S>::dec(h[j], sc);
    } else {
        #pragma unroll
        for (int j = 0; j < VL; ++j) v[j] = St<S>::dec(p[j], sc);
    }
}

template <int S, int VL>
__device__ __forceinline__ void st_row(typename St<S>::T *p, const typename St<S>::T (&h)[VL]) {
    constexpr int B = VL * (int)sizeof(typename St<S>::T);
    if constexpr (B == 16) {
        *reinterpret_cast<uint4 *>(p) = *reinterpret_cast<const uint4 *>(h);
    } else if constexpr (B == 8) {
        *reinterpret_cast<uint2 *>(p) = *reinterpret_cast<const uint2 *>(h);
    } else {
        #pragma unroll
        for (int j = 0; j < VL; ++j) p[j] = h[j];
    }
}

// ---- plane-tile decoding ---------------------------------------------------------------------
struct PT {
    int tile, k, d, plane, y0, z0, nyt, nzt;
};

template <int DIM, int WPR>
__device__ __forceinline__ PT decode(const StepArgs &a, const TiledArgs &p, int t) {
    PT r;
    const int npl = a.nb * a.nd;
    r.tile = t / npl;
    r.plane = t - r.tile * npl;
    r.k = r.plane / a.nd;
    r.d = r.plane - r.k * a.nd;
    const int ty = r.tile % p.nty, tz = r.tile / p.nty;
    r.y0 = ty * Geo<DIM, WPR>::TY;
    r.z0 = tz * Geo<DIM, WPR>::TZ;
    r.nyt = min(Geo<DIM, WPR>::TY, a.n[1] - r.y0);
    r.nzt = DIM == 3 ? min(Geo<DIM, WPR>::TZ, a.n[2] - r.z0) : 1;
    return r;
}

// ---- producer warp ----------------------------------------------------------------------------
enum { kSkip = 0, kCopy = 1, kConst = 2 };

// What fills box row (y, z): a bulk copy from src, a constant, or nothing (box corner).
template <int S, int NX, int DIM>
__device__ __forceinline__ int classify_row(const StepArgs &a, const PT &q, int y, int z, float nuy, float nuz,
                                            const typename St<S>::T *&src, float &cval) {
    using T = typename St<S>::T;
    const int ny = a.n[1], nz = a.n[2];
    const bool inY = y >= 0 && y < ny;
    const bool inZ = DIM == 2 || (z >= 0 && z < nz);
    const bool coreY = y >= q.y0 && y < q.y0 + q.nyt;
    const bool coreZ = DIM == 2 || (z >= q.z0 && z < q.z0 + q.nzt);
    if (!coreY && !coreZ) return kSkip;  // box corner: no stencil reads it
    const T *e = static_cast<const T *>(a.e_in);
    const long long pbase = (long long)q.plane * a.ncell;
    if (inY && inZ) {
        src = e + pbase + ((long long)z * ny + y) * NX;
        return kCopy;
    }
    const int ax = inY ? 2 : 1;
    const int pos = ax == 1 ? y : z;
    const int n = ax == 1 ? ny : nz;
    const int side = pos < 0 ? 0 : 1;
    const int wall = 2 * ax + side;
    const int bc = a.bc[wall];
    const float nu = ax == 1 ? nuy : nuz;
    auto row_at = [&](long long base, int yy, int zz) { return e + base + ((long long)zz * ny + yy) * NX; };
    if (bc == kBcPeriodic) {
        const int p2 = side ? pos - n : pos + n;
        src = ax == 1 ? row_at(pbase, p2, z) : row_at(pbase, y, p2);
        return kCopy;
    }
    if (bc == kBcSpecular) {
        const int layer = side ? pos - n + 1 : -pos;
        const int mpos = side ? n - layer : layer - 1;
        const long long mbase = ((long long)q.k * a.nd + a.mirror[ax * a.nd + q.d]) * a.ncell;
        src = ax == 1 ? row_at(mbase, mpos, z) : row_at(mbase, y, mpos);
        return kCopy;
    }
    const bool incoming = side == 0 ? (nu > 0.f) : (nu < 0.f);
    if (!incoming) {
        const int wpos = side ? n - 1 : 0;
        src = ax == 1 ? row_at(pbase, wpos, z) : row_at(pbase, y, wpos);
        return kCopy;
    }
    if (bc == kBcIsothermal) {
        cval = a.iso[wall * a.nb + q.k];
        return kConst;
    }
    // diffuse wall: the row of incoming values (wall cells of a y-wall are indexed z*nx + x,
    // those of a z-wall y*nx + x)
    src = static_cast<const T *>(a.ediff_in) + ((long long)wall * a.nb + q.k) * a.wc_max + (long long)(ax == 1 ? z : y) * NX;
    return kCopy;
}

template <int S, int VL, int WPR, int DIM>
__device__ void producer(const StepArgs &a, const TiledArgs &p, char *smem, uint64_t *full, uint64_t *empty, int t0,
                         int t1) {
    using T = typename St<S>::T;
    constexpr int NX = 32 * VL * WPR, TY = Geo<DIM, WPR>::TY;
    constexpr uint32_t rowb = NX * sizeof(T);
    const int lane = threadIdx.x & 31;
    const int ny = a.n[1];
    const T *e = static_cast<const T *>(a.e_in);
    const T *ed = static_cast<const T *>(a.ediff_in);
    int i = 0;
    for (int t = t0; t < t1; ++t, ++i) {
        const int s = i % p.ns;
        const uint32_t ph = (uint32_t)(i / p.ns) & 1u;
        if (i >= p.ns && !mbar_wait(&empty[s], ph ^ 1u, p.err, 2)) return;
        fence_proxy_async();
        __syncwarp();
        const PT q = decode<DIM, WPR>(a, p, t);
        const float nux = a.nu[3 * q.plane], nuy = a.nu[3 * q.plane + 1];
        const float nuz = DIM == 3 ? a.nu[3 * q.plane + 2] : 0.f;
        const int ybox0 = q.y0 - (nuy > 0.f ? 2 : 1);
        const int zbox0 = DIM == 3 ? q.z0 - (nuz > 0.f ? 2 : 1) : 0;
        const int nrow = (q.nyt + 3) * (DIM == 3 ? q.nzt + 3 : 1);
        char *stage = smem + p.stage0 + (size_t)s * p.stage_bytes;
        const BandConst b = a.band[q.k];
        // bytes the bulk copies of this stage deliver
        uint32_t bytes = 0;
        for (int r = lane; r < nrow; r += 32) {
            const T *src;
            float cv;
            if (classify_row<S, NX, DIM>(a, q, ybox0 + r % (q.nyt + 3), zbox0 + r / (q.nyt + 3), nuy, nuz, src, cv) ==
                kCopy)
                bytes += rowb;
        }
        bytes = __reduce_add_sync(0xffffffffu, bytes);
        if (lane == 0) mbar_expect_tx(&full[s], bytes);
        __syncwarp();
        for (int base = 0; base < nrow; base += 32) {
            const int r = base + lane;
            const T *src = nullptr;
            float cv = 0.f;
            const int kind = r < nrow ? classify_row<S, NX, DIM>(a, q, ybox0 + r % (q.nyt + 3),
                                                                   zbox0 + r / (q.nyt + 3), nuy, nuz, src, cv)
                                      : kSkip;
            // box rows are stored with the full-tile stride: row (ry, rz) at (rz (TY + 3) + ry) NX
            if (kind == kCopy)
                bulk_g2s(reinterpret_cast<T *>(stage) + ((size_t)(r / (q.nyt + 3)) * (TY + 3) + r % (q.nyt + 3)) * NX,
                         src, rowb, &full[s]);
            // thermalizing-wall rows: the whole warp writes each one, 16 bytes per lane and store
            unsigned m = __ballot_sync(0xffffffffu, kind == kConst);
            while (m) {
                const int j = __ffs(m) - 1;
                m &= m - 1;
                const float v = __shfl_sync(0xffffffffu, cv, j);
                const T h = St<S>::enc(v, b.inv_scale);
                T pack[16 / sizeof(T)];
                #pragma unroll
                for (int c = 0; c < (int)(16 / sizeof(T)); ++c) pack[c] = h;
                const int rj = base + j;
                uint4 *row = reinterpret_cast<uint4 *>(reinterpret_cast<T *>(stage) +
                                                       ((size_t)(rj / (q.nyt + 3)) * (TY + 3) + rj % (q.nyt + 3)) * NX);
                for (int c = lane; c < (int)(rowb / 16); c += 32) row[c] = *reinterpret_cast<const uint4 *>(pack);
            }
        }
        // x-wall ghosts that are not in the tile: specular (mirror plane at x = 0, 1 / nx-1, nx-2)
        // and diffuse incoming values; four floats per core row
        const int bx0 = a.bc[0], bx1 = a.bc[1];
        if (bx0 == kBcSpecular || bx0 == kBcDiffuse || bx1 == kBcSpecular || bx1 == kBcDiffuse) {
            float *side = reinterpret_cast<float *>(stage + p.side_off);
            for (int j = lane; j < q.nyt * q.nzt; j += 32) {
                const int yl = j % q.nyt, zl = j / q.nyt;
                const int y = q.y0 + yl, z = q.z0 + zl;
                const long long rowoff = ((long long)z * ny + y) * NX;
                float g[4] = {0.f, 0.f, 0.f, 0.f};
                #pragma unroll
                for (int sd = 0; sd < 2; ++sd) {
                    const int bc = sd ? bx1 : bx0;
                    if (bc == kBcSpecular) {
                        const long long mb = ((long long)q.k * a.nd + a.mirror[q.d]) * a.ncell + rowoff;
                        g[2 * sd] = St<S>::dec(e[mb + (sd ? NX - 1 : 0)], b.scale);
                        g[2 * sd + 1] = St<S>::dec(e[mb + (sd ? NX - 2 : 1)], b.scale);
                    } else if (bc == kBcDiffuse && (sd ? nux < 0.f : nux > 0.f)) {
                        const float v = St<S>::dec(ed[((long long)sd * a.nb + q.k) * a.wc_max + (long long)z * ny + y], b.scale);
                        g[2 * sd] = g[2 * sd + 1] = v;
                    }
                }
                *reinterpret_cast<float4 *>(side + ((size_t)zl * TY + yl) * 4) = make_float4(g[0], g[1], g[2], g[3]);
            }
        }
        // per-plane constants for the consumers
        if (lane == 0) {
            float *hd = reinterpret_cast<float *>(stage + p.hdr_off);
            hd[0] = nux;
            hd[1] = nuy;
            hd[2] = nuz;
            hd[3] = a.wmom[q.plane];
            hd[4] = b.dtinv;
            hd[5] = b.scale;
            hd[6] = b.inv_scale;
            hd[7] = a.iso[0 * a.nb + q.k];
            hd[8] = a.iso[1 * a.nb + q.k];
            #pragma unroll
            for (int w = 0; w < 6; ++w) hd[9 + w] = (w < 2 * DIM && a.bc[w] == kBcDiffuse) ? a.wdiff[w * a.nd + q.d] : 0.f;
            hd[15] = 0.f;
        }
        mbar_arrive(&full[s]);
    }
}

// ---- consumer warps -----------------------------------------------------------------------
template <int S, int LIM, int VL, int WPR, int DIM, int SY>
__device__ __forceinline__ void rows_of_warp(const StepArgs &a, const TiledArgs &p, const PT &q, const char *stage,
                                             int zl, int rb, int half, float (&acc)[kR][VL], const float *btsm,
                                             float *wsm) {
    using T = typename St<S>::T;
    constexpr int NX = 32 * VL * WPR, TY = Geo<DIM, WPR>::TY;
    const int lane = threadIdx.x & 31, x0 = (half * 32 + lane) * VL;
    const int ny = a.n[1], nz = a.n[2];
    const float *hd = reinterpret_cast<const float *>(stage + p.hdr_off);  // per-plane constants
    const float4 h0 = reinterpret_cast<const float4 *>(hd)[0];
    const float nux = h0.x, nuy = h0.y, nuz = h0.z, wm = h0.w;
    const float dtinv = hd[4], sc = hd[5], isc = hd[6];
    const float any = fabsf(nuy), anz = fabsf(nuz);
    const int sz = nuz > 0.f ? 1 : -1;
    const int ybox0 = q.y0 - (SY > 0 ? 2 : 1);
    const int zbox0 = DIM == 3 ? q.z0 - (nuz > 0.f ? 2 : 1) : 0;
    const int z = q.z0 + zl;
    const int rz = z - zbox0;
    const T *box = reinterpret_cast<const T *>(stage);
    const float *side = reinterpret_cast<const float *>(stage + p.side_off);
    auto rowbase = [&](int y, int zr) { return box + ((size_t)zr * (TY + 3) + (y - ybox0)) * NX; };
    const int bx0 = a.bc[0], bx1 = a.bc[1];
    const bool left_edge = lane == 0, right_edge = lane == 31;
    const bool xlo = left_edge && half == 0, xhi = right_edge && half == WPR - 1;
    T *eo = static_cast<T *>(a.e_out) + (long long)q.plane * a.ncell;

    float wm2[VL], wm1[VL], w0[VL], wp1[VL], fin[VL];
    bool started = false;
    #pragma unroll
    for (int jj = 0; jj < kR; ++jj) {
        const int r = SY > 0 ? jj : kR - 1 - jj;  // row of the warp, compile-time after unrolling
        const int yl = rb + r;
        if (yl >= q.nyt) continue;  // ragged tile (uniform across the warp)
        const int y = q.y0 + yl;
        const T *rb0 = rowbase(y, rz);
        if (!started) {
            ld_row<S, VL>(wm2, rowbase(y - 2 * SY, rz) + x0, sc);
            ld_row<S, VL>(wm1, rowbase(y - SY, rz) + x0, sc);
            ld_row<S, VL>(w0, rb0 + x0, sc);
            #pragma unroll
            for (int v = 0; v < VL; ++v) fin[v] = face<LIM>(wm2[v], wm1[v], w0[v]);
            started = true;
        }
        ld_row<S, VL>(wp1, rowbase(y + SY, rz) + x0, sc);
        float div[VL], fout[VL];
        // y: out face between y and y + SY (upwind y); the in face is the previous row's out face
        #pragma unroll
        for (int v = 0; v < VL; ++v) {
            fout[v] = face<LIM>(wm1[v], w0[v], wp1[v]);
            div[v] = any * (fout[v] - fin[v]);
        }
        // x: neighbours from the adjacent lanes; at a warp's two ends from shared memory (the
        // neighbouring warp's cells, or the periodic wrap), at the domain walls the ghosts
        float ex[VL + 4];
        #pragma unroll
        for (int v = 0; v < VL; ++v) ex[v + 2] = w0[v];
        ex[0] = __shfl_sync(0xffffffffu, w0[VL - 2], (lane + 31) & 31);
        ex[1] = __shfl_sync(0xffffffffu, w0[VL - 1], (lane + 31) & 31);
        ex[VL + 2] = __shfl_sync(0xffffffffu, w0[0], (lane + 1) & 31);
        ex[VL + 3] = __shfl_sync(0xffffffffu, w0[1], (lane + 1) & 31);
        if (left_edge) {
            if (!xlo) {
                ex[0] = St<S>::dec(rb0[x0 - 2], sc);
                ex[1] = St<S>::dec(rb0[x0 - 1], sc);
            } else if (bx0 == kBcPeriodic) {
                ex[0] = St<S>::dec(rb0[NX - 2], sc);
                ex[1] = St<S>::dec(rb0[NX - 1], sc);
            } else {
                const float *g = side + ((size_t)zl * TY + yl) * 4;
                if (bx0 == kBcSpecular) { ex[1] = g[0]; ex[0] = g[1]; }
                else if (nux <= 0.f) { ex[1] = ex[0] = w0[0]; }
                else if (bx0 == kBcIsothermal) { ex[1] = ex[0] = hd[7]; }
                else { ex[1] = ex[0] = g[0]; }
            }
        }
        if (right_edge) {
            if (!xhi) {
                ex[VL + 2] = St<S>::dec(rb0[x0 + VL], sc);
                ex[VL + 3] = St<S>::dec(rb0[x0 + VL + 1], sc);
            } else if (bx1 == kBcPeriodic) {
                ex[VL + 2] = St<S>::dec(rb0[0], sc);
                ex[VL + 3] = St<S>::dec(rb0[1], sc);
            } else {
                const float *g = side + ((size_t)zl * TY + yl) * 4;
                if (bx1 == kBcSpecular) { ex[VL + 2] = g[2]; ex[VL + 3] = g[3]; }
                else if (nux >= 0.f) { ex[VL + 2] = ex[VL + 3] = w0[VL - 1]; }
                else if (bx1 == kBcIsothermal) { ex[VL + 2] = ex[VL + 3] = hd[8]; }
                else { ex[VL + 2] = ex[VL + 3] = g[2]; }
            }
        }
        // faces F_j between x0+j and x0+j+1, j = -1..VL-1 (index j+1); flux in signed form
        float F[VL + 1];
        if (nux > 0.f) {
            #pragma unroll
            for (int j = -1; j < VL; ++j) F[j + 1] = face<LIM>(ex[j + 1], ex[j + 2], ex[j + 3]);
        } else {
            #pragma unroll
            for (int j = -1; j < VL; ++j) F[j + 1] = face<LIM>(ex[j + 4], ex[j + 3], ex[j + 2]);
        }
        #pragma unroll
        for (int v = 0; v < VL; ++v) div[v] = fmaf(nux, F[v + 1] - F[v], div[v]);
        if constexpr (DIM == 3) {
            float zm1[VL], zm2[VL], zp1[VL];
            ld_row<S, VL>(zm1, rowbase(y, rz - sz) + x0, sc);
            ld_row<S, VL>(zm2, rowbase(y, rz - 2 * sz) + x0, sc);
            ld_row<S, VL>(zp1, rowbase(y, rz + sz) + x0, sc);
            #pragma unroll
            for (int v = 0; v < VL; ++v) div[v] = fmaf(anz, face<LIM>(zm1[v], w0[v], zp1[v]) - face<LIM>(zm2[v], zm1[v], w0[v]), div[v]);
        }
        // update, store, moment and diffuse-wall partials
        float bt[VL];
        {
            const float *bp = btsm + ((size_t)zl * TY + yl) * NX + x0;
            if constexpr (VL == 4) {
                const float4 f = *reinterpret_cast<const float4 *>(bp);
                bt[0] = f.x;
                bt[1] = f.y;
                bt[2] = f.z;
                bt[3] = f.w;
            } else {
                #pragma unroll
                for (int v = 0; v < VL; ++v) bt[v] = bp[v];
            }
        }
        T h[VL];
        float es[VL];
        #pragma unroll
        for (int v = 0; v < VL; ++v) {
            const float en = fmaf(-dtinv, w0[v], w0[v] - div[v]) + bt[v];
            h[v] = St<S>::enc(en, isc);
            es[v] = St<S>::dec(h[v], sc);
            acc[r][v] = fmaf(wm, es[v], acc[r][v]);
        }
        st_row<S, VL>(eo + ((long long)z * ny + y) * NX + x0, h);
        // diffuse-wall sums of Eq. (diff_bound) for the next step: cells next to a diffuse wall
        // add w_d (s_d.n) e for directions leaving through it (weight 0 otherwise)
        if (xlo && hd[9] != 0.f) wsm[p.wslot[0] * p.tw + zl * TY + yl] += hd[9] * es[0];
        if (xhi && hd[10] != 0.f) wsm[p.wslot[1] * p.tw + zl * TY + yl] += hd[10] * es[VL - 1];
        if (y == 0 && hd[11] != 0.f) {
            float *w = wsm + p.wslot[2] * p.tw + zl * NX + x0;
            #pragma unroll
            for (int v = 0; v < VL; ++v) w[v] += hd[11] * es[v];
        }
        if (y == ny - 1 && hd[12] != 0.f) {
            float *w = wsm + p.wslot[3] * p.tw + zl * NX + x0;
            #pragma unroll
            for (int v = 0; v < VL; ++v) w[v] += hd[12] * es[v];
        }
        if (DIM == 3 && z == 0 && hd[13] != 0.f) {
            float *w = wsm + p.wslot[4] * p.tw + yl * NX + x0;
            #pragma unroll
            for (int v = 0; v < VL; ++v) w[v] += hd[13] * es[v];
        }
        if (DIM == 3 && z == nz - 1 && hd[14] != 0.f) {
            float *w = wsm + p.wslot[5] * p.tw + yl * NX + x0;
            #pragma unroll
            for (int v = 0; v < VL; ++v) w[v] += hd[14] * es[v];
        }
        #pragma unroll
        for (int v = 0; v < VL; ++v) {
            wm2[v] = wm1[v];
            wm1[v] = w0[v];
            w0[v] = wp1[v];
            fin[v] = fout[v];
        }
    }
}

template <int VL, int WPR, int DIM>
__device__ __forceinline__ void warp_place(int &zl, int &rb, int &half) {
    const int warp = threadIdx.x >> 5;
    half = warp % WPR;
    const int u = warp / WPR;
    zl = u % Geo<DIM, WPR>::TZ;
    rb = (u / Geo<DIM, WPR>::TZ) * kR;
}

template <int VL, int WPR, int DIM>
__device__ __forceinline__ void flush_segment(const StepArgs &a, const TiledArgs &p, int seg, const PT &q,
                                              float (&acc)[kR][VL], float *wsm) {
    constexpr int NX = 32 * VL * WPR, TY = Geo<DIM, WPR>::TY;
    int zl, rb, half;
    warp_place<VL, WPR, DIM>(zl, rb, half);
    const int x0 = (half * 32 + (threadIdx.x & 31)) * VL;
    float *P = a.P + (size_t)seg * p.tcells;
    #pragma unroll
    for (int r = 0; r < kR; ++r) {
        const int yl = rb + r;
        if (yl < q.nyt && zl < q.nzt) {
            #pragma unroll
            for (int v = 0; v < VL; ++v) P[((size_t)zl * TY + yl) * NX + x0 + v] = acc[r][v];
        }
        #pragma unroll
        for (int v = 0; v < VL; ++v) acc[r][v] = 0.f;
    }
    constexpr int NCW = Geo<DIM, WPR>::NCW;
    consumer_sync<NCW>();
    for (int idx = threadIdx.x; idx < p.nwd * p.tw; idx += NCW * 32) {
        p.PW[(size_t)seg * p.nwd * p.tw + idx] = wsm[idx];
        wsm[idx] = 0.f;
    }
    consumer_sync<NCW>();
}

template <int S, int LIM, int VL, int WPR, int DIM>
__device__ void consumer(const StepArgs &a, const TiledArgs &p, char *smem, uint64_t *full, uint64_t *empty, int t0,
                         int t1, int seg0) {
    constexpr int NX = 32 * VL * WPR, TY = Geo<DIM, WPR>::TY;
    const int lane = threadIdx.x & 31;
    int zl, rb, half;
    warp_place<VL, WPR, DIM>(zl, rb, half);
    const int x0 = (half * 32 + lane) * VL;
    const int ny = a.n[1];
    float acc[kR][VL];
    #pragma unroll
    for (int r = 0; r < kR; ++r)
        #pragma unroll
        for (int v = 0; v < VL; ++v) acc[r][v] = 0.f;
    float *wsm = reinterpret_cast<float *>(smem + p.wall_off);
    float *btsm = reinterpret_cast<float *>(smem + p.bt_off);
    int seg = seg0 - 1, cur_tile = -1, cur_band = -1;
    PT cur{};
    int i = 0;
    for (int t = t0; t < t1; ++t, ++i) {
        const PT q = decode<DIM, WPR>(a, p, t);
        if (q.tile != cur_tile || q.k != cur_band) {
            if (seg >= seg0) flush_segment<VL, WPR, DIM>(a, p, seg, cur, acc, wsm);
            ++seg;
            cur_tile = q.tile;
            cur_band = q.k;
            cur = q;
            // per-cell relaxation target and source of this band: dt/tau C T_L / W + a dt C Q/(sum C W)
            const BandConst b = a.band[q.k];
            #pragma unroll
            for (int r = 0; r < kR; ++r) {
                const int yl = rb + r;
                if (yl < q.nyt && zl < q.nzt) {
                    const long long i0 = ((long long)(q.z0 + zl) * ny + (q.y0 + yl)) * NX + x0;
                    float *bp = btsm + ((size_t)zl * TY + yl) * NX + x0;
                    #pragma unroll
                    for (int v = 0; v < VL; ++v) {
                        const float src = a.Q ? b.srck * (a.amp * a.Q[i0 + v]) : 0.f;
                        bp[v] = fmaf(b.dtinv, b.ck * a.TL[i0 + v], src);
                    }
                }
            }
        }
        const int s = i % p.ns;
        const uint32_t ph = (uint32_t)(i / p.ns) & 1u;
        if (!mbar_wait(&full[s], ph, p.err, 1)) return;
        const char *stage = smem + p.stage0 + (size_t)s * p.stage_bytes;
        if (zl < q.nzt && rb < q.nyt) {
            if (a.nu[3 * q.plane + 1] > 0.f)
                rows_of_warp<S, LIM, VL, WPR, DIM, 1>(a, p, q, stage, zl, rb, half, acc, btsm, wsm);
            else
                rows_of_warp<S, LIM, VL, WPR, DIM, -1>(a, p, q, stage, zl, rb, half, acc, btsm, wsm);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
    }
    if (seg >= seg0) flush_segment<VL, WPR, DIM>(a, p, seg, cur, acc, wsm);
}

template <int S, int LIM, int VL, int WPR, int DIM>
__global__ void __launch_bounds__((Geo<DIM, WPR>::NCW + 1) * 32, 1) k_step_tiled(const StepArgs a, const TiledArgs p) {
    extern __shared__ __align__(128) char smem[];
    uint64_t *full = reinterpret_cast<uint64_t *>(smem);
    uint64_t *empty = full + p.ns;
    const int t0 = p.cta_begin[blockIdx.x], t1 = p.cta_begin[blockIdx.x + 1];
    if (threadIdx.x == 0) {
        for (int s = 0; s < p.ns; ++s) {
            mbar_init(&full[s], 32);
            mbar_init(&empty[s], Geo<DIM, WPR>::NCW);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    float *wsm = reinterpret_cast<float *>(smem + p.wall_off);
    for (int j = threadIdx.x; j < p.nwd * p.tw; j += blockDim.x) wsm[j] = 0.f;
    __syncthreads();
    if ((int)(threadIdx.x >> 5) == Geo<DIM, WPR>::NCW)
        producer<S, VL, WPR, DIM>(a, p, smem, full, empty, t0, t1);
    else
        consumer<S, LIM, VL, WPR, DIM>(a, p, smem, full, empty, t0, t1, p.seg_first[blockIdx.x]);
}

typedef void (*StepKernel)(const StepArgs, const TiledArgs);

// nx = 96: VL 3, one warp per row; nx = 128: VL 4, one warp; nx = 256 (2-D only): VL 4, two warps
template <int S, int LIM, int DIM>
StepKernel pick_nx(int nx) {
    if (nx == 96) return k_step_tiled<S, LIM, 3, 1, DIM>;
    if (nx == 128) return k_step_tiled<S, LIM, 4, 1, DIM>;
    if constexpr (DIM == 2) {
        if (nx == 256) return k_step_tiled<S, LIM, 4, 2, DIM>;
    }
    return nullptr;
}

template <int S, int DIM>
StepKernel pick_instance(int lim, int nx) {
    if (lim == kLimFirst) return pick_nx<S, kLimFirst, DIM>(nx);
    if (lim == kLimMinmod) return pick_nx<S, kLimMinmod, DIM>(nx);
    return pick_nx<S, kLimVanAlbada, DIM>(nx);
}

// one definition per instantiation unit
StepKernel pick_f32_2d(int lim, int nx);
StepKernel pick_f32_3d(int lim, int nx);
StepKernel pick_f16_2d(int lim, int nx);
StepKernel pick_f16_3d(int lim, int nx);
StepKernel pick_bf16_2d(int lim, int nx);
StepKernel pick_bf16_3d(int lim, int nx);

}  // namespace tiled
}  // namespace bte
