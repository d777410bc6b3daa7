// Tiled adjoint step (the transpose of the forward step; the algebra is in bte_adjoint.cu), on
// the forward kernel's tiles and plane-synchronous unit schedule.  Included by the
// instantiation units bte_adjoint_tiled_<storage>.cu.
//
// Face form of the transpose: a face with upwind position m (orientation sg along an axis)
// has value F_m = u_m + L(u_m - u_l, u_r - u_m)/2 and enters cell m with -|nu|, cell m+sg with
// +|nu|; with phi_m = |nu| (lambda_{m+sg} - lambda_m) it adds
//   A_m = phi_m dF/du_l to cell m-sg,  B_m = phi_m dF/du_m to cell m,  C_m = phi_m dF/du_r to m+sg.
// The limiter's partials are homogeneous of degree 0, so faces are evaluated on e / s_k
// directly for 16-bit codes.  This kernel takes every face whose three values lie in the
// domain (or wrap on a periodic axis): y faces streamed in registers from upwind to downwind
// (one new face per row), x faces per lane with the neighbour lanes' values and end-face terms
// by shuffles, and in 3-D one z face per cell, shared between neighbouring slices through
// shared memory.  The faces next to a non-periodic wall that read a ghost value (the first
// cell's in-face and out-face, the last cell's out-face) and every ghost transpose are added
// by k_adj_walls afterwards, which keeps this kernel free of wall rules.  2-D rows come
// straight from global memory (neighbouring units' rows are L2-resident); a 3-D plane-tile is
// first staged, with its two-cell halo, in shared memory by all warps together.
#pragma once

#include "bte_adjoint.h"
#include "bte_tiled_kernel.cuh"

namespace bte {
namespace tiled {

template <int LIM> __device__ __forceinline__ void adj_lim_grad(float a, float b, float &La, float &Lb);
template <> __device__ __forceinline__ void adj_lim_grad<kLimFirst>(float, float, float &La, float &Lb) {
    La = Lb = 0.f;
}
template <> __device__ __forceinline__ void adj_lim_grad<kLimMinmod>(float a, float b, float &La, float &Lb) {
    const bool on = a * b > 0.f, pa = fabsf(a) < fabsf(b);
    La = on && pa ? 1.f : 0.f;
    Lb = on && !pa ? 1.f : 0.f;
}
template <> __device__ __forceinline__ void adj_lim_grad<kLimVanAlbada>(float a, float b, float &La, float &Lb) {
    // L = ab(a+b)/(a^2+b^2): dL/da = b^2 (2ab + b^2 - a^2)/(a^2+b^2)^2, symmetric in b
    const float ab = a * b, aa = a * a, bb = b * b;
    const float rq = rcp_approx(aa + bb);
    const float t = 2.f * ab;
    const float la = (bb * rq) * ((t + bb - aa) * rq);
    const float lb = (aa * rq) * ((t + aa - bb) * rq);
    La = ab > 1e-30f ? la : 0.f;
    Lb = ab > 1e-30f ? lb : 0.f;
}

// A, B, C of a face with values (ul, um, ur) and weight phi.
template <int LIM>
__device__ __forceinline__ void face_terms(float ul, float um, float ur, float phi, float &A, float &B, float &C) {
    float La, Lb;
    adj_lim_grad<LIM>(um - ul, ur - um, La, Lb);
    A = -0.5f * La * phi;
    B = fmaf(0.5f * (La - Lb), phi, phi);
    C = 0.5f * Lb * phi;
}

// Row index of position pos along an axis of n cells: itself, the wrapped row on a periodic
// axis, or -1 outside a wall (faces reading it belong to the wall pass).
__device__ __forceinline__ int adj_row(int pos, int n, bool per) {
    if (pos >= 0 && pos < n) return pos;
    if (!per) return -1;
    return pos < 0 ? pos + n : pos - n;
}

// VL values of e (16-bit: e / s_k = h + rho) at global cell index `cell` of plane `base`; rho
// points at the same cells' references R / T_scale in the unit's shared reference box.
template <int S, int VL>
__device__ __forceinline__ void adj_ld_e(float (&v)[VL], const typename St<S>::T *e, long long base, long long cell,
                                         const float *rho) {
    using Q = St<S>;
    if constexpr (!Q::kRef) {
        if constexpr (VL == 4) {
            const float4 f = *reinterpret_cast<const float4 *>(e + base + cell);
            v[0] = f.x; v[1] = f.y; v[2] = f.z; v[3] = f.w;
        } else {
            #pragma unroll
            for (int j = 0; j < VL; ++j) v[j] = e[base + cell + j];
        }
    } else {
        if constexpr (VL == 4) {
            const uint2 q = *reinterpret_cast<const uint2 *>(e + base + cell);
            const float4 r = *reinterpret_cast<const float4 *>(rho);
            v[0] = r.x + Q::val(q.x & 0xffffu);
            v[1] = r.y + Q::val(q.x >> 16);
            v[2] = r.z + Q::val(q.y & 0xffffu);
            v[3] = r.w + Q::val(q.y >> 16);
        } else {
            #pragma unroll
            for (int j = 0; j < VL; ++j) v[j] = rho[j] + Q::val(Q::bits(e[base + cell + j]));
        }
    }
}

template <int VL>
__device__ __forceinline__ void adj_ld_l(float (&v)[VL], const float *lam, long long idx) {
    if constexpr (VL == 4) {
        const float4 f = *reinterpret_cast<const float4 *>(lam + idx);
        v[0] = f.x; v[1] = f.y; v[2] = f.z; v[3] = f.w;
    } else {
        #pragma unroll
        for (int j = 0; j < VL; ++j) v[j] = lam[idx + j];
    }
}

// One value of e / s_k (or lambda) at x position xp of a row (used by the end lanes of a warp).
template <int S>
__device__ __forceinline__ float adj_e1(const StepArgs &a, const typename St<S>::T *e, long long base, long long cell) {
    using Q = St<S>;
    if constexpr (!Q::kRef) return e[base + cell];
    else return fmaf(a.R[cell], a.invTs, Q::val(Q::bits(e[base + cell])));
}

// x faces of one lane: upwind cell m = x0-1+f, f = 0 .. VL+1 (orientation SX); index i of ex /
// lx is position x0-2+i.  A face is taken when its three values are in the domain or wrap.
// Cell x0+j (face index j+1) gets A of face x0+j+SX, B of face x0+j, C of face x0+j-SX.
template <int LIM, int VL, int SX>
__device__ __forceinline__ void adj_xfaces(const float (&ex)[VL + 4], const float (&lx)[VL + 4], int x0, int NX,
                                           bool perx, float anx, float (&acc)[VL]) {
    float fA[VL + 2], fB[VL + 2], fC[VL + 2];
    #pragma unroll
    for (int f = 0; f < VL + 2; ++f) {
        const int m = x0 - 1 + f;
        const bool ok = perx || (m >= 1 && m + 1 < NX);
        float A = 0.f, B = 0.f, C = 0.f;
        if (ok) face_terms<LIM>(ex[f + 1 - SX], ex[f + 1], ex[f + 1 + SX], anx * (lx[f + 1 + SX] - lx[f + 1]), A, B, C);
        fA[f] = A;
        fB[f] = B;
        fC[f] = C;
    }
    #pragma unroll
    for (int j = 0; j < VL; ++j) acc[j] += fA[j + 1 + SX] + fB[j + 1] + fC[j + 1 - SX];
}

// x faces of one lane when one warp covers a row (WPR = 1): the lane takes the faces whose
// upwind cells are its own, x0 .. x0+VL-1, and receives by shuffle the one term of each
// neighbour lane's end face that lands on its cells (the A of the face downwind of its last
// cell ... in orientation SX: cell x0+j gets A of face x0+j+SX, B of face x0+j, C of face
// x0+j-SX).  The row's two ends meet by the same shuffles, which is the wrap of a periodic
// axis; on a wall axis those end faces read ghost values and belong to the wall pass (zero).
template <int LIM, int VL, int SX>
__device__ __forceinline__ void adj_xfaces_w(const float (&e0)[VL], const float (&l0)[VL], int x0, int NX, bool perx,
                                             float anx, int lane, float (&acc)[VL]) {
    const int lft = (lane + 31) & 31, rgt = (lane + 1) & 31;
    float ex[VL + 2], lx[VL + 2];  // positions x0-1 .. x0+VL
    #pragma unroll
    for (int j = 0; j < VL; ++j) {
        ex[j + 1] = e0[j];
        lx[j + 1] = l0[j];
    }
    ex[0] = __shfl_sync(0xffffffffu, e0[VL - 1], lft);
    ex[VL + 1] = __shfl_sync(0xffffffffu, e0[0], rgt);
    if constexpr (SX > 0) {
        lx[VL + 1] = __shfl_sync(0xffffffffu, l0[0], rgt);
        lx[0] = 0.f;
    } else {
        lx[0] = __shfl_sync(0xffffffffu, l0[VL - 1], lft);
        lx[VL + 1] = 0.f;
    }
    float fA[VL], fB[VL], fC[VL];
    #pragma unroll
    for (int f = 0; f < VL; ++f) {
        const int m = x0 + f;
        const bool ok = perx || (m >= 1 && m + 1 < NX);
        float A = 0.f, B = 0.f, C = 0.f;
        if (ok) face_terms<LIM>(ex[f + 1 - SX], ex[f + 1], ex[f + 1 + SX], anx * (lx[f + 1 + SX] - lx[f + 1]), A, B, C);
        fA[f] = A;
        fB[f] = B;
        fC[f] = C;
    }
    // A of the face at x0+VL-1+SX... from the lane downwind, C of the face upwind from the lane upwind
    float nA = __shfl_sync(0xffffffffu, SX > 0 ? fA[0] : fA[VL - 1], SX > 0 ? rgt : lft);
    float nC = __shfl_sync(0xffffffffu, SX > 0 ? fC[VL - 1] : fC[0], SX > 0 ? lft : rgt);
    if (!perx) {
        if (lane == (SX > 0 ? 31 : 0)) nA = 0.f;
        if (lane == (SX > 0 ? 0 : 31)) nC = 0.f;
    }
    #pragma unroll
    for (int j = 0; j < VL; ++j) {
        const float ta = SX > 0 ? (j + 1 < VL ? fA[j + 1 < VL ? j + 1 : 0] : nA) : (j >= 1 ? fA[j >= 1 ? j - 1 : 0] : nA);
        const float tc = SX > 0 ? (j >= 1 ? fC[j >= 1 ? j - 1 : 0] : nC) : (j + 1 < VL ? fC[j + 1 < VL ? j + 1 : 0] : nC);
        acc[j] += ta + fB[j] + tc;
    }
}

struct AdjTiledArgs {
    const float *lam_in;  // lambda^{n+1}
    float *lam_out;       // lambda^n
    const float *mu_in;   // mu^{n+1} [ncell]
    float *Pm, *Pq;       // per segment rows [G][tcells]: sum_d lambda^n dt C_k/(W tau_k), sum_d lambda^n dt C_k/(sum C W)
    float *Ps;            // per segment [G][2]: sum lambda^{n+1} (C_k T_L/W - e), sum w_d mu^{n+1} e
    const float *w;       // [nd]
    int cache_r;          // 16-bit references of the unit's box held in shared memory
    int cache_mt;         // mu^{n+1} and T_L^n of the unit's tile held in shared memory
};

// lambda^n of VL cells to global memory, and their per-cell partials of mu and of the source
// gradient (four contiguous floats per lane move as one 16-byte access, free of bank conflicts)
template <int VL>
__device__ __forceinline__ void adj_emit(const AdjTiledArgs &g, float *accm, float *accq, int c, long long gi, float bm,
                                         float bq, const float (&out)[VL]) {
    if constexpr (VL == 4) {
        float4 m = *reinterpret_cast<float4 *>(accm + c), qq = *reinterpret_cast<float4 *>(accq + c);
        m.x = fmaf(bm, out[0], m.x); m.y = fmaf(bm, out[1], m.y); m.z = fmaf(bm, out[2], m.z); m.w = fmaf(bm, out[3], m.w);
        qq.x = fmaf(bq, out[0], qq.x); qq.y = fmaf(bq, out[1], qq.y); qq.z = fmaf(bq, out[2], qq.z); qq.w = fmaf(bq, out[3], qq.w);
        *reinterpret_cast<float4 *>(accm + c) = m;
        *reinterpret_cast<float4 *>(accq + c) = qq;
        *reinterpret_cast<float4 *>(g.lam_out + gi) = make_float4(out[0], out[1], out[2], out[3]);
    } else {
        #pragma unroll
        for (int j = 0; j < VL; ++j) {
            accm[c + j] = fmaf(bm, out[j], accm[c + j]);
            accq[c + j] = fmaf(bq, out[j], accq[c + j]);
            g.lam_out[gi + j] = out[j];
        }
    }
}

// 2-D: the rows one warp streams for one plane-tile, values straight from global memory (the
// 16-bit references, mu and T_L from the unit's shared copies).
template <int S, int LIM, int VL, int WPR, int DIM>
__device__ __forceinline__ void adj_rows(const StepArgs &a, const AdjTiledArgs &g, const PT &q, int zl, int rb, int half,
                                         float *accm, float *accq, float &s1, float &s2, const float *rbox,
                                         const float *mtbox) {
    static_assert(DIM == 2, "3-D plane-tiles go through adj_tile3");
    using T = typename St<S>::T;
    constexpr int NX = 32 * VL * WPR, TY = Geo<DIM, WPR>::TY;
    const int lane = threadIdx.x & 31, x0 = (half * 32 + lane) * VL;
    const int ny = a.n[1];
    const int plane = q.plane;
    const long long base = (long long)plane * a.ncell;
    const BandConst b = a.band[q.k];
    const float nux = a.nu[3 * plane], nuy = a.nu[3 * plane + 1];
    const float anx = fabsf(nux), any = fabsf(nuy);
    const int sx = nux > 0.f ? 1 : -1, sy = nuy > 0.f ? 1 : -1;
    const bool perx = a.bc[0] == kBcPeriodic, pery = a.bc[2] == kBcPeriodic;
    const float diag = 1.f - b.dtinv, wmD = a.wmom[plane] * a.invD, wd = g.w[q.d];
    const float sc = St<S>::kRef ? b.scale : 1.f;  // e = sc * (value in the kernel)
    const float bm = b.dtinv * b.ck, bq = b.srck;
    const T *e = static_cast<const T *>(a.e_in);
    const float *lam = g.lam_in;
    constexpr int kR = Geo<DIM, WPR>::KR;
    const int nrows = min(kR, q.nyt - rb);
    const int z = q.z0 + zl;
    // streaming order along y: t = 0 .. nrows-1 are this warp's rows, upwind to downwind
    const int y0w = q.y0 + (sy > 0 ? rb : rb + nrows - 1);
    auto cell_of = [&](int zz, int yy) { return ((long long)zz * ny + yy) * NX + x0; };
    // this lane's cells of (unwrapped) row yu of slice zu in the reference box: rows y0-2 ..
    // y0+TY+1 (and slices z0-2 .. z0+TZ+1 in 3-D)
    constexpr int RY = TY + 4;
    auto rho_at = [&](int zu, int yu) {
        return rbox + ((DIM == 3 ? zu - (q.z0 - 2) : 0) * RY + (yu - (q.y0 - 2))) * NX + x0;
    };

    // y window: e at t-2 .. t+2 (rows), lambda at t-1 .. t+2; faces F_{t+1} computed per step
    float e_m2[VL], e_m1[VL], e_0[VL], e_p1[VL], e_p2[VL], l_m1[VL], l_0[VL], l_p1[VL], l_p2[VL];
    float Bprev[VL], Cprev[VL], Cprev2[VL];  // B_t (face t), C_{t-1} (face t-1), C_{t-2}
    bool ok_m2, ok_m1, ok_0, ok_p1, ok_p2;
    auto load_row = [&](float (&ev)[VL], float (&lv)[VL], int t, bool &ok) {
        const int yy = adj_row(y0w + t * sy, ny, pery);
        ok = yy >= 0;
        if (ok) {
            const long long cl = cell_of(z, yy);
            adj_ld_e<S, VL>(ev, e, base, cl, rho_at(z, y0w + t * sy));
            adj_ld_l<VL>(lv, lam, base + cl);
        } else {
            #pragma unroll
            for (int j = 0; j < VL; ++j) ev[j] = lv[j] = 0.f;
        }
    };
    const int p_tcells = TY * Geo<DIM, WPR>::TZ * NX;
    float dummy[VL];
    load_row(e_m2, dummy, -2, ok_m2);
    load_row(e_m1, l_m1, -1, ok_m1);
    load_row(e_0, l_0, 0, ok_0);
    load_row(e_p1, l_p1, 1, ok_p1);
    // faces t-1 = -1 (values -2, -1, 0) and t = 0 (values -1, 0, 1)
    #pragma unroll
    for (int j = 0; j < VL; ++j) {
        float A, B, C;
        if (ok_m2 && ok_m1 && ok_0) face_terms<LIM>(e_m2[j], e_m1[j], e_0[j], any * (l_0[j] - l_m1[j]), A, B, C);
        else A = B = C = 0.f;
        Cprev[j] = C;  // C_{-1} goes to row 0
        if (ok_m1 && ok_0 && ok_p1) face_terms<LIM>(e_m1[j], e_0[j], e_p1[j], any * (l_p1[j] - l_0[j]), A, B, C);
        else A = B = C = 0.f;
        Bprev[j] = B;  // B_0 goes to row 0
        Cprev2[j] = C; // C_0 goes to row 1
    }
    #pragma unroll
    for (int t = 0; t < kR; ++t) {
        if (t >= nrows) break;
        const int y = y0w + t * sy;
        const long long cl = cell_of(z, y);
        load_row(e_p2, l_p2, t + 2, ok_p2);
        float acc[VL];
        // y: face t+1 (values t, t+1, t+2) adds A to row t
        #pragma unroll
        for (int j = 0; j < VL; ++j) {
            float A, B, C;
            if (ok_0 && ok_p1 && ok_p2) face_terms<LIM>(e_0[j], e_p1[j], e_p2[j], any * (l_p2[j] - l_p1[j]), A, B, C);
            else A = B = C = 0.f;
            acc[j] = A + Bprev[j] + Cprev[j];
            Cprev[j] = Cprev2[j];
            Bprev[j] = B;
            Cprev2[j] = C;
        }
        // x: values e and lambda at x0-2 .. x0+VL+1 from the neighbour lanes; the end lanes of
        // a warp read theirs (wrapped on a periodic axis; positions outside a wall are never
        // used: the faces reading them belong to the wall pass)
        if constexpr (WPR == 1) {
            if (sx > 0) adj_xfaces_w<LIM, VL, 1>(e_0, l_0, x0, NX, perx, anx, lane, acc);
            else adj_xfaces_w<LIM, VL, -1>(e_0, l_0, x0, NX, perx, anx, lane, acc);
        } else {
            float ex[VL + 4], lx[VL + 4];
            #pragma unroll
            for (int j = 0; j < VL; ++j) {
                ex[j + 2] = e_0[j];
                lx[j + 2] = l_0[j];
            }
            const int lft = (lane + 31) & 31, rgt = (lane + 1) & 31;
            ex[0] = __shfl_sync(0xffffffffu, e_0[VL - 2], lft);
            ex[1] = __shfl_sync(0xffffffffu, e_0[VL - 1], lft);
            ex[VL + 2] = __shfl_sync(0xffffffffu, e_0[0], rgt);
            ex[VL + 3] = __shfl_sync(0xffffffffu, e_0[1], rgt);
            lx[0] = __shfl_sync(0xffffffffu, l_0[VL - 2], lft);
            lx[1] = __shfl_sync(0xffffffffu, l_0[VL - 1], lft);
            lx[VL + 2] = __shfl_sync(0xffffffffu, l_0[0], rgt);
            lx[VL + 3] = __shfl_sync(0xffffffffu, l_0[1], rgt);
            const bool lo = lane == 0, hi = lane == 31;
            if ((lo && (half > 0 || perx)) || (hi && (half < WPR - 1 || perx))) {
                const long long rowc = ((long long)z * ny + y) * NX;
                const int xa = lo ? (x0 - 2 + NX) % NX : (x0 + VL) % NX;
                const int xb = lo ? (x0 - 1 + NX) % NX : (x0 + VL + 1) % NX;
                const float ea = adj_e1<S>(a, e, base, rowc + xa), eb = adj_e1<S>(a, e, base, rowc + xb);
                const float la = lam[base + rowc + xa], lb = lam[base + rowc + xb];
                if (lo) {
                    ex[0] = ea; ex[1] = eb; lx[0] = la; lx[1] = lb;
                } else {
                    ex[VL + 2] = ea; ex[VL + 3] = eb; lx[VL + 2] = la; lx[VL + 3] = lb;
                }
            }
            if (sx > 0) adj_xfaces<LIM, VL, 1>(ex, lx, x0, NX, perx, anx, acc);
            else adj_xfaces<LIM, VL, -1>(ex, lx, x0, NX, perx, anx, acc);
        }
        const int c = (zl * TY + (y - q.y0)) * NX + x0;
        // relaxation, T_L coupling; store; per-cell and per-segment partials
        float mu[VL], tl[VL];
        if (mtbox) {
            adj_ld_l<VL>(mu, mtbox, c);
            adj_ld_l<VL>(tl, mtbox + p_tcells, c);
        } else {
            adj_ld_l<VL>(mu, g.mu_in, cl);
            adj_ld_l<VL>(tl, a.TL, cl);
        }
        float out[VL];
        #pragma unroll
        for (int j = 0; j < VL; ++j) {
            const float lv = l_0[j];
            out[j] = fmaf(diag, lv, fmaf(wmD, mu[j], acc[j]));
            const float ev = sc * e_0[j];
            s1 = fmaf(lv, fmaf(b.ck, tl[j], -ev), s1);
            s2 = fmaf(wd * mu[j], ev, s2);
        }
        adj_emit<VL>(g, accm, accq, c, base + cl, bm, bq, out);
        // slide the window
        #pragma unroll
        for (int j = 0; j < VL; ++j) {
            e_m2[j] = e_m1[j];
            e_m1[j] = e_0[j];
            e_0[j] = e_p1[j];
            e_p1[j] = e_p2[j];
            l_m1[j] = l_0[j];
            l_0[j] = l_p1[j];
            l_p1[j] = l_p2[j];
        }
        ok_m2 = ok_m1;
        ok_m1 = ok_0;
        ok_0 = ok_p1;
        ok_p1 = ok_p2;
    }
}

// ---- 3-D plane-tiles: the box staged in shared memory ------------------------------------------
// Box of a 3-D plane-tile: rows y0-2 .. y0+TY+1 by slices z0-2 .. z0+TZ+1 of every x, index
// ((z - z0 + 2) RY + (y - y0 + 2)) NX + x (the reference box's layout).  All warps fill it with
// 16-byte loads, e (16-bit: decoded against the references) in Eb and lambda^{n+1} in Lb;
// positions beyond a wall hold 0 and are never used, and the corners (a halo row of a halo
// slice) are not read at all.
template <int S, int VL, int WPR, int DIM>
__device__ __forceinline__ void adj_stage_box(const StepArgs &a, const AdjTiledArgs &g, const PT &q, const float *rbox,
                                              float *Eb, float *Lb) {
    using T = typename St<S>::T;
    using Q = St<S>;
    constexpr int NX = 32 * VL * WPR, TY = Geo<DIM, WPR>::TY, TZ = Geo<DIM, WPR>::TZ;
    constexpr int RY = TY + 4, RZ = TZ + 4, NG = NX / 4, NT = Geo<DIM, WPR>::NCW * 32;
    static_assert(NX % 4 == 0, "rows move in groups of four cells");
    const int ny = a.n[1], nz = a.n[2];
    const bool pery = a.bc[2] == kBcPeriodic, perz = a.bc[4] == kBcPeriodic;
    const long long base = (long long)q.plane * a.ncell;
    const T *e = static_cast<const T *>(a.e_in);
    // groups of four cells, UB per thread in flight before their stores
    constexpr int TOT = RZ * RY * NG, UB = 8;
    for (int g0 = 0; g0 < TOT; g0 += UB * NT) {
        float4 ev[UB], lv[UB];
        #pragma unroll
        for (int u = 0; u < UB; ++u) {
            ev[u] = lv[u] = make_float4(0.f, 0.f, 0.f, 0.f);
            const int gi = g0 + u * NT + (int)threadIdx.x;
            const int xg = gi % NG, by = (gi / NG) % RY, bz = gi / (NG * RY);
            const int yy = adj_row(q.y0 - 2 + by, ny, pery), zz = adj_row(q.z0 - 2 + bz, nz, perz);
            const bool corner = (by < 2 || by >= TY + 2) && (bz < 2 || bz >= TZ + 2);
            if (gi < TOT && !corner && yy >= 0 && zz >= 0) {
                const int idx = (bz * RY + by) * NX + 4 * xg;
                const long long cell = ((long long)zz * ny + yy) * NX + 4 * xg;
                lv[u] = *reinterpret_cast<const float4 *>(g.lam_in + base + cell);
                if constexpr (Q::kRef) {
                    const uint2 h = *reinterpret_cast<const uint2 *>(e + base + cell);
                    float4 r;
                    if (rbox) {
                        r = *reinterpret_cast<const float4 *>(rbox + idx);
                    } else {
                        const float4 R = *reinterpret_cast<const float4 *>(a.R + cell);
                        r = make_float4(R.x * a.invTs, R.y * a.invTs, R.z * a.invTs, R.w * a.invTs);
                    }
                    ev[u] = make_float4(r.x + Q::val(h.x & 0xffffu), r.y + Q::val(h.x >> 16),
                                        r.z + Q::val(h.y & 0xffffu), r.w + Q::val(h.y >> 16));
                } else {
                    ev[u] = *reinterpret_cast<const float4 *>(e + base + cell);
                }
            }
        }
        #pragma unroll
        for (int u = 0; u < UB; ++u) {
            const int gi = g0 + u * NT + (int)threadIdx.x;
            const int xg = gi % NG, by = (gi / NG) % RY, bz = gi / (NG * RY);
            const bool corner = (by < 2 || by >= TY + 2) && (bz < 2 || bz >= TZ + 2);
            if (gi < TOT && !corner) {
                const int idx = (bz * RY + by) * NX + 4 * xg;
                *reinterpret_cast<float4 *>(Eb + idx) = ev[u];
                *reinterpret_cast<float4 *>(Lb + idx) = lv[u];
            }
        }
    }
}

template <int VL>
__device__ __forceinline__ void ld_box(float (&v)[VL], const float *p) {
    if constexpr (VL == 4) {
        const float4 f = *reinterpret_cast<const float4 *>(p);
        v[0] = f.x; v[1] = f.y; v[2] = f.z; v[3] = f.w;
    } else {
        #pragma unroll
        for (int j = 0; j < VL; ++j) v[j] = p[j];
    }
}

// One 3-D plane-tile, called by every warp of the block.  (0) All warps stage the box.  (1)
// Each warp streams its rows along y from the box: y faces in registers, x faces by shuffle,
// and the z face at its own slice (values z-sz, z, z+sz), whose B stays here while A (for
// slice z-sz) and C (for slice z+sz) go to xa / xa + tcells; a tile-edge slice also takes the
// face just outside the tile.  (2) After the second barrier each warp adds the terms its
// neighbour slices left and writes lambda^n.  The two barriers also order the reuse of the
// box and of xa by the next plane-tile.
template <int S, int LIM, int VL, int WPR, int DIM>
__device__ __forceinline__ void adj_tile3(const StepArgs &a, const AdjTiledArgs &g, const PT &q, int zl, int rb, int half,
                                          float *accm, float *accq, float &s1, float &s2, float *xa, const float *rbox,
                                          const float *mtbox, float *Eb, float *Lb) {
    static_assert(DIM == 3, "3-D plane-tiles");
    constexpr int NX = 32 * VL * WPR, TY = Geo<DIM, WPR>::TY, TZ = Geo<DIM, WPR>::TZ, NCW = Geo<DIM, WPR>::NCW;
    constexpr int RY = TY + 4, kR = Geo<DIM, WPR>::KR, TC = TY * TZ * NX;
    adj_stage_box<S, VL, WPR, DIM>(a, g, q, rbox, Eb, Lb);
    consumer_sync<NCW>();  // the box is complete
    const bool act = zl < q.nzt && rb < q.nyt;
    const int lane = threadIdx.x & 31, x0 = (half * 32 + lane) * VL;
    const int ny = a.n[1], nz = a.n[2];
    const int plane = q.plane;
    const long long base = (long long)plane * a.ncell;
    const BandConst b = a.band[q.k];
    const float nux = a.nu[3 * plane], nuy = a.nu[3 * plane + 1], nuz = a.nu[3 * plane + 2];
    const float anx = fabsf(nux), any = fabsf(nuy), anz = fabsf(nuz);
    const int sx = nux > 0.f ? 1 : -1, sy = nuy > 0.f ? 1 : -1, sz = nuz > 0.f ? 1 : -1;
    const bool perx = a.bc[0] == kBcPeriodic, pery = a.bc[2] == kBcPeriodic, perz = a.bc[4] == kBcPeriodic;
    const float diag = 1.f - b.dtinv, wmD = a.wmom[plane] * a.invD, wd = g.w[q.d];
    const float sc = St<S>::kRef ? b.scale : 1.f;  // e = sc * (value in the kernel)
    const float bm = b.dtinv * b.ck, bq = b.srck;
    const int nrows = act ? min(kR, q.nyt - rb) : 0;
    const int z = q.z0 + zl;
    const int y0w = q.y0 + (sy > 0 ? rb : rb + nrows - 1);
    // this lane's cells of (unwrapped) row yu at slice offset dzs from z in the box
    auto box_at = [&](const float *B, int dzs, int yu) { return B + ((zl + 2 + dzs) * RY + (yu - q.y0 + 2)) * NX + x0; };
    const bool in_up = zl - sz >= 0 && zl - sz < q.nzt, in_dn = zl + sz >= 0 && zl + sz < q.nzt;
    const bool zok1 = adj_row(z - sz, nz, perz) >= 0, zok3 = adj_row(z + sz, nz, perz) >= 0;
    const bool zok0 = adj_row(z - 2 * sz, nz, perz) >= 0, zok4 = adj_row(z + 2 * sz, nz, perz) >= 0;
    float outp[kR][VL];
    if (act) {
        // y window: e at t-2 .. t+2 (rows), lambda at t-1 .. t+2; faces F_{t+1} computed per step
        float e_m2[VL], e_m1[VL], e_0[VL], e_p1[VL], e_p2[VL], l_m1[VL], l_0[VL], l_p1[VL], l_p2[VL];
        float Bprev[VL], Cprev[VL], Cprev2[VL];
        bool ok_m2, ok_m1, ok_0, ok_p1, ok_p2;
        auto load_row = [&](float (&ev)[VL], float (&lv)[VL], int t, bool &ok, bool withl) {
            const int yu = y0w + t * sy;
            ok = adj_row(yu, ny, pery) >= 0;
            ld_box<VL>(ev, box_at(Eb, 0, yu));
            if (withl) ld_box<VL>(lv, box_at(Lb, 0, yu));
        };
        float dummy[VL];
        load_row(e_m2, dummy, -2, ok_m2, false);
        load_row(e_m1, l_m1, -1, ok_m1, true);
        load_row(e_0, l_0, 0, ok_0, true);
        load_row(e_p1, l_p1, 1, ok_p1, true);
        #pragma unroll
        for (int j = 0; j < VL; ++j) {
            float A, B, C;
            if (ok_m2 && ok_m1 && ok_0) face_terms<LIM>(e_m2[j], e_m1[j], e_0[j], any * (l_0[j] - l_m1[j]), A, B, C);
            else A = B = C = 0.f;
            Cprev[j] = C;
            if (ok_m1 && ok_0 && ok_p1) face_terms<LIM>(e_m1[j], e_0[j], e_p1[j], any * (l_p1[j] - l_0[j]), A, B, C);
            else A = B = C = 0.f;
            Bprev[j] = B;
            Cprev2[j] = C;
        }
        #pragma unroll
        for (int t = 0; t < kR; ++t) {
            if (t >= nrows) break;
            const int y = y0w + t * sy;
            const int c = (zl * TY + (y - q.y0)) * NX + x0;
            load_row(e_p2, l_p2, t + 2, ok_p2, true);
            float acc[VL];
            #pragma unroll
            for (int j = 0; j < VL; ++j) {
                float A, B, C;
                if (ok_0 && ok_p1 && ok_p2) face_terms<LIM>(e_0[j], e_p1[j], e_p2[j], any * (l_p2[j] - l_p1[j]), A, B, C);
                else A = B = C = 0.f;
                acc[j] = A + Bprev[j] + Cprev[j];
                Cprev[j] = Cprev2[j];
                Bprev[j] = B;
                Cprev2[j] = C;
            }
            if (sx > 0) adj_xfaces_w<LIM, VL, 1>(e_0, l_0, x0, NX, perx, anx, lane, acc);
            else adj_xfaces_w<LIM, VL, -1>(e_0, l_0, x0, NX, perx, anx, lane, acc);
            // z: the face at this slice, and the tile-edge faces
            {
                float e1[VL], e3[VL], l3[VL];
                ld_box<VL>(e1, box_at(Eb, -sz, y));
                ld_box<VL>(e3, box_at(Eb, sz, y));
                ld_box<VL>(l3, box_at(Lb, sz, y));
                float xA[VL], xC[VL];
                #pragma unroll
                for (int j = 0; j < VL; ++j) {
                    float A = 0.f, B = 0.f, C = 0.f;
                    if (zok1 && zok3) face_terms<LIM>(e1[j], e_0[j], e3[j], anz * (l3[j] - l_0[j]), A, B, C);
                    acc[j] += B;
                    xA[j] = A;
                    xC[j] = C;
                }
                #pragma unroll
                for (int j = 0; j < VL; ++j) {
                    xa[c + j] = xA[j];
                    xa[TC + c + j] = xC[j];
                }
                if (!in_up && zok0 && zok1) {
                    float e0v[VL], l1[VL];
                    ld_box<VL>(e0v, box_at(Eb, -2 * sz, y));
                    ld_box<VL>(l1, box_at(Lb, -sz, y));
                    #pragma unroll
                    for (int j = 0; j < VL; ++j) {
                        float A, B, C;
                        face_terms<LIM>(e0v[j], e1[j], e_0[j], anz * (l_0[j] - l1[j]), A, B, C);
                        acc[j] += C;
                    }
                }
                if (!in_dn && zok3 && zok4) {
                    float e4[VL], l4[VL];
                    ld_box<VL>(e4, box_at(Eb, 2 * sz, y));
                    ld_box<VL>(l4, box_at(Lb, 2 * sz, y));
                    #pragma unroll
                    for (int j = 0; j < VL; ++j) {
                        float A, B, C;
                        face_terms<LIM>(e_0[j], e3[j], e4[j], anz * (l4[j] - l3[j]), A, B, C);
                        acc[j] += A;
                    }
                }
            }
            // relaxation, T_L coupling and the segment scalars
            float mu[VL], tl[VL];
            const long long cl = ((long long)z * ny + y) * NX + x0;
            if (mtbox) {
                adj_ld_l<VL>(mu, mtbox, c);
                adj_ld_l<VL>(tl, mtbox + TC, c);
            } else {
                adj_ld_l<VL>(mu, g.mu_in, cl);
                adj_ld_l<VL>(tl, a.TL, cl);
            }
            #pragma unroll
            for (int j = 0; j < VL; ++j) {
                const float lv = l_0[j];
                outp[t][j] = fmaf(diag, lv, fmaf(wmD, mu[j], acc[j]));
                const float ev = sc * e_0[j];
                s1 = fmaf(lv, fmaf(b.ck, tl[j], -ev), s1);
                s2 = fmaf(wd * mu[j], ev, s2);
            }
            #pragma unroll
            for (int j = 0; j < VL; ++j) {
                e_m2[j] = e_m1[j];
                e_m1[j] = e_0[j];
                e_0[j] = e_p1[j];
                e_p1[j] = e_p2[j];
                l_m1[j] = l_0[j];
                l_0[j] = l_p1[j];
                l_p1[j] = l_p2[j];
            }
            ok_m2 = ok_m1;
            ok_m1 = ok_0;
            ok_0 = ok_p1;
            ok_p1 = ok_p2;
        }
    }
    consumer_sync<NCW>();  // every slice's A and C of this plane-tile are written
    if (act) {
        const int dzc = sz * TY * NX;
        #pragma unroll
        for (int t = 0; t < kR; ++t) {
            if (t >= nrows) break;
            const int y = y0w + t * sy;
            const int c = (zl * TY + (y - q.y0)) * NX + x0;
            float out[VL];
            #pragma unroll
            for (int j = 0; j < VL; ++j) {
                float v = outp[t][j];
                if (in_up) v += xa[TC + c - dzc + j];  // C of the face at slice z-sz
                if (in_dn) v += xa[c + dzc + j];       // A of the face at slice z+sz
                out[j] = v;
            }
            adj_emit<VL>(g, accm, accq, c, base + ((long long)z * ny + y) * NX + x0, bm, bq, out);
        }
    }
}

// A unit's shared copies: the code references R / T_scale of rows y0-2 .. y0+TY+1 (and slices
// z0-2 .. z0+TZ+1) of every x, wrapped on a periodic axis (positions beyond a wall are never
// read: faces reading them belong to the wall pass), and mu^{n+1}, T_L^n of the tile's cells.
template <int S, int VL, int WPR, int DIM>
__device__ void adj_fill_boxes(const StepArgs &a, const AdjTiledArgs &g, const PT &q, float *rbox, float *mtbox) {
    constexpr int NX = 32 * VL * WPR, TY = Geo<DIM, WPR>::TY, TZ = Geo<DIM, WPR>::TZ;
    constexpr int RY = TY + 4, RZ = DIM == 3 ? TZ + 4 : 1, NT = Geo<DIM, WPR>::NCW * 32;
    const int ny = a.n[1], nz = a.n[2];
    const bool pery = a.bc[2] == kBcPeriodic, perz = DIM == 3 && a.bc[4] == kBcPeriodic;
    if constexpr (St<S>::kRef) {
        for (int idx = threadIdx.x; idx < RZ * RY * NX; idx += NT) {
            const int x = idx % NX, ry = (idx / NX) % RY, rz = idx / (NX * RY);
            const int y = adj_row(q.y0 - 2 + ry, ny, pery);
            const int z = DIM == 3 ? adj_row(q.z0 - 2 + rz, nz, perz) : 0;
            rbox[idx] = (y >= 0 && z >= 0) ? a.R[((long long)z * ny + y) * NX + x] * a.invTs : 0.f;
        }
    }
    if (mtbox) {
        constexpr int TC = TY * TZ * NX;
        for (int idx = threadIdx.x; idx < TC; idx += NT) {
            const int x = idx % NX, yl = (idx / NX) % TY, zl = idx / (NX * TY);
            float mu = 0.f, tl = 0.f;
            if (yl < q.nyt && zl < q.nzt) {
                const long long cell = ((long long)(q.z0 + zl) * ny + q.y0 + yl) * NX + x;
                mu = g.mu_in[cell];
                tl = a.TL[cell];
            }
            mtbox[idx] = mu;
            mtbox[TC + idx] = tl;
        }
    }
}

template <int S, int LIM, int VL, int WPR, int DIM>
__global__ void __launch_bounds__(Geo<DIM, WPR>::NCW * 32, 1) k_adj_tiled(const StepArgs a, const TiledArgs p,
                                                                          const AdjTiledArgs g) {
    constexpr int NX = 32 * VL * WPR, TY = Geo<DIM, WPR>::TY, NCW = Geo<DIM, WPR>::NCW;
    extern __shared__ __align__(128) char smem[];
    float *accm = reinterpret_cast<float *>(smem);
    float *accq = accm + p.tcells;
    float *red = accq + p.tcells;  // [2][NCW]
    // 3-D: the z-face terms passed between slices [A, C][tcells], then the plane-tile's box of
    // e and of lambda^{n+1}
    constexpr int RB = (TY + 4) * (DIM == 3 ? Geo<DIM, WPR>::TZ + 4 : 1) * NX;
    float *xbuf = red + 2 * NCW;
    float *Eb = xbuf + (DIM == 3 ? 2 * p.tcells : 0), *Lb = Eb + RB;
    // 16-bit storage: the unit's reference box (where it fits); then, if they fit, mu and T_L of
    // the tile
    float *rbox = g.cache_r ? (DIM == 3 ? Lb + RB : xbuf) : nullptr;
    float *mtbox = g.cache_mt ? (rbox ? rbox + RB : (DIM == 3 ? Lb + RB : xbuf)) : nullptr;
    for (int j = threadIdx.x; j < 2 * p.tcells; j += blockDim.x) accm[j] = 0.f;
    __syncthreads();
    int zl, rb, half;
    warp_place<VL, WPR, DIM>(zl, rb, half);
    const int lane = threadIdx.x & 31, x0 = (half * 32 + lane) * VL;
    int seg = -1, cur_unit = -1, cur_band = -1;
    PT cur{};
    float s1 = 0.f, s2 = 0.f;
    auto flush = [&]() {
        float *Pm = g.Pm + (size_t)seg * p.tcells, *Pq = g.Pq + (size_t)seg * p.tcells;
        #pragma unroll
        for (int r = 0; r < Geo<DIM, WPR>::KR; ++r) {
            const int yl = rb + r;
            const int c = (zl * TY + yl) * NX + x0;
            if constexpr (VL == 4) {
                if (yl < cur.nyt && zl < cur.nzt) {
                    *reinterpret_cast<float4 *>(Pm + c) = *reinterpret_cast<const float4 *>(accm + c);
                    *reinterpret_cast<float4 *>(Pq + c) = *reinterpret_cast<const float4 *>(accq + c);
                }
                *reinterpret_cast<float4 *>(accm + c) = make_float4(0.f, 0.f, 0.f, 0.f);
                *reinterpret_cast<float4 *>(accq + c) = make_float4(0.f, 0.f, 0.f, 0.f);
            } else {
                if (yl < cur.nyt && zl < cur.nzt) {
                    #pragma unroll
                    for (int v = 0; v < VL; ++v) {
                        Pm[c + v] = accm[c + v];
                        Pq[c + v] = accq[c + v];
                    }
                }
                #pragma unroll
                for (int v = 0; v < VL; ++v) accm[c + v] = accq[c + v] = 0.f;
            }
        }
        // segment scalars: warp sums, then warp 0 adds the warps in order
        #pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            s1 += __shfl_xor_sync(0xffffffffu, s1, o);
            s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        }
        if (lane == 0) {
            red[threadIdx.x >> 5] = s1;
            red[NCW + (threadIdx.x >> 5)] = s2;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            float t1 = 0.f, t2 = 0.f;
            for (int w = 0; w < NCW; ++w) {
                t1 += red[w];
                t2 += red[NCW + w];
            }
            g.Ps[2 * seg] = t1;
            g.Ps[2 * seg + 1] = t2;
        }
        __syncthreads();
        s1 = s2 = 0.f;
    };
    Cursor<DIM, WPR> c;
    bool more = c.start(a, p);
    for (; more; more = c.next(a, p)) {
        const PT q = c.q;
        if (c.u != cur_unit || q.k != cur_band) {
            if (seg >= 0) flush();  // ends with a block barrier: no warp reads the old unit's boxes
            if (c.u != cur_unit && (rbox || mtbox)) {
                adj_fill_boxes<S, VL, WPR, DIM>(a, g, q, rbox, mtbox);
                __syncthreads();
            }
            seg = p.unit_seg0[c.u] + q.k - c.p0 / a.nd;
            cur_unit = c.u;
            cur_band = q.k;
            cur = q;
        }
        if constexpr (DIM == 3)
            adj_tile3<S, LIM, VL, WPR, DIM>(a, g, q, zl, rb, half, accm, accq, s1, s2, xbuf, rbox, mtbox, Eb, Lb);
        else if (zl < q.nzt && rb < q.nyt)
            adj_rows<S, LIM, VL, WPR, DIM>(a, g, q, zl, rb, half, accm, accq, s1, s2, rbox, mtbox);
    }
    if (seg >= 0) flush();
}

typedef void (*AdjKernel)(const StepArgs, const TiledArgs, const AdjTiledArgs);

template <int S, int LIM, int DIM>
AdjKernel adj_pick_nx(int nx) {
    if (nx == 96) return k_adj_tiled<S, LIM, 3, 1, DIM>;
    if (nx == 128) return k_adj_tiled<S, LIM, 4, 1, DIM>;
    if constexpr (DIM == 2) {
        if (nx == 256) return k_adj_tiled<S, LIM, 4, 2, DIM>;
    }
    return nullptr;
}

template <int S>
AdjKernel adj_pick_instance(int lim, int nx, int dim) {
    if (dim == 2) {
        if (lim == kLimFirst) return adj_pick_nx<S, kLimFirst, 2>(nx);
        if (lim == kLimMinmod) return adj_pick_nx<S, kLimMinmod, 2>(nx);
        return adj_pick_nx<S, kLimVanAlbada, 2>(nx);
    }
    if (lim == kLimFirst) return adj_pick_nx<S, kLimFirst, 3>(nx);
    if (lim == kLimMinmod) return adj_pick_nx<S, kLimMinmod, 3>(nx);
    return adj_pick_nx<S, kLimVanAlbada, 3>(nx);
}

AdjKernel adj_pick_f32(int lim, int nx, int dim);
AdjKernel adj_pick_f16(int lim, int nx, int dim);
AdjKernel adj_pick_bf16(int lim, int nx, int dim);

}  // namespace tiled
}  // namespace bte
