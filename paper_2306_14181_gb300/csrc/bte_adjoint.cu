// Discrete adjoint of the explicit DOM transient step (arXiv 2306.14181, Sec. 4).  The paper
// has no adjoint; this is the exact transpose of the forward step of bte_kernels.cu /
// bte_tiled.cu, derived by hand.  One step is e^{n+1} = F(e^n, T_L(e^n)) with T_L of
// Eq. (BTE_get_e0) linear in e, so for J = sum_i p_i T_L,i(e^N)
//   lambda^N           = dT_L/de^T p,
//   lambda^n           = dF/de^T lambda^{n+1} + dT_L/de^T mu^{n+1},
//   mu^{n+1}_i         = sum_{k,d} lambda^{n+1}_{k,d,i} dt C_k/(W tau_k),
//   dJ/dQ_i           += dt a_n sum_{k,d} lambda^{n+1}_{k,d,i} C_k/(sum C W),
//   dJ/dlog tau_k     += sum_{d,i} lambda^{n+1} (-dt/tau_k)(C_k T_L/W - e)
//                        + sum_i mu^{n+1}_i (C_k T_L,i - sum_d w_d e_{k,d,i})/(tau_k D).
// dF/de^T is a gather over the downwind-transposed stencil: a face with upwind cell m,
// value F_m = u_m + L(u_m - u_l, u_r - u_m)/2, enters cell m with -|nu| and cell m+sg with
// +|nu|, so its adjoint weight is phi_m = |nu| (lambda_{m+sg} - lambda_m), and cell j
// collects phi_{j+sg} dF/du_l + phi_j dF/du_m + phi_{j-sg} dF/du_r, the limiter Jacobian
// evaluated at e^n.  Ghost values transpose as: periodic -> wrap; thermalizing incoming -> 0;
// outgoing (thermalizing or diffuse wall) -> the wall cell itself; specular -> the mirrored
// direction's cells (gathered from that plane's faces next to the wall); diffuse incoming ->
// spread back over the wall cell's outgoing directions with weights w (s.n) / sum_in w|s.n|.
// One thread per (cell, band) loops over the band's directions, as the generic forward does.
#include <algorithm>
#include <cstdlib>

#include "bte_device.cuh"
#include "bte_adjoint.h"

namespace bte {

// Partial derivatives of the limiter L(a, b) (0 where ab <= 0).
template <int LIM> __device__ __forceinline__ void lim_grad(float a, float b, float &La, float &Lb);
template <> __device__ __forceinline__ void lim_grad<kLimFirst>(float, float, float &La, float &Lb) {
    La = Lb = 0.f;
}
template <> __device__ __forceinline__ void lim_grad<kLimMinmod>(float a, float b, float &La, float &Lb) {
    const bool on = a * b > 0.f, pa = fabsf(a) < fabsf(b);
    La = on && pa ? 1.f : 0.f;
    Lb = on && !pa ? 1.f : 0.f;
}
template <> __device__ __forceinline__ void lim_grad<kLimVanAlbada>(float a, float b, float &La, float &Lb) {
    // L = ab(a+b)/(a^2+b^2):  dL/da = b^2 (2ab + b^2 - a^2)/(a^2+b^2)^2, symmetric in b.  L is
    // homogeneous of degree 1, so its partials are of degree 0: they are evaluated on
    // (a, b) / max(|a|, |b|), which keeps a^2 + b^2 in [1, 2].  (On the raw slopes, tiny ones --
    // a state barely off its reference -- overflow 1/(a^2+b^2)^2 to infinity and the product
    // to NaN.)
    La = Lb = 0.f;
    if (a * b > 0.f) {
        const float r = 1.f / fmaxf(fabsf(a), fabsf(b));
        const float an = a * r, bn = b * r;
        const float q = fmaf(an, an, bn * bn);
        const float rq = 1.f / q;
        La = (bn * bn * rq) * ((2.f * an * bn + bn * bn - an * an) * rq);
        Lb = (an * an * rq) * ((2.f * an * bn + an * an - bn * bn) * rq);
    }
}

// dF/du_l, dF/du_m, dF/du_r of the face with upwind position m (orientation sg) of plane
// (k, d) on the line of cell i along axis ax.
template <class Cd, int LIM>
__device__ __forceinline__ void face_grad(const StepArgs &a, const typename Cd::T *e, const BandConst &b, int k,
                                          int d, long long base, long long i, const int c[3], int ax, int m, int sg,
                                          float nu, float g[3]) {
    const float ul = ext_value<Cd>(a, e, b, k, d, base, i, c, ax, m - sg, nu);
    const float um = ext_value<Cd>(a, e, b, k, d, base, i, c, ax, m, nu);
    const float ur = ext_value<Cd>(a, e, b, k, d, base, i, c, ax, m + sg, nu);
    float La, Lb;
    lim_grad<LIM>(um - ul, ur - um, La, Lb);
    g[0] = -0.5f * La;
    g[1] = 1.f + 0.5f * (La - Lb);
    g[2] = 0.5f * Lb;
}

// lambda^{n+1} of plane base at position pos along ax through cell i: 0 outside the domain
// (ghost cells are not updated), wrapped on a periodic axis.
__device__ __forceinline__ float lam_at(const StepArgs &a, const float *lam, long long base, long long i,
                                        const int c[3], int ax, int pos) {
    const int n = a.n[ax];
    if (pos < 0 || pos >= n) {
        if (a.bc[2 * ax + (pos < 0 ? 0 : 1)] != kBcPeriodic) return 0.f;
        pos = pos < 0 ? pos + n : pos - n;
    }
    return lam[base + i + (long long)(pos - c[ax]) * a.stride[ax]];
}

template <int S, int LIM>
__global__ void __launch_bounds__(256) k_adj_step(const StepArgs a, const AdjArgs g) {
    using Cd = Codec<S>;
    using T = typename Cd::T;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.ncell) return;
    const int k = blockIdx.y;
    int c[3];
    cell_coords(a, i, c);
    const BandConst b = a.band[k];
    const T *e = static_cast<const T *>(a.e_in);
    const float *lam = g.lam_in;
    const float mu = g.mu_in[i];
    const float TLi = a.TL[i];
    const float rho_i = rho_at<Cd>(a.R, a.invTs, i);

    // Diffuse walls at this cell: adjoint of the incoming ghost value (both layers hold it),
    // summed over the incoming directions of the band.
    int wl[6];
    const int nw = diffuse_walls_of(a, c, wl);
    float gam[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int j = 0; j < nw; ++j) {
        const int w = wl[j], ax = w >> 1, side = w & 1;
        for (int d = 0; d < a.nd; ++d) {
            const int plane = k * a.nd + d;
            const float nu = a.nu[3 * plane + ax];
            if (!(side == 0 ? nu > 0.f : nu < 0.f)) continue;
            const int sg = nu > 0.f ? 1 : -1;
            const long long base = (long long)plane * a.ncell;
            const int f = c[ax];  // first cell of this orientation
            float g1[3], g0[3];
            face_grad<Cd, LIM>(a, e, b, k, d, base, i, c, ax, f - sg, sg, nu, g1);
            face_grad<Cd, LIM>(a, e, b, k, d, base, i, c, ax, f, sg, nu, g0);
            const float anu = fabsf(nu);
            const float l0 = lam_at(a, lam, base, i, c, ax, f), l1 = lam_at(a, lam, base, i, c, ax, f + sg);
            gam[j] += anu * l0 * (g1[0] + g1[1]) + anu * (l1 - l0) * g0[0];
        }
    }

    float sq = 0.f, st = 0.f, sm = 0.f, se = 0.f;
    for (int d = 0; d < a.nd; ++d) {
        const int plane = k * a.nd + d;
        const long long base = (long long)plane * a.ncell;
        const float l = lam[base + i];
        const float e0 = Cd::ld(e, base + i, b, rho_i);
        sq += l;
        st = fmaf(l, fmaf(b.ck, TLi, -e0), st);
        se = fmaf(g.w[d], e0, se);
        // relaxation -dt/tau e^n and the T_L coupling
        float acc = fmaf(1.f - b.dtinv, l, a.wmom[plane] * a.invD * mu);
        for (int ax = 0; ax < a.dim; ++ax) {
            const float nu = a.nu[3 * plane + ax];
            if (nu == 0.f) continue;
            const int sg = nu > 0.f ? 1 : -1, n = a.n[ax], j = c[ax];
            const float anu = fabsf(nu);
            const bool per = a.bc[2 * ax] == kBcPeriodic;
            float fg[3];
            // the stencil u_{-2..2} = e(j + m sg) (ghosts by the wall rules) and
            // lambda_{-1..2}; the three faces that read this cell are F_{j-sg} = (u-2, u-1, u0),
            // F_j = (u-1, u0, u1) and F_{j+sg} = (u0, u1, u2)
            const float um2 = ext_value<Cd>(a, e, b, k, d, base, i, c, ax, j - 2 * sg, nu);
            const float um1 = ext_value<Cd>(a, e, b, k, d, base, i, c, ax, j - sg, nu);
            const float u0 = e0;
            const float up1 = ext_value<Cd>(a, e, b, k, d, base, i, c, ax, j + sg, nu);
            const float lm1 = lam_at(a, lam, base, i, c, ax, j - sg), lp1 = lam_at(a, lam, base, i, c, ax, j + sg);
            // face j+sg reads this cell as its upwind-left value (a face of the forward step
            // only if its upwind cell is in the domain)
            if (per || (j + sg >= 0 && j + sg < n)) {
                const float up2 = ext_value<Cd>(a, e, b, k, d, base, i, c, ax, j + 2 * sg, nu);
                float La, Lb;
                lim_grad<LIM>(up1 - u0, up2 - up1, La, Lb);
                acc += anu * (lam_at(a, lam, base, i, c, ax, j + 2 * sg) - lp1) * (-0.5f * La);
            }
            // face j: this cell is its upwind value (and its downwind ghost when that ghost is
            // the wall cell itself: a direction leaving through a thermalizing or diffuse wall)
            {
                float La, Lb;
                lim_grad<LIM>(u0 - um1, up1 - u0, La, Lb);
                fg[1] = 1.f + 0.5f * (La - Lb);
                fg[2] = 0.5f * Lb;
            }
            const float phj = anu * (lp1 - l);
            acc += phj * fg[1];
            if (!per && (j + sg < 0 || j + sg >= n)) {
                const int bcd = a.bc[2 * ax + (sg > 0 ? 1 : 0)];
                if (bcd == kBcIsothermal || bcd == kBcDiffuse) acc += phj * fg[2];
            }
            // face j-sg reads this cell as its downwind value
            {
                float La, Lb;
                lim_grad<LIM>(um1 - um2, u0 - um1, La, Lb);
                acc += anu * (l - lm1) * (0.5f * Lb);
            }
            // specular walls: faces of the mirrored direction that read this element as a ghost
            for (int side = 0; side < 2; ++side) {
                if (a.bc[2 * ax + side] != kBcSpecular) continue;
                const int w0 = side ? n - 1 : 0, in = side ? -1 : 1;
                const int layer = j == w0 ? 1 : (j == w0 + in ? 2 : 0);
                if (layer == 0) continue;
                const int dm = a.mirror[ax * a.nd + d];
                const long long mbase = ((long long)k * a.nd + dm) * a.ncell;
                const float num = a.nu[3 * (k * a.nd + dm) + ax];
                if (num == 0.f) continue;
                const int sgm = num > 0.f ? 1 : -1;
                if (sgm == in) {
                    // the mirrored direction enters through this wall: its ghosts w0 - sgm
                    // (layer 1) and w0 - 2 sgm (layer 2) are this plane's cells w0, w0 + in
                    float ga[3], gb[3];
                    face_grad<Cd, LIM>(a, e, b, k, dm, mbase, i, c, ax, w0 - sgm, sgm, num, ga);
                    const float la = anu * lam_at(a, lam, mbase, i, c, ax, w0);
                    if (layer == 1) {
                        face_grad<Cd, LIM>(a, e, b, k, dm, mbase, i, c, ax, w0, sgm, num, gb);
                        const float lb = anu * (lam_at(a, lam, mbase, i, c, ax, w0 + sgm) -
                                                lam_at(a, lam, mbase, i, c, ax, w0));
                        acc += la * ga[1] + lb * gb[0];
                    } else {
                        acc += la * ga[0];
                    }
                } else if (layer == 1) {
                    // the mirrored direction leaves through this wall: its downwind ghost is
                    // this plane's wall cell
                    face_grad<Cd, LIM>(a, e, b, k, dm, mbase, i, c, ax, w0, sgm, num, fg);
                    acc -= anu * lam_at(a, lam, mbase, i, c, ax, w0) * fg[2];
                }
            }
        }
        // diffuse walls: this direction leaving through one spreads the ghost adjoint back
        for (int jw = 0; jw < nw; ++jw) acc = fmaf(a.wdiff[wl[jw] * a.nd + d] * a.inv_den[wl[jw]], gam[jw], acc);
        g.lam_out[base + i] = acc;
        sm += acc;
    }
    g.pmu[(long long)k * a.ncell + i] = sm * (b.dtinv * b.ck);
    g.pq[(long long)k * a.ncell + i] = sq;
    g.pt[(long long)k * a.ncell + i] = fmaf(-b.dtinv, st, mu * (b.ck * g.W * TLi - se) * b.wtau * a.invD);
}

// lambda^N = dT_L/de^T p with the final T_L's own log-tau derivative: writes lam_out, pmu, pt
// and pq = sum_d lambda^N.
template <int S>
__global__ void __launch_bounds__(256) k_adj_init(const StepArgs a, const AdjArgs g, const float *probe) {
    using Cd = Codec<S>;
    using T = typename Cd::T;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.ncell) return;
    const int k = blockIdx.y;
    const BandConst b = a.band[k];
    const T *e = static_cast<const T *>(a.e_in);
    const float rho_i = rho_at<Cd>(a.R, a.invTs, i);
    const float p = probe[i];
    float sm = 0.f, se = 0.f;
    for (int d = 0; d < a.nd; ++d) {
        const int plane = k * a.nd + d;
        const long long base = (long long)plane * a.ncell;
        const float l = p * a.wmom[plane] * a.invD;
        g.lam_out[base + i] = l;
        sm += l;
        se = fmaf(g.w[d], Cd::ld(e, base + i, b, rho_i), se);
    }
    g.pmu[(long long)k * a.ncell + i] = sm * (b.dtinv * b.ck);
    g.pq[(long long)k * a.ncell + i] = sm;
    g.pt[(long long)k * a.ncell + i] = p * (b.ck * g.W * a.TL[i] - se) * b.wtau * a.invD;
}

// mu^n_i = sum_k pmu[k][i] and dJ/dQ_i += a_n sum_k dt C_k/(sum C W) pq[k][i], in band order.
__global__ void __launch_bounds__(256) k_adj_cells(const StepArgs a, const AdjArgs g, float amp, float *mu_out,
                                                   double *gQ) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.ncell) return;
    float m = 0.f;
    double q = 0.0;
    for (int k = 0; k < a.nb; ++k) {
        m += g.pmu[(long long)k * a.ncell + i];
        q += (double)a.band[k].srck * (double)g.pq[(long long)k * a.ncell + i];
    }
    mu_out[i] = m;
    gQ[i] += (double)amp * q;
}

// dJ/dlog tau_k += sum_i pt[k][i]: fixed-range block sums in FP64, then the blocks in order.
constexpr int kTauBlock = 256, kTauPerBlock = 8192;
__global__ void __launch_bounds__(kTauBlock) k_adj_tau_blocks(const AdjArgs g, long long ncell, double *part,
                                                              int nblk) {
    __shared__ double sh[kTauBlock];
    const int k = blockIdx.y;
    const long long lo = (long long)blockIdx.x * kTauPerBlock;
    const long long hi = lo + kTauPerBlock < ncell ? lo + kTauPerBlock : ncell;
    double s = 0.0;
    for (long long i = lo + threadIdx.x; i < hi; i += kTauBlock) s += (double)g.pt[(long long)k * ncell + i];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int h = kTauBlock / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) sh[threadIdx.x] += sh[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[(long long)k * nblk + blockIdx.x] = sh[0];
}

__global__ void k_adj_tau_sum(const double *part, int nblk, int nb, double *gtau) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nb) return;
    double s = 0.0;
    for (int j = 0; j < nblk; ++j) s += part[(long long)k * nblk + j];
    gtau[k] += s;
}

int adj_tau_blocks(long long ncell) { return (int)((ncell + kTauPerBlock - 1) / kTauPerBlock); }


// ------------------------------------------------------------------------------------------
// Wall pass of the tiled adjoint: along axis ax, one thread per (band, line of cells) adds the
// faces next to a non-periodic wall that read a ghost value (the first cell's in-face F_{f-sg}
// and out-face F_f for directions entering through the wall, the last cell's out-face F_l for
// directions leaving through it) and the ghost transposes: thermalizing incoming -> nothing,
// outgoing -> the wall cell itself, specular -> the mirrored direction's wall and next cells,
// diffuse incoming -> spread over the wall cell's outgoing directions.  Axis passes run one
// after another (corner cells are touched by two).  The per-cell sums of the additions for
// cells 0, 1, n-2, n-1 of the line go to corr[k][slot][line] for the finalize.
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ int wall_slot(int pos, int n) { return pos < 2 ? pos : 2 + pos - (n - 2); }

// Phase 1: one thread per (line, direction, band), threads along the lines (coalesced for y and
// z walls).  scratch[((k nd + d) 8 + 4 side + j) nlines + line], j = 0, 1: additions to the
// wall cell and the next cell of the same plane; j = 2, 3: adjoints of ghost layers 1 and 2.
constexpr int kWallThreads = 128;
constexpr long long kWallLineThreads = 65536;  // (line, band) pairs from which phase 2 takes a thread each

template <int S, int LIM>
__global__ void __launch_bounds__(kWallThreads) k_adj_walls_a(const StepArgs a, const AdjArgs g, int ax,
                                                              float *scratch, long long nlines) {
    using Cd = Codec<S>;
    using T = typename Cd::T;
    const long long line = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (line >= nlines) return;
    const int d = blockIdx.y, k = blockIdx.z;
    const int n = a.n[ax];
    int c[3];
    {
        const int o1 = ax == 0 ? 1 : 0, o2 = ax == 2 ? 1 : 2;
        c[ax] = 0;
        c[o1] = (int)(line % a.n[o1]);
        c[o2] = (int)(line / a.n[o1]);
    }
    const long long i0 = ((long long)c[2] * a.n[1] + c[1]) * a.n[0] + c[0];
    const long long st = a.stride[ax];
    const BandConst b = a.band[k];
    const T *e = static_cast<const T *>(a.e_in);
    const float *lam = g.lam_in;
    const int plane = k * a.nd + d;
    const float nu = a.nu[3 * plane + ax];
    const int sg = nu > 0.f ? 1 : -1;
    const float anu = fabsf(nu);
    const long long base = (long long)plane * a.ncell;
    float *out = scratch + (long long)plane * 8 * nlines + line;
    for (int side = 0; side < 2; ++side) {
        float v[4] = {0.f, 0.f, 0.f, 0.f};
        if (a.bc[2 * ax + side] != kBcPeriodic && nu != 0.f) {
            const int w0 = side ? n - 1 : 0, in = side ? -1 : 1;
            int cw[3] = {c[0], c[1], c[2]};
            cw[ax] = w0;
            const long long iw = i0 + (long long)w0 * st;
            if (sg == in) {
                // entering through this wall: first cell w0, faces F_{w0-sg} and F_{w0}
                float ga[3], gb[3];
                face_grad<Cd, LIM>(a, e, b, k, d, base, iw, cw, ax, w0 - sg, sg, nu, ga);
                face_grad<Cd, LIM>(a, e, b, k, d, base, iw, cw, ax, w0, sg, nu, gb);
                const float l0 = lam_at(a, lam, base, iw, cw, ax, w0), l1 = lam_at(a, lam, base, iw, cw, ax, w0 + sg);
                const float pa = anu * l0, pb = anu * (l1 - l0);
                v[0] = pa * ga[2] + pb * gb[1];
                v[1] = pb * gb[2];
                v[2] = pa * ga[1] + pb * gb[0];
                v[3] = pa * ga[0];
            } else {
                // leaving through this wall: last cell w0, face F_{w0} reads ghost layer 1
                float gc[3];
                face_grad<Cd, LIM>(a, e, b, k, d, base, iw, cw, ax, w0, sg, nu, gc);
                const float ph = -anu * lam_at(a, lam, base, iw, cw, ax, w0);
                v[1] = ph * gc[0];
                v[0] = ph * gc[1];
                v[2] = ph * gc[2];
            }
        }
        #pragma unroll
        for (int j = 0; j < 4; ++j) out[(long long)(4 * side + j) * nlines] = v[j];
    }
}

// Phase 2 for many lines: one thread per (line, band), threads along the lines, each looping
// over the directions in order: the ghost transposes (specular: the mirrored direction's ghost adjoints;
// thermalizing or diffuse outgoing: the direction's own; diffuse incoming: summed over the
// entering directions, in order, and spread over the leaving ones), each direction's additions
// added to lambda^n, and the per-position sums over the directions, in order, to corr.  Reads of
// the scratch rows and, for y and z walls, the lambda^n updates are coalesced across threads.
__global__ void __launch_bounds__(kWallThreads) k_adj_walls_bl(const StepArgs a, int ax, const float *scratch,
                                                               float *lam_out, float *corr, long long nlines) {
    const long long line = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (line >= nlines) return;
    const int k = blockIdx.y;
    const int nd = a.nd, n = a.n[ax];
    int c[3];
    {
        const int o1 = ax == 0 ? 1 : 0, o2 = ax == 2 ? 1 : 2;
        c[ax] = 0;
        c[o1] = (int)(line % a.n[o1]);
        c[o2] = (int)(line / a.n[o1]);
    }
    const long long i0 = ((long long)c[2] * a.n[1] + c[1]) * a.n[0] + c[0];
    const long long st = a.stride[ax];
    auto sc = [&](int d, int j) { return scratch[((long long)(k * nd + d) * 8 + j) * nlines + line]; };
    float gam[2] = {0.f, 0.f};
    for (int side = 0; side < 2; ++side) {
        const int in = side ? -1 : 1;
        if (a.bc[2 * ax + side] != kBcDiffuse) continue;
        float sum = 0.f;
        for (int d = 0; d < nd; ++d) {
            const float nu = a.nu[3 * (k * nd + d) + ax];
            if (nu != 0.f && (nu > 0.f ? 1 : -1) == in) sum += sc(d, 4 * side + 2) + sc(d, 4 * side + 3);
        }
        gam[side] = sum;
    }
    float tot[4] = {0.f, 0.f, 0.f, 0.f};
    for (int d = 0; d < nd; ++d) {
        const float nu = a.nu[3 * (k * nd + d) + ax];
        float dv[4] = {0.f, 0.f, 0.f, 0.f};
        for (int side = 0; side < 2; ++side) {
            const int wall = 2 * ax + side, bc = a.bc[wall];
            if (bc == kBcPeriodic) continue;
            const int w0 = side ? n - 1 : 0, in = side ? -1 : 1;
            float v0 = sc(d, 4 * side), v1 = sc(d, 4 * side + 1);
            const bool leaving = nu != 0.f && (nu > 0.f ? 1 : -1) != in;
            if (bc == kBcSpecular) {
                const int dm = a.mirror[ax * nd + d];
                v0 += sc(dm, 4 * side + 2);
                v1 += sc(dm, 4 * side + 3);
            } else if (leaving) {
                v0 += sc(d, 4 * side + 2);
            }
            if (bc == kBcDiffuse) v0 = fmaf(a.wdiff[wall * nd + d] * a.inv_den[wall], gam[side], v0);
            dv[wall_slot(w0, n)] += v0;
            dv[wall_slot(w0 + in, n)] += v1;
        }
        const long long pb = (long long)(k * nd + d) * a.ncell + i0;
        #pragma unroll
        for (int sl = 0; sl < 4; ++sl) {
            tot[sl] += dv[sl];
            const int pos = sl < 2 ? sl : n - 2 + (sl - 2);
            if (dv[sl] != 0.f && (sl < 2 || pos >= 2)) lam_out[pb + (long long)pos * st] += dv[sl];
        }
    }
    #pragma unroll
    for (int sl = 0; sl < 4; ++sl) corr[((long long)k * 4 + sl) * nlines + line] = tot[sl];
}

// Phase 2 for few lines: one block per (line, band), threads over the directions (the same
// sums, in the same order): the ghost transposes
// (specular: the mirrored direction's ghost adjoints; thermalizing or diffuse outgoing: the
// direction's own; diffuse incoming: summed over the entering directions, in order, and spread
// over the leaving ones), each direction's additions written to lambda^n by its own thread,
// and the per-position sums over the directions, in order, to corr.  Dynamic shared memory:
// 8 nd floats.
__global__ void __launch_bounds__(kWallThreads) k_adj_walls_b(const StepArgs a, int ax, const float *scratch,
                                                              float *lam_out, float *corr, long long nlines) {
    extern __shared__ float wsh[];
    const int nd = a.nd;
    float *gh = wsh;            // [side][layer][d]: ghost adjoints
    float *tot = wsh + 4 * nd;  // [slot][d]
    __shared__ float gam[2];
    const long long line = blockIdx.x;
    const int k = blockIdx.y;
    const int n = a.n[ax];
    int c[3];
    {
        const int o1 = ax == 0 ? 1 : 0, o2 = ax == 2 ? 1 : 2;
        c[ax] = 0;
        c[o1] = (int)(line % a.n[o1]);
        c[o2] = (int)(line / a.n[o1]);
    }
    const long long i0 = ((long long)c[2] * a.n[1] + c[1]) * a.n[0] + c[0];
    const long long st = a.stride[ax];
    auto sc = [&](int d, int j) { return scratch[((long long)(k * nd + d) * 8 + j) * nlines + line]; };
    for (int d = threadIdx.x; d < nd; d += blockDim.x)
        for (int side = 0; side < 2; ++side) {
            gh[(2 * side) * nd + d] = sc(d, 4 * side + 2);
            gh[(2 * side + 1) * nd + d] = sc(d, 4 * side + 3);
        }
    __syncthreads();
    if (threadIdx.x < 2) {
        const int side = threadIdx.x, in = side ? -1 : 1;
        float sum = 0.f;
        if (a.bc[2 * ax + side] == kBcDiffuse)
            for (int d = 0; d < nd; ++d) {
                const float nu = a.nu[3 * (k * nd + d) + ax];
                if (nu != 0.f && (nu > 0.f ? 1 : -1) == in) sum += gh[(2 * side) * nd + d] + gh[(2 * side + 1) * nd + d];
            }
        gam[side] = sum;
    }
    __syncthreads();
    for (int d = threadIdx.x; d < nd; d += blockDim.x) {
        const float nu = a.nu[3 * (k * nd + d) + ax];
        float dv[4] = {0.f, 0.f, 0.f, 0.f};
        for (int side = 0; side < 2; ++side) {
            const int wall = 2 * ax + side, bc = a.bc[wall];
            if (bc == kBcPeriodic) continue;
            const int w0 = side ? n - 1 : 0, in = side ? -1 : 1;
            float v0 = sc(d, 4 * side), v1 = sc(d, 4 * side + 1);
            const bool leaving = nu != 0.f && (nu > 0.f ? 1 : -1) != in;
            if (bc == kBcSpecular) {
                const int dm = a.mirror[ax * nd + d];
                v0 += gh[(2 * side) * nd + dm];
                v1 += gh[(2 * side + 1) * nd + dm];
            } else if (leaving) {
                v0 += gh[(2 * side) * nd + d];
            }
            if (bc == kBcDiffuse) v0 = fmaf(a.wdiff[wall * nd + d] * a.inv_den[wall], gam[side], v0);
            dv[wall_slot(w0, n)] += v0;
            dv[wall_slot(w0 + in, n)] += v1;
        }
        const long long pb = (long long)(k * nd + d) * a.ncell + i0;
        #pragma unroll
        for (int sl = 0; sl < 4; ++sl) {
            tot[sl * nd + d] = dv[sl];
            const int pos = sl < 2 ? sl : n - 2 + (sl - 2);
            if (dv[sl] != 0.f && (sl < 2 || pos >= 2)) lam_out[pb + (long long)pos * st] += dv[sl];
        }
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        float sum = 0.f;
        for (int d = 0; d < nd; ++d) sum += tot[threadIdx.x * nd + d];
        corr[((long long)k * 4 + threadIdx.x) * nlines + line] = sum;
    }
}

// Tiled finalize: mu^n_i = sum of the tile's segment rows (Pm) plus the wall corrections;
// q^n_i likewise (Pq); dJ/dQ_i += amp q^n_i; the band-independent log-tau sum
// sum_i mu^{n+1}_i T_L,i^n in FP64 block partials.
__global__ void __launch_bounds__(256) k_adj_tfinal(const StepArgs a, AdjTFinal f, float amp, float *mu_out,
                                                    double *gQ, double *mt_part) {
    __shared__ double sh[256];
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double mt = 0.0;
    if (i < a.ncell) {
        const int nx = a.n[0], ny = a.n[1];
        const int c[3] = {(int)(i % nx), (int)((i / nx) % ny), (int)(i / ((long long)nx * ny))};
        const int ty = c[1] / f.ty, tz = c[2] / f.tz;
        const int tile = tz * f.nty + ty;
        const int li = ((c[2] - tz * f.tz) * f.ty + (c[1] - ty * f.ty)) * nx + c[0];
        float m = 0.f, q = 0.f;
        for (int s = f.tile_seg0[tile]; s < f.tile_seg0[tile + 1]; ++s) {
            m += f.Pm[(size_t)s * f.tcells + li];
            q += f.Pq[(size_t)s * f.tcells + li];
        }
        for (int ax = 0; ax < a.dim; ++ax) {
            if (a.bc[2 * ax] == kBcPeriodic) continue;
            const int n = a.n[ax], pos = c[ax];
            if (pos >= 2 && pos < n - 2) continue;
            const int o1 = ax == 0 ? 1 : 0, o2 = ax == 2 ? 1 : 2;
            const long long nl = (long long)a.n[o1] * a.n[o2], line = (long long)c[o2] * a.n[o1] + c[o1];
            const int sl = wall_slot(pos, n);
            for (int k = 0; k < a.nb; ++k) {
                const float v = f.corr[ax][((long long)k * 4 + sl) * nl + line];
                const BandConst b = a.band[k];
                m = fmaf(b.dtinv * b.ck, v, m);
                q = fmaf(b.srck, v, q);
            }
        }
        mu_out[i] = m;
        gQ[i] += (double)amp * (double)q;
        mt = (double)f.mu_in[i] * (double)a.TL[i];
    }
    sh[threadIdx.x] = mt;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) sh[threadIdx.x] += sh[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) mt_part[blockIdx.x] = sh[0];
}

// dJ/dlog tau_k += sum over band k's segments of (-dt/tau_k Ps0 - Ps1/(tau_k D))
//                 + C_k/(tau_k D) sum_i mu^{n+1}_i T_L,i^n: one block per band, each thread a fixed
// strided subset, then a fixed-order tree.
constexpr int kTauThreads = 256;
__global__ void __launch_bounds__(kTauThreads) k_adj_ttau(const StepArgs a, AdjTFinal f, const double *mt_part, int nmt,
                                                          double W, double *gtau) {
    __shared__ double sh[2][kTauThreads];
    const int k = blockIdx.x;
    const BandConst b = a.band[k];
    double s = 0.0, mt = 0.0;
    for (int g = threadIdx.x; g < f.G; g += kTauThreads)
        if (f.seg_band[g] == k)
            s += -(double)b.dtinv * (double)f.Ps[2 * g] - (double)f.Ps[2 * g + 1] * (double)b.wtau * (double)a.invD;
    for (int j = threadIdx.x; j < nmt; j += kTauThreads) mt += mt_part[j];
    sh[0][threadIdx.x] = s;
    sh[1][threadIdx.x] = mt;
    __syncthreads();
    for (int h = kTauThreads / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + h];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + h];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) gtau[k] += sh[0][0] + (double)b.ck * W * (double)b.wtau * (double)a.invD * sh[1][0];
}

cudaError_t launch_adj_walls(const StepArgs &a, const AdjArgs &g, int storage, int limiter, float *lam_out,
                             float *const corr[3], float *scratch, cudaStream_t s) {
    for (int ax = 0; ax < a.dim; ++ax) {
        if (a.bc[2 * ax] == kBcPeriodic) continue;
        const int o1 = ax == 0 ? 1 : 0, o2 = ax == 2 ? 1 : 2;
        const long long nl = (long long)a.n[o1] * a.n[o2];
        const unsigned nbl = (unsigned)((nl + kWallThreads - 1) / kWallThreads);
        const dim3 ga(nbl, (unsigned)a.nd, (unsigned)a.nb);
#define BTE_ADJW(SS, LL) k_adj_walls_a<SS, LL><<<ga, kWallThreads, 0, s>>>(a, g, ax, scratch, nl)
        if (storage == kStoreF32) {
            if (limiter == kLimFirst) BTE_ADJW(kStoreF32, kLimFirst);
            else if (limiter == kLimMinmod) BTE_ADJW(kStoreF32, kLimMinmod);
            else BTE_ADJW(kStoreF32, kLimVanAlbada);
        } else if (storage == kStoreF16) {
            if (limiter == kLimFirst) BTE_ADJW(kStoreF16, kLimFirst);
            else if (limiter == kLimMinmod) BTE_ADJW(kStoreF16, kLimMinmod);
            else BTE_ADJW(kStoreF16, kLimVanAlbada);
        } else {
            if (limiter == kLimFirst) BTE_ADJW(kStoreBF16, kLimFirst);
            else if (limiter == kLimMinmod) BTE_ADJW(kStoreBF16, kLimMinmod);
            else BTE_ADJW(kStoreBF16, kLimVanAlbada);
        }
#undef BTE_ADJW
        // a thread per (line, band) when they fill the GPU many times over, else a block each
        // (BTE_ADJ_WALL_LINES overrides the bound, for tests of both forms)
        long long lines_min = kWallLineThreads;
        if (const char *env = std::getenv("BTE_ADJ_WALL_LINES")) lines_min = std::atoll(env);
        if (nl * a.nb >= lines_min) {
            k_adj_walls_bl<<<dim3(nbl, (unsigned)a.nb), kWallThreads, 0, s>>>(a, ax, scratch, lam_out, corr[ax], nl);
        } else {
            const int tb = std::min(kWallThreads, (a.nd + 31) / 32 * 32);  // no idle warp for nd < 128
            k_adj_walls_b<<<dim3((unsigned)nl, (unsigned)a.nb), tb, (size_t)8 * a.nd * sizeof(float), s>>>(
                a, ax, scratch, lam_out, corr[ax], nl);
        }
    }
    return cudaGetLastError();
}

int adj_walls_max_dirs() { return 6144; }  // 8 nd floats of dynamic shared memory <= 192 KB

long long adj_walls_scratch_floats(const StepArgs &a) {
    long long m = 0;
    for (int ax = 0; ax < a.dim; ++ax) {
        if (a.bc[2 * ax] == kBcPeriodic) continue;
        const int o1 = ax == 0 ? 1 : 0, o2 = ax == 2 ? 1 : 2;
        m = std::max(m, (long long)a.n[o1] * a.n[o2]);
    }
    return m * 8 * (long long)a.nb * a.nd;
}

cudaError_t launch_adj_tfinal(const StepArgs &a, const AdjTFinal &f, float amp, float *mu_out, double *gQ,
                              double *mt_part, double W, double *gtau, cudaStream_t s) {
    const int nblk = (int)((a.ncell + 255) / 256);
    k_adj_tfinal<<<nblk, 256, 0, s>>>(a, f, amp, mu_out, gQ, mt_part);
    k_adj_ttau<<<a.nb, kTauThreads, 0, s>>>(a, f, mt_part, nblk, W, gtau);
    return cudaGetLastError();
}

template <int S>
static void adj_step_s(const StepArgs &a, const AdjArgs &g, int limiter, cudaStream_t s) {
    const dim3 grid((unsigned)((a.ncell + 255) / 256), (unsigned)a.nb);
    if (limiter == kLimFirst) k_adj_step<S, kLimFirst><<<grid, 256, 0, s>>>(a, g);
    else if (limiter == kLimMinmod) k_adj_step<S, kLimMinmod><<<grid, 256, 0, s>>>(a, g);
    else k_adj_step<S, kLimVanAlbada><<<grid, 256, 0, s>>>(a, g);
}

cudaError_t launch_adj_step(const StepArgs &a, const AdjArgs &g, int storage, int limiter, cudaStream_t s) {
    if (storage == kStoreF32) adj_step_s<kStoreF32>(a, g, limiter, s);
    else if (storage == kStoreF16) adj_step_s<kStoreF16>(a, g, limiter, s);
    else adj_step_s<kStoreBF16>(a, g, limiter, s);
    return cudaGetLastError();
}

cudaError_t launch_adj_init(const StepArgs &a, const AdjArgs &g, int storage, const float *probe, cudaStream_t s) {
    const dim3 grid((unsigned)((a.ncell + 255) / 256), (unsigned)a.nb);
    if (storage == kStoreF32) k_adj_init<kStoreF32><<<grid, 256, 0, s>>>(a, g, probe);
    else if (storage == kStoreF16) k_adj_init<kStoreF16><<<grid, 256, 0, s>>>(a, g, probe);
    else k_adj_init<kStoreBF16><<<grid, 256, 0, s>>>(a, g, probe);
    return cudaGetLastError();
}

cudaError_t launch_adj_reduce(const StepArgs &a, const AdjArgs &g, float amp, float *mu_out, double *gQ,
                              double *tau_part, double *gtau, cudaStream_t s) {
    k_adj_cells<<<(unsigned)((a.ncell + 255) / 256), 256, 0, s>>>(a, g, amp, mu_out, gQ);
    const int nblk = adj_tau_blocks(a.ncell);
    k_adj_tau_blocks<<<dim3((unsigned)nblk, (unsigned)a.nb), kTauBlock, 0, s>>>(g, a.ncell, tau_part, nblk);
    k_adj_tau_sum<<<(a.nb + 127) / 128, 128, 0, s>>>(tau_part, nblk, a.nb, gtau);
    return cudaGetLastError();
}

}  // namespace bte
