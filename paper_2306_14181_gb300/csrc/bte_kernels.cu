// Generic kernels of the GB300 explicit DOM transient step (arXiv 2306.14181, Sec. 4):
// equilibrium fill, the per-(cell, band) forward step for any grid shape, the moment-only
// pass, the T_L finalisation and the FP64 diagnostics.  The shared-memory tiled forward
// kernel lives in bte_tiled.cu.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <mutex>

#include "bte_device.cuh"

namespace bte {

// ------------------------------------------------------------------------------------------
// Generic forward step: one thread per (cell, band), looping over the band's directions.
// Eq. (disretized_transientBTE) with the limited upwind face value of Sec. 4.1, in upwind
// orientation: with sg = sign(nu_a) and u_j = e(i + j sg),
//   e_out = u_0 + L(u_0 - u_-1, u_1 - u_0)/2,  e_in = u_-1 + L(u_-1 - u_-2, u_0 - u_-1)/2,
//   e^{n+1} = e - sum_a |nu_a| (e_out - e_in) + dt/tau (C T_L / W - e) + a Q dt C/(sum C W).
// The same pass accumulates the T_L moment sum_d w_d e^{n+1}/tau_k (Eq. BTE_get_e0) into
// P[k][i] and, at diffuse walls, the outgoing sums of Eq. (diff_bound) for the next step.
// ------------------------------------------------------------------------------------------
// Threads of a block: blockDim.x cells by blockDim.y direction groups (256 in all); group g
// takes the directions g, g + blockDim.y, ...  Small grids (few cells and bands) split a band's
// directions over up to 32 groups so that the launch still fills the GPU; the groups' moment and
// diffuse-wall partials are then summed in group order in shared memory, so the result is
// deterministic for a given grid.
template <int S, int LIM>
__global__ void __launch_bounds__(256) k_step_generic(const StepArgs a) {
    using Cd = Codec<S>;
    using T = typename Cd::T;
    __shared__ float red[4][256];  // moment and up to three diffuse walls (one per axis) per thread
    const int ng = blockDim.y, grp = threadIdx.y, tid = threadIdx.y * blockDim.x + threadIdx.x;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = i < a.ncell;
    const int k = blockIdx.y;
    int c[3] = {0, 0, 0};
    const BandConst b = a.band[k];
    int wl[6];
    int nw = 0;
    float wacc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    float acc = 0.f;
    float rho_new = 0.f;
    if (valid) {
        cell_coords(a, i, c);
        const T *ein = static_cast<const T *>(a.e_in);
        T *eout = static_cast<T *>(a.e_out);
        const float eq = b.ck * a.TL[i];
        const float rho_i = rho_at<Cd>(a.R, a.invTs, i);
        rho_new = rho_at<Cd>(a.TL, a.invTs, i);
        const float src = a.Q ? b.srck * (a.amp * a.Q[i]) : 0.f;
        nw = diffuse_walls_of(a, c, wl);
        for (int d = grp; d < a.nd; d += ng) {
            const int plane = k * a.nd + d;
            const long long base = (long long)plane * a.ncell;
            const float e0 = Cd::ld(ein, base + i, b, rho_i);
            float div = 0.f;
            for (int ax = 0; ax < a.dim; ++ax) {
                const float nu = a.nu[plane * 3 + ax];
                if (nu == 0.f) continue;
                const int sg = nu > 0.f ? 1 : -1;
                const float um2 = ext_value<Cd>(a, ein, b, k, d, base, i, c, ax, c[ax] - 2 * sg, nu);
                const float um1 = ext_value<Cd>(a, ein, b, k, d, base, i, c, ax, c[ax] - sg, nu);
                const float up1 = ext_value<Cd>(a, ein, b, k, d, base, i, c, ax, c[ax] + sg, nu);
                const float fo = e0 + 0.5f * limit<LIM>(e0 - um1, up1 - e0);
                const float fi = um1 + 0.5f * limit<LIM>(um1 - um2, e0 - um1);
                div += fabsf(nu) * (fo - fi);
            }
            const float en = e0 - div + b.dtinv * (eq - e0) + src;
            const float es = a.sr ? Cd::st_sr(eout, base + i, en, b, rho_new, mix32(plane_key(a.srkey, plane) ^ (uint32_t)i))
                                  : Cd::st(eout, base + i, en, b, rho_new);
            acc += a.wmom[plane] * es;
            for (int j = 0; j < nw; ++j) wacc[j] += a.wdiff[wl[j] * a.nd + d] * es;
        }
    }
    if (ng > 1) {
        // group partials, summed in group order by group 0
        red[0][tid] = acc;
        for (int j = 0; j < 3; ++j) red[1 + j][tid] = j < nw ? wacc[j] : 0.f;
        __syncthreads();
        if (grp == 0) {
            for (int g = 1; g < ng; ++g) {
                const int t = g * blockDim.x + threadIdx.x;
                acc += red[0][t];
                for (int j = 0; j < nw && j < 3; ++j) wacc[j] += red[1 + j][t];
            }
        }
    }
    if (!valid || grp != 0) return;
    a.P[(long long)k * a.ncell + i] = acc;
    for (int j = 0; j < nw; ++j) {
        const int w = wl[j];
        Cd::st(static_cast<T *>(a.ediff_out), ((long long)w * a.nb + k) * a.wc_max + wall_cell(a, w >> 1, c),
               wacc[j] * a.inv_den[w], b, rho_new);
    }
}

// Thermalizing-wall emission C_k T_w / W of band k as a ghost code against the reference rho of
// wall cell i (16-bit storage; the tiled kernel copies these rows like diffuse-wall rows).
template <class Cd>
__device__ __forceinline__ void store_iso_codes(const StepArgs &a, int k, long long i, const int c[3], float rho,
                                                const BandConst &b) {
    if constexpr (Cd::kRef) {
        for (int w = 0; w < 2 * a.dim; ++w) {
            const int ax = w >> 1;
            if (a.bc[w] != kBcIsothermal || c[ax] != ((w & 1) ? a.n[ax] - 1 : 0)) continue;
            Cd::st(static_cast<typename Cd::T *>(a.ediff_out), ((long long)w * a.nb + k) * a.wc_max + wall_cell(a, ax, c),
                   a.iso[w * a.nb + k], b, rho);
        }
    }
}

// Moment partials and wall ghost values of the current state without stepping (after an
// equilibrium fill or a state upload).  Writes P[k][i] and ediff_out.
template <int S>
__global__ void __launch_bounds__(256) k_moment_only(const StepArgs a) {
    using Cd = Codec<S>;
    using T = typename Cd::T;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.ncell) return;
    const int k = blockIdx.y;
    int c[3];
    cell_coords(a, i, c);
    const BandConst b = a.band[k];
    const T *e = static_cast<const T *>(a.e_in);
    const float rho_i = rho_at<Cd>(a.R, a.invTs, i);
    int wl[6];
    const int nw = diffuse_walls_of(a, c, wl);
    float wacc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    float acc = 0.f;
    for (int d = 0; d < a.nd; ++d) {
        const int plane = k * a.nd + d;
        const float es = Cd::ld(e, (long long)plane * a.ncell + i, b, rho_i);
        acc += a.wmom[plane] * es;
        for (int j = 0; j < nw; ++j) wacc[j] += a.wdiff[wl[j] * a.nd + d] * es;
    }
    a.P[(long long)k * a.ncell + i] = acc;
    for (int j = 0; j < nw; ++j) {
        const int w = wl[j];
        Cd::st(static_cast<T *>(a.ediff_out), ((long long)w * a.nb + k) * a.wc_max + wall_cell(a, w >> 1, c),
               wacc[j] * a.inv_den[w], b, rho_i);
    }
    store_iso_codes<Cd>(a, k, i, c, rho_i, b);
}

// T_L_i = (sum_g P[g][i]) / sum_k C_k/tau_k, Eq. (BTE_get_e0), summed in fixed g order.
__global__ void __launch_bounds__(256) k_finalize(const float *__restrict__ P, int G, long long ncell, float invD,
                                                  float *__restrict__ TL) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ncell) return;
    float s = 0.f;
    for (int g = 0; g < G; ++g) s += P[(long long)g * ncell + i];
    TL[i] = s * invD;
}

// Equilibrium fill e_{k,d,i} = C_k dT0_i / W (Algorithm 2, initial state); the code reference
// of the filled state is dT0 itself (written to R_out by the plane-0 threads).
template <int S>
__global__ void __launch_bounds__(256) k_fill(const StepArgs a, const double *dT0, float *R_out) {
    using Cd = Codec<S>;
    using T = typename Cd::T;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.ncell) return;
    const int plane = blockIdx.y;
    const int k = plane / a.nd;
    const BandConst b = a.band[k];
    const float t = dT0 ? (float)dT0[i] : 0.f;
    if (plane == 0 && R_out) R_out[i] = t;
    Cd::st(static_cast<T *>(a.e_out), (long long)plane * a.ncell + i, b.ck * t, b, t * a.invTs);
}

// Decoded values e = s_k (h + rho_i) (or e itself for FP32) of the state e_in.
template <int S>
__global__ void __launch_bounds__(256) k_decode(const StepArgs a, float *out) {
    using Cd = Codec<S>;
    using T = typename Cd::T;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.ncell) return;
    const int plane = blockIdx.y;
    const BandConst b = a.band[plane / a.nd];
    const long long j = (long long)plane * a.ncell + i;
    out[j] = Cd::ld(static_cast<const T *>(a.e_in), j, b, rho_at<Cd>(a.R, a.invTs, i));
}

static dim3 cell_grid(long long ncell, int y) { return dim3((unsigned)((ncell + 255) / 256), (unsigned)y); }

template <int S>
static void fill_s(const StepArgs &a, const double *dT0, float *R_out, cudaStream_t s) {
    k_fill<S><<<cell_grid(a.ncell, a.nb * a.nd), 256, 0, s>>>(a, dT0, R_out);
}

cudaError_t launch_fill(const StepArgs &a, int storage, const double *dT0, float *R_out, cudaStream_t s) {
    if (storage == kStoreF32) fill_s<kStoreF32>(a, dT0, R_out, s);
    else if (storage == kStoreF16) fill_s<kStoreF16>(a, dT0, R_out, s);
    else fill_s<kStoreBF16>(a, dT0, R_out, s);
    return cudaGetLastError();
}

cudaError_t launch_decode(const StepArgs &a, int storage, float *out, cudaStream_t s) {
    const dim3 g = cell_grid(a.ncell, a.nb * a.nd);
    if (storage == kStoreF32) k_decode<kStoreF32><<<g, 256, 0, s>>>(a, out);
    else if (storage == kStoreF16) k_decode<kStoreF16><<<g, 256, 0, s>>>(a, out);
    else k_decode<kStoreBF16><<<g, 256, 0, s>>>(a, out);
    return cudaGetLastError();
}

cudaError_t launch_moment_only(const StepArgs &a, int storage, cudaStream_t s) {
    const dim3 g = cell_grid(a.ncell, a.nb);
    if (storage == kStoreF32) k_moment_only<kStoreF32><<<g, 256, 0, s>>>(a);
    else if (storage == kStoreF16) k_moment_only<kStoreF16><<<g, 256, 0, s>>>(a);
    else k_moment_only<kStoreBF16><<<g, 256, 0, s>>>(a);
    return cudaGetLastError();
}

// Direction groups of the generic step: one while cells x bands give at least 4096 blocks of 256
// threads' worth of work, else more (up to 32, no more than the directions), so that small grids
// still spread over the GPU's SMs.  In 1-D and 2-D at least 16 when there are 32 directions or
// more: a block of 16 cells by 16 groups ran the 256^2 hot spot 12 % faster than 256 cells by one
// group (in 3-D, with six neighbour rows a direction, it ran 3 % slower).
static int generic_direction_groups(long long ncell, int nb, int nd, int dim) {
    int ng = 1;
    while (ng < 32 && 2 * ng <= nd && ncell * nb * ng < 4096LL * 256) ng *= 2;
    if (dim <= 2 && nd >= 32 && ng < 16) ng = 16;
    return ng;
}

template <int S>
static void step_generic_s(const StepArgs &a, int limiter, cudaStream_t s) {
    const int ng = generic_direction_groups(a.ncell, a.nb, a.nd, a.dim);
    const dim3 blk(256 / ng, ng);
    const dim3 g((unsigned)((a.ncell + blk.x - 1) / blk.x), (unsigned)a.nb);
    if (limiter == kLimFirst) k_step_generic<S, kLimFirst><<<g, blk, 0, s>>>(a);
    else if (limiter == kLimMinmod) k_step_generic<S, kLimMinmod><<<g, blk, 0, s>>>(a);
    else k_step_generic<S, kLimVanAlbada><<<g, blk, 0, s>>>(a);
}

cudaError_t launch_step_generic(const StepArgs &a, int storage, int limiter, cudaStream_t s) {
    if (storage == kStoreF32) step_generic_s<kStoreF32>(a, limiter, s);
    else if (storage == kStoreF16) step_generic_s<kStoreF16>(a, limiter, s);
    else step_generic_s<kStoreBF16>(a, limiter, s);
    return cudaGetLastError();
}

cudaError_t launch_finalize(const StepArgs &a, int G, float *TL_out, cudaStream_t s) {
    k_finalize<<<cell_grid(a.ncell, 1), 256, 0, s>>>(a.P, G, a.ncell, a.invD, TL_out);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------
// FP64 diagnostics (off the timed path).
// ------------------------------------------------------------------------------------------

// Per-cell moments of Eq. (getTQ) and Eq. (BTE_get_e0), FP64 accumulation.
template <int S>
__global__ void __launch_bounds__(256) k_moments64(const StepArgs a, const double *w, const double *sv,
                                                   const double *v, const double *invtau, double sumC, double D,
                                                   DiagOut o) {
    using Cd = Codec<S>;
    using T = typename Cd::T;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.ncell) return;
    const T *e = static_cast<const T *>(a.e_in);
    const float rho_i = rho_at<Cd>(a.R, a.invTs, i);
    double et = 0.0, tl = 0.0, qx = 0.0, qy = 0.0, qz = 0.0;
    bool bad = false;
    for (int k = 0; k < a.nb; ++k) {
        const BandConst b = a.band[k];
        double sk = 0.0, sx = 0.0, sy = 0.0, sz = 0.0;
        for (int d = 0; d < a.nd; ++d) {
            const double ed = Cd::ld64(e, ((long long)k * a.nd + d) * a.ncell + i, b, rho_i);
            bad |= !isfinite(ed);
            const double we = w[d] * ed;
            sk += we;
            sx += we * sv[3 * d];
            sy += we * sv[3 * d + 1];
            sz += we * sv[3 * d + 2];
        }
        et += sk;
        tl += invtau[k] * sk;
        qx += v[k] * sx;
        qy += v[k] * sy;
        qz += v[k] * sz;
    }
    if (bad) atomicOr(o.nonfinite, 1);
    if (o.T) o.T[i] = et / sumC;
    if (o.TL) o.TL[i] = tl / D;
    if (o.q) {
        o.q[i] = qx;
        o.q[a.ncell + i] = qy;
        o.q[2 * a.ncell + i] = qz;
    }
    if (o.cellE) o.cellE[i] = et;
}

template <class Cd>
__device__ double ext64(const StepArgs &a, const typename Cd::T *e, const BandConst &b, int k, int d, long long i,
                        const int c[3], int ax, int pos, double sa) {
    const int n = a.n[ax];
    const long long st = a.stride[ax];
    const long long base = ((long long)k * a.nd + d) * a.ncell;
    if (pos >= 0 && pos < n) {
        const long long j = i + (long long)(pos - c[ax]) * st;
        return Cd::ld64(e, base + j, b, rho_at<Cd>(a.R, a.invTs, j));
    }
    const int side = pos < 0 ? 0 : 1;
    const int wall = 2 * ax + side;
    const int bc = a.bc[wall];
    if (bc == kBcPeriodic) {
        const long long j = i + (long long)((side ? pos - n : pos + n) - c[ax]) * st;
        const double off = (double)a.jmp[ax * a.nb + k];  // the step's FP32 jump offset
        return Cd::ld64(e, base + j, b, rho_at<Cd>(a.R, a.invTs, j)) + (side ? -off : off);
    }
    if (bc == kBcSpecular) {
        const int layer = side ? pos - n + 1 : -pos;
        const long long j = i + (long long)((side ? n - layer : layer - 1) - c[ax]) * st;
        const long long mbase = ((long long)k * a.nd + a.mirror[ax * a.nd + d]) * a.ncell;
        return Cd::ld64(e, mbase + j, b, rho_at<Cd>(a.R, a.invTs, j));
    }
    const bool incoming = side == 0 ? (sa > 0.0) : (sa < 0.0);
    const long long jw = i + (long long)((side ? n - 1 : 0) - c[ax]) * st;
    if (!incoming) return Cd::ld64(e, base + jw, b, rho_at<Cd>(a.R, a.invTs, jw));
    if (bc == kBcIsothermal) return (double)a.iso[wall * a.nb + k];
    return Cd::ld64(static_cast<const typename Cd::T *>(a.ediff_in),
                    ((long long)wall * a.nb + k) * a.wc_max + wall_cell(a, ax, c), b, rho_at<Cd>(a.R, a.invTs, jw));
}

// Outward heat flow through one wall, per (wall cell j, band k): sum_d w v (s.n) e_face, with
// e_face the wall-face value of the step (upwind side chosen by the sign of s_a).
template <int S>
__global__ void __launch_bounds__(256) k_wallflux64(const StepArgs a, int wall, int lim, const double *w,
                                                    const double *sv, const double *v, DiagOut o) {
    using Cd = Codec<S>;
    using T = typename Cd::T;
    const int ax = wall >> 1, side = wall & 1;
    const int n0 = ax == 0 ? a.n[1] : a.n[0];
    const int n1 = ax == 2 ? a.n[1] : a.n[2];
    const long long nwc = (long long)n0 * n1;
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int k = blockIdx.y;
    if (j >= nwc) return;
    int c[3];
    const int ja = (int)(j % n0), jb = (int)(j / n0);
    c[ax] = side ? a.n[ax] - 1 : 0;
    if (ax == 0) { c[1] = ja; c[2] = jb; }
    else if (ax == 1) { c[0] = ja; c[2] = jb; }
    else { c[0] = ja; c[1] = jb; }
    const long long i = c[0] + a.stride[1] * c[1] + a.stride[2] * c[2];
    const T *e = static_cast<const T *>(a.e_in);
    const BandConst b = a.band[k];
    const int n = a.n[ax];
    const double nsign = side ? 1.0 : -1.0;
    double F = 0.0;
    for (int d = 0; d < a.nd; ++d) {
        const double sa = sv[3 * d + ax];
        if (sa == 0.0) continue;
        const int sg = sa > 0.0 ? 1 : -1;
        // the wall face lies between p and p + sg along the flow, p = upwind cell
        const int pin = side ? n - 1 : 0;          // wall cell
        const int pg = side ? n : -1;              // first ghost
        const int pu = (sa * nsign > 0.0) ? pin : pg;  // upwind position: wall cell if leaving
        const double um = ext64<Cd>(a, e, b, k, d, i, c, ax, pu, sa);
        const double ul = ext64<Cd>(a, e, b, k, d, i, c, ax, pu - sg, sa);
        const double ur = ext64<Cd>(a, e, b, k, d, i, c, ax, pu + sg, sa);
        const double ef = um + 0.5 * limit64(lim, um - ul, ur - um);
        F += w[d] * v[k] * (nsign * sa) * ef;
    }
    o.wallpart[((long long)wall * a.nb + k) * a.wc_max + j] = F;
}

cudaError_t launch_moments64(const StepArgs &a, int storage, const double *w, const double *sv, const double *v,
                             const double *invtau, double sumC, double D, DiagOut o, cudaStream_t s) {
    const dim3 g = cell_grid(a.ncell, 1);
    if (storage == kStoreF32) k_moments64<kStoreF32><<<g, 256, 0, s>>>(a, w, sv, v, invtau, sumC, D, o);
    else if (storage == kStoreF16) k_moments64<kStoreF16><<<g, 256, 0, s>>>(a, w, sv, v, invtau, sumC, D, o);
    else k_moments64<kStoreBF16><<<g, 256, 0, s>>>(a, w, sv, v, invtau, sumC, D, o);
    return cudaGetLastError();
}

cudaError_t launch_wallflux64(const StepArgs &a, int storage, int limiter, const double *w, const double *sv,
                              const double *v, DiagOut o, cudaStream_t s) {
    for (int wall = 0; wall < 2 * a.dim; ++wall) {
        const int ax = wall >> 1;
        const long long nwc = ax == 0 ? (long long)a.n[1] * a.n[2]
                                      : (ax == 1 ? (long long)a.n[0] * a.n[2] : (long long)a.n[0] * a.n[1]);
        const dim3 g((unsigned)((nwc + 255) / 256), (unsigned)a.nb);
        if (storage == kStoreF32) k_wallflux64<kStoreF32><<<g, 256, 0, s>>>(a, wall, limiter, w, sv, v, o);
        else if (storage == kStoreF16) k_wallflux64<kStoreF16><<<g, 256, 0, s>>>(a, wall, limiter, w, sv, v, o);
        else k_wallflux64<kStoreBF16><<<g, 256, 0, s>>>(a, wall, limiter, w, sv, v, o);
    }
    return cudaGetLastError();
}

// Deterministic FP64 sum: fixed per-thread chunks, fixed tree order, then one block.
__global__ void __launch_bounds__(256) k_sum64_a(const double *x, long long n, double *part) {
    __shared__ double sm[256];
    const long long nb = gridDim.x;
    const long long chunk = (n + nb - 1) / nb;
    const long long lo = blockIdx.x * chunk;
    const long long hi = lo + chunk < n ? lo + chunk : n;
    double s = 0.0;
    for (long long t = lo + threadIdx.x; t < hi; t += blockDim.x) s += x[t];
    sm[threadIdx.x] = s;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) sm[threadIdx.x] += sm[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sm[0];
}

__global__ void __launch_bounds__(256) k_sum64_b(const double *part, int np, double *out) {
    __shared__ double sm[256];
    double s = 0.0;
    for (int t = threadIdx.x; t < np; t += blockDim.x) s += part[t];
    sm[threadIdx.x] = s;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) sm[threadIdx.x] += sm[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sm[0];
}

cudaError_t launch_sum64(const double *x, long long n, double *scratch, double *out, cudaStream_t s) {
    const int np = 1024;
    k_sum64_a<<<np, 256, 0, s>>>(x, n, scratch);
    k_sum64_b<<<1, 256, 0, s>>>(scratch, np, out);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------
// Residuals of the transient solver's loop condition (Algorithm 2) between consecutive states:
//   eps_T = sqrt(sum_i (T_i^n - T_i^{n+1})^2 / N) / T_max,
//   eps_q = sqrt(sum_i (|q|_i^n - |q|_i^{n+1})^2 / N) / |q|_max,
// T and q of Eq. (getTQ) in FP64.  k_resid_keep stores T^n and |q|^n; k_resid_a forms per-block
// partials of the two sums and the two maxima (T_max = max_i (T_ref + T_i^{n+1}), the absolute
// temperature; |q|_max = max_i |q_i^{n+1}|) in a fixed order; k_resid_b combines them.
// ------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_resid_keep(const double *T, const double *q, long long n, double *Tp,
                                                    double *qp) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    Tp[i] = T[i];
    qp[i] = sqrt(q[i] * q[i] + q[n + i] * q[n + i] + q[2 * n + i] * q[2 * n + i]);
}

__global__ void __launch_bounds__(256) k_resid_a(const double *T, const double *q, const double *Tp, const double *qp,
                                                 long long n, double Tref, double *part) {
    __shared__ double sm[4][256];
    const long long nb = gridDim.x;
    const long long chunk = (n + nb - 1) / nb;
    const long long lo = blockIdx.x * chunk;
    const long long hi = lo + chunk < n ? lo + chunk : n;
    double s1 = 0.0, s2 = 0.0, m1 = 0.0, m2 = 0.0;
    for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        const double qm = sqrt(q[i] * q[i] + q[n + i] * q[n + i] + q[2 * n + i] * q[2 * n + i]);
        const double dT = Tp[i] - T[i], dq = qp[i] - qm;
        s1 += dT * dT;
        s2 += dq * dq;
        m1 = fmax(m1, fabs(Tref + T[i]));
        m2 = fmax(m2, qm);
    }
    sm[0][threadIdx.x] = s1;
    sm[1][threadIdx.x] = s2;
    sm[2][threadIdx.x] = m1;
    sm[3][threadIdx.x] = m2;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) {
            sm[0][threadIdx.x] += sm[0][threadIdx.x + h];
            sm[1][threadIdx.x] += sm[1][threadIdx.x + h];
            sm[2][threadIdx.x] = fmax(sm[2][threadIdx.x], sm[2][threadIdx.x + h]);
            sm[3][threadIdx.x] = fmax(sm[3][threadIdx.x], sm[3][threadIdx.x + h]);
        }
        __syncthreads();
    }
    if (threadIdx.x < 4) part[threadIdx.x * nb + blockIdx.x] = sm[threadIdx.x][0];
}

__global__ void __launch_bounds__(256) k_resid_b(const double *part, int np, double *out) {
    __shared__ double sm[4][256];
    double r[4] = {0.0, 0.0, 0.0, 0.0};
    for (int t = threadIdx.x; t < np; t += blockDim.x) {
        r[0] += part[t];
        r[1] += part[np + t];
        r[2] = fmax(r[2], part[2 * np + t]);
        r[3] = fmax(r[3], part[3 * np + t]);
    }
    for (int j = 0; j < 4; ++j) sm[j][threadIdx.x] = r[j];
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) {
            sm[0][threadIdx.x] += sm[0][threadIdx.x + h];
            sm[1][threadIdx.x] += sm[1][threadIdx.x + h];
            sm[2][threadIdx.x] = fmax(sm[2][threadIdx.x], sm[2][threadIdx.x + h]);
            sm[3][threadIdx.x] = fmax(sm[3][threadIdx.x], sm[3][threadIdx.x + h]);
        }
        __syncthreads();
    }
    if (threadIdx.x < 4) out[threadIdx.x] = sm[threadIdx.x][0];
}

// ---- interface between two materials (Sec. 2.2 (v)) ------------------------------------------
__global__ void __launch_bounds__(256) k_iface_mix(float *__restrict__ eA, float *__restrict__ pa, int pure_a, int sa,
                                                   float *__restrict__ eB, float *__restrict__ pb, int pure_b, int sb,
                                                   const float *__restrict__ beta, int nb, int ncw) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x, k = blockIdx.y;
    if (j >= ncw) return;
    float *a = eA + (size_t)k * sa + j, *b = eB + (size_t)k * sb + j;
    float *qa = pa + (size_t)k * ncw + j, *qb = pb + (size_t)k * ncw + j;
    const float SA = pure_a ? *a : *qa, SB = pure_b ? *b : *qb;
    *qa = SA;
    *qb = SB;
    *a = fmaf(beta[2 * nb + k], SB, beta[nb + k] * SA);
    *b = fmaf(beta[k], SA, beta[3 * nb + k] * SB);
}

cudaError_t launch_iface_mix(float *eA, float *pa, int pure_a, int sa, float *eB, float *pb, int pure_b, int sb,
                             const float *beta, int nb, int ncw, cudaStream_t s) {
    const dim3 g((unsigned)((ncw + 255) / 256), (unsigned)nb);
    k_iface_mix<<<g, 256, 0, s>>>(eA, pa, pure_a, sa, eB, pb, pure_b, sb, beta, nb, ncw);
    return cudaGetLastError();
}

cudaError_t launch_resid_keep(const double *T, const double *q, long long n, double *Tp, double *qp, cudaStream_t s) {
    k_resid_keep<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(T, q, n, Tp, qp);
    return cudaGetLastError();
}

cudaError_t launch_residuals(const double *T, const double *q, const double *Tp, const double *qp, long long n,
                             double Tref, double *scratch, double *out4, cudaStream_t s) {
    const int np = kResidBlocks;
    k_resid_a<<<np, 256, 0, s>>>(T, q, Tp, qp, n, Tref, scratch);
    k_resid_b<<<1, 256, 0, s>>>(scratch, np, out4);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------
// Allocation-free variant of the FP64 energy-balance reduction.
//
// bte_energy stages per-cell sums and block partials in device buffers it allocates on first
// use.  This variant fuses the per-cell work into per-block FP64 partials and keeps them, the
// seven results and a non-finite flag in one file-scope device array, so a caller that may not
// allocate device memory can still take the reductions.  Each reduction (total energy and the
// six wall flows) has kNaSlots partial slots and a block covers kNaPerBlock items, which bounds
// the grids it accepts.  Every call overwrites the slots it reads and clears the flag, so no
// state carries over between calls; calls that overlap on the GPU share the array and race.
// ------------------------------------------------------------------------------------------
constexpr int kNaThreads = 256;
constexpr int kNaSlots = 2048;                      // block partials per reduction
constexpr long long kNaPerBlock = kNaThreads * 16;  // items a block covers
constexpr int kNaReductions = 7;                    // E_total, wall flows -x..+z
constexpr int kNaResults = kNaReductions * kNaSlots;   // 7 results follow the partials
constexpr int kNaFlag = kNaResults + kNaReductions;    // then the non-finite flag (as a double slot)
static __device__ __align__(256) double g_na_scratch[kNaFlag + 1];

long long energy_noalloc_max_items() { return (long long)kNaSlots * kNaPerBlock; }

// fixed-order block sum of one double per thread
__device__ __forceinline__ double na_block_sum(double v) {
    __shared__ double sm[kNaThreads];
    sm[threadIdx.x] = v;
    __syncthreads();
    for (int h = kNaThreads / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) sm[threadIdx.x] += sm[threadIdx.x + h];
        __syncthreads();
    }
    return sm[0];
}

// partial[b] = sum over the cells b covers of sum_k sum_d w_d e (Eq. getTQ numerator)
template <int S>
__global__ void __launch_bounds__(kNaThreads) k_na_energy(const StepArgs a, const double *w, double *scratch) {
    using Cd = Codec<S>;
    using T = typename Cd::T;
    const T *e = static_cast<const T *>(a.e_in);
    const long long lo = (long long)blockIdx.x * kNaPerBlock;
    const long long hi = lo + kNaPerBlock < a.ncell ? lo + kNaPerBlock : a.ncell;
    double acc = 0.0;
    bool bad = false;
    for (long long i = lo + threadIdx.x; i < hi; i += kNaThreads) {
        const float rho_i = rho_at<Cd>(a.R, a.invTs, i);
        double et = 0.0;
        for (int k = 0; k < a.nb; ++k) {
            const BandConst b = a.band[k];
            double sk = 0.0;
            for (int d = 0; d < a.nd; ++d) {
                const double ed = Cd::ld64(e, ((long long)k * a.nd + d) * a.ncell + i, b, rho_i);
                bad |= !isfinite(ed);
                sk += w[d] * ed;
            }
            et += sk;
        }
        acc += et;
    }
    const double tot = na_block_sum(acc);
    if (bad) scratch[kNaFlag] = 1.0;
    if (threadIdx.x == 0) scratch[blockIdx.x] = tot;
}

// partial[b] of wall `wall` = sum over the (wall cell, band) items b covers of
// sum_d w_d v_k (s_d.n) e_face, e_face the wall-face value of the step
template <int S>
__global__ void __launch_bounds__(kNaThreads) k_na_wallflux(const StepArgs a, int wall, int lim, const double *w,
                                                            const double *sv, const double *v, double *scratch) {
    using Cd = Codec<S>;
    using T = typename Cd::T;
    const int ax = wall >> 1, side = wall & 1;
    const int n0 = ax == 0 ? a.n[1] : a.n[0];
    const int n1 = ax == 2 ? a.n[1] : a.n[2];
    const long long nwc = (long long)n0 * n1, nitem = nwc * a.nb;
    const long long lo = (long long)blockIdx.x * kNaPerBlock;
    const long long hi = lo + kNaPerBlock < nitem ? lo + kNaPerBlock : nitem;
    const T *e = static_cast<const T *>(a.e_in);
    const int n = a.n[ax];
    const double nsign = side ? 1.0 : -1.0;
    double acc = 0.0;
    for (long long it = lo + threadIdx.x; it < hi; it += kNaThreads) {
        const int k = (int)(it / nwc);
        const long long j = it - (long long)k * nwc;
        int c[3];
        const int ja = (int)(j % n0), jb = (int)(j / n0);
        c[ax] = side ? n - 1 : 0;
        if (ax == 0) { c[1] = ja; c[2] = jb; }
        else if (ax == 1) { c[0] = ja; c[2] = jb; }
        else { c[0] = ja; c[1] = jb; }
        const long long i = c[0] + a.stride[1] * c[1] + a.stride[2] * c[2];
        const BandConst b = a.band[k];
        double F = 0.0;
        for (int d = 0; d < a.nd; ++d) {
            const double sa = sv[3 * d + ax];
            if (sa == 0.0) continue;
            const int sg = sa > 0.0 ? 1 : -1;
            const int pu = (sa * nsign > 0.0) ? (side ? n - 1 : 0) : (side ? n : -1);  // upwind position
            const double um = ext64<Cd>(a, e, b, k, d, i, c, ax, pu, sa);
            const double ul = ext64<Cd>(a, e, b, k, d, i, c, ax, pu - sg, sa);
            const double ur = ext64<Cd>(a, e, b, k, d, i, c, ax, pu + sg, sa);
            F += w[d] * v[k] * (nsign * sa) * (um + 0.5 * limit64(lim, um - ul, ur - um));
        }
        acc += F;
    }
    const double tot = na_block_sum(acc);
    if (threadIdx.x == 0) scratch[(1 + wall) * kNaSlots + blockIdx.x] = tot;
}

// result[r] = sum of the nblk[r] partials of reduction r, in slot order (one block per r)
struct NaCounts {
    int nblk[kNaReductions];
};
__global__ void __launch_bounds__(kNaThreads) k_na_finish(NaCounts cnt, double *scratch) {
    const int r = blockIdx.x;
    double acc = 0.0;
    for (int t = threadIdx.x; t < cnt.nblk[r]; t += kNaThreads) acc += scratch[r * kNaSlots + t];
    const double tot = na_block_sum(acc);
    if (threadIdx.x == 0) scratch[kNaResults + r] = tot;
}

// Device address of g_na_scratch, looked up once per device on the first call made with that
// device current (that first call must come before any stream capture).
static double *na_scratch_address(cudaError_t *err) {
    static std::mutex mu;
    static double *addr[64] = {};
    int dev = 0;
    if ((*err = cudaGetDevice(&dev)) != cudaSuccess) return nullptr;
    if (dev < 0 || dev >= 64) {
        *err = cudaErrorInvalidDevice;
        return nullptr;
    }
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev]) {
        void *p = nullptr;
        if ((*err = cudaGetSymbolAddress(&p, g_na_scratch)) != cudaSuccess) return nullptr;
        addr[dev] = static_cast<double *>(p);
    }
    *err = cudaSuccess;
    return addr[dev];
}

int launch_energy_noalloc(const StepArgs &a, int storage, int limiter, const double *w, const double *sv,
                          const double *v, double *host7, int *nonfinite, cudaStream_t s, cudaError_t *err) {
    // item counts of the seven reductions, checked against the fixed partial slots
    NaCounts cnt;
    long long items[kNaReductions];
    items[0] = a.ncell;
    for (int wl = 0; wl < 6; ++wl) {
        const int ax = wl >> 1;
        const long long nwc = ax == 0 ? (long long)a.n[1] * a.n[2] : (ax == 1 ? (long long)a.n[0] * a.n[2] : (long long)a.n[0] * a.n[1]);
        items[1 + wl] = wl < 2 * a.dim ? nwc * a.nb : 0;
    }
    for (int r = 0; r < kNaReductions; ++r) {
        if (items[r] > energy_noalloc_max_items()) return 1;  // too large for the fixed slots
        cnt.nblk[r] = (int)((items[r] + kNaPerBlock - 1) / kNaPerBlock);
    }
    double *scratch = na_scratch_address(err);
    if (!scratch) return 2;
    // the flag must start at zero; partials and results are overwritten before they are read
    if ((*err = cudaMemsetAsync(scratch + kNaFlag, 0, sizeof(double), s)) != cudaSuccess) return 2;
    if (cnt.nblk[0] > 0) {
        if (storage == kStoreF32) k_na_energy<kStoreF32><<<cnt.nblk[0], kNaThreads, 0, s>>>(a, w, scratch);
        else if (storage == kStoreF16) k_na_energy<kStoreF16><<<cnt.nblk[0], kNaThreads, 0, s>>>(a, w, scratch);
        else k_na_energy<kStoreBF16><<<cnt.nblk[0], kNaThreads, 0, s>>>(a, w, scratch);
    }
    for (int wl = 0; wl < 2 * a.dim; ++wl) {
        if (cnt.nblk[1 + wl] == 0) continue;
        if (storage == kStoreF32) k_na_wallflux<kStoreF32><<<cnt.nblk[1 + wl], kNaThreads, 0, s>>>(a, wl, limiter, w, sv, v, scratch);
        else if (storage == kStoreF16) k_na_wallflux<kStoreF16><<<cnt.nblk[1 + wl], kNaThreads, 0, s>>>(a, wl, limiter, w, sv, v, scratch);
        else k_na_wallflux<kStoreBF16><<<cnt.nblk[1 + wl], kNaThreads, 0, s>>>(a, wl, limiter, w, sv, v, scratch);
    }
    k_na_finish<<<kNaReductions, kNaThreads, 0, s>>>(cnt, scratch);
    if ((*err = cudaGetLastError()) != cudaSuccess) return 2;
    double flag = 0.0;
    if ((*err = cudaMemcpyAsync(host7, scratch + kNaResults, kNaReductions * sizeof(double), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (*err = cudaMemcpyAsync(&flag, scratch + kNaFlag, sizeof(double), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (*err = cudaStreamSynchronize(s)) != cudaSuccess)
        return 2;
    *nonfinite = flag != 0.0;
    return 0;
}

}  // namespace bte
