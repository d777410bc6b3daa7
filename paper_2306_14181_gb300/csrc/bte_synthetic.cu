// Synthetic iterative scheme of the steady solver (Sec. 3.5 of arXiv 2306.14181).
//
// After the sweep of an iteration, the lattice temperature the next sweep relaxes towards is
// corrected by the macroscopic equation of Eq. (disretized_macro).  With the scheme's own face
// fluxes for q, its right-hand side div q_nonFourier - sum Q equals k_bulk L T_L(e) - r(e), r
// being the energy the steady equation's right-hand side R (with e0 of T_L(e)) leaves in a cell,
//     r_i = sum_k sum_d w_d R_{k,d,i},
// so the new lattice temperature is T_L(e) + dT with
//     k_bulk L dT = -r,
// L the cell-centred Laplacian of the grid: a thermalizing wall holds the temperature (the ghost
// is minus the wall cell), reflecting walls pass no heat (the ghost equals the wall cell),
// periodic pairs wrap.  With no thermalizing wall L is singular; r is then made mean-free and
// the solution is the mean-free one.
//
// Here: the energy residual from the forward step's output (two passes: a band's directions,
// then the bands), then on 1-D grids with a thermalizing wall the Thomas algorithm (one thread),
// else conjugate gradients in FP64 on the cells, each iteration short launches with the scalars
// on the device (no host synchronisation but a convergence check every 16 iterations); the dot
// products are block partials summed in a fixed order.
#include <cuda_runtime.h>

#include <cmath>

#include "bte_internal.h"

namespace bte {
namespace {

constexpr int kThreads = 256;

// Pr[k][i] = sum_d w_d (e_out - e_in)_{k,d,i}   (dt R summed over the band's directions)
__global__ void __launch_bounds__(kThreads) k_eres_band(const StepArgs a, const float *__restrict__ w,
                                                        const float *__restrict__ e_in,
                                                        const float *__restrict__ e_out, float *__restrict__ Pr) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.ncell) return;
    const int k = blockIdx.y;
    float acc = 0.f;
    for (int d = 0; d < a.nd; ++d) {
        const long long j = ((long long)k * a.nd + d) * a.ncell + i;
        acc = fmaf(w[d], e_out[j] - e_in[j], acc);
    }
    Pr[(long long)k * a.ncell + i] = acc;
}

// b_i = -r_i / k_bulk, the right-hand side of L dT = b, with r_i = sum_k Pr[k][i] / dt
__global__ void __launch_bounds__(kThreads) k_eres_rhs(const float *__restrict__ Pr, int nb, long long n, double inv_dt_k,
                                                       double *__restrict__ b) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double s = 0.0;
    for (int k = 0; k < nb; ++k) s += (double)Pr[(long long)k * n + i];
    b[i] = -s * inv_dt_k;
}

struct Grid {
    int dim, n[3];
    double ih2[3];  // 1 / h_a^2
    int bc[6];
};

// y = L x with the walls' ghost rules
__device__ __forceinline__ double lap_at(const Grid &g, const double *__restrict__ x, long long i) {
    const int c[3] = {(int)(i % g.n[0]), (int)((i / g.n[0]) % g.n[1]), (int)(i / ((long long)g.n[0] * g.n[1]))};
    const long long st[3] = {1, g.n[0], (long long)g.n[0] * g.n[1]};
    const double xi = x[i];
    double y = 0.0;
    for (int a = 0; a < g.dim; ++a) {
        double lo, hi;
        if (c[a] > 0) lo = x[i - st[a]];
        else if (g.bc[2 * a] == kBcPeriodic) lo = x[i + (long long)(g.n[a] - 1) * st[a]];
        else lo = g.bc[2 * a] == kBcIsothermal ? -xi : xi;
        if (c[a] < g.n[a] - 1) hi = x[i + st[a]];
        else if (g.bc[2 * a + 1] == kBcPeriodic) hi = x[i - (long long)(g.n[a] - 1) * st[a]];
        else hi = g.bc[2 * a + 1] == kBcIsothermal ? -xi : xi;
        y += (lo - 2.0 * xi + hi) * g.ih2[a];
    }
    return y;
}

// Block partial of sum u_i v_i (tree order within the block) into part[blockIdx.x]; grid of
// fixed size, each block strides over the cells.
__device__ __forceinline__ void block_sum(double v, double *part) {
    __shared__ double sm[kThreads];
    sm[threadIdx.x] = v;
    __syncthreads();
    for (int s = kThreads / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sm[threadIdx.x] += sm[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sm[0];
}

// CG scalars in device memory: [0] rr, [1] pAp, [2] alpha, [3] beta, [4] bb, [5] mean of b
enum { kRR = 0, kPAP = 1, kALPHA = 2, kBETA = 3, kBB = 4, kMEAN = 5 };

__global__ void __launch_bounds__(kThreads) k_partial_sum(const double *__restrict__ u, const double *__restrict__ v,
                                                          long long n, double *part) {
    double s = 0.0;
    for (long long i = (long long)blockIdx.x * kThreads + threadIdx.x; i < n; i += (long long)gridDim.x * kThreads)
        s += v ? u[i] * v[i] : u[i];
    block_sum(s, part);
}

// one block: out = sum of the partials in order; mode 0: scal[slot] = out; mode 1: the mean of b
// (scal[kMEAN] = out / n); mode 2: rr update (beta = out / rr, rr = out); mode 3: alpha = rr / out
__global__ void __launch_bounds__(kThreads) k_finish(const double *__restrict__ part, int np, double *scal, int slot,
                                                     int mode, long long n) {
    __shared__ double sm[kThreads];
    double s = 0.0;
    for (int j = threadIdx.x; j < np; j += kThreads) s += part[j];
    sm[threadIdx.x] = s;
    __syncthreads();
    for (int t = kThreads / 2; t > 0; t >>= 1) {
        if (threadIdx.x < t) sm[threadIdx.x] += sm[threadIdx.x + t];
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    const double out = sm[0];
    if (mode == 0) scal[slot] = out;
    else if (mode == 1) scal[kMEAN] = out / (double)n;
    else if (mode == 2) {
        scal[kBETA] = scal[kRR] > 0.0 ? out / scal[kRR] : 0.0;
        scal[kRR] = out;
    } else {
        scal[kPAP] = out;
        scal[kALPHA] = out != 0.0 ? scal[kRR] / out : 0.0;
    }
}

// b -= mean(b) (singular L); x = 0, r = p = b
__global__ void __launch_bounds__(kThreads) k_cg_init(double *__restrict__ b, const double *scal, int project, long long n,
                                                      double *__restrict__ x, double *__restrict__ r,
                                                      double *__restrict__ p) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double v = b[i];
    if (project) v -= scal[kMEAN];
    b[i] = v;
    x[i] = 0.0;
    r[i] = v;
    p[i] = v;
}

// Ap = L p (partials of p.Ap are taken by k_partial_sum afterwards)
__global__ void __launch_bounds__(kThreads) k_cg_matvec(const Grid g, const double *__restrict__ p, long long n,
                                                        double *__restrict__ Ap) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    Ap[i] = lap_at(g, p, i);
}

// x += alpha p, r -= alpha Ap
__global__ void __launch_bounds__(kThreads) k_cg_update(const double *scal, long long n, const double *__restrict__ p,
                                                        const double *__restrict__ Ap, double *__restrict__ x,
                                                        double *__restrict__ r) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double al = scal[kALPHA];
    x[i] = fma(al, p[i], x[i]);
    r[i] = fma(-al, Ap[i], r[i]);
}

// p = r + beta p
__global__ void __launch_bounds__(kThreads) k_cg_dir(const double *scal, long long n, const double *__restrict__ r,
                                                     double *__restrict__ p) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    p[i] = fma(scal[kBETA], p[i], r[i]);
}

// TL += dT, dT = x less its mean when L is singular (scal[kMEAN]; 0 otherwise)
__global__ void __launch_bounds__(kThreads) k_tl_correct(const double *__restrict__ x, const double *scal, int project,
                                                         long long n, float *__restrict__ TL) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    TL[i] = (float)((double)TL[i] + (project ? x[i] - scal[kMEAN] : x[i]));
}

// 1-D grids with a thermalizing wall and no periodic pair: L is tridiagonal and regular; one
// thread solves L x = b by the Thomas algorithm (forward elimination, back substitution), the
// elimination's ratios kept in cp.
__global__ void k_thomas_1d(const double *__restrict__ b, long long n, double ih2, int lo_iso, int hi_iso,
                            double *__restrict__ cp, double *__restrict__ x) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    auto diag = [&](long long i) {
        double d = -2.0 * ih2;
        if (i == 0) d += lo_iso ? -ih2 : ih2;
        if (i == n - 1) d += hi_iso ? -ih2 : ih2;
        return d;
    };
    double m = diag(0);
    cp[0] = ih2 / m;
    x[0] = b[0] / m;
    for (long long i = 1; i < n; ++i) {
        m = diag(i) - ih2 * cp[i - 1];
        cp[i] = ih2 / m;
        x[i] = (b[i] - ih2 * x[i - 1]) / m;
    }
    for (long long i = n - 2; i >= 0; --i) x[i] -= cp[i] * x[i + 1];
}

}  // namespace

size_t synthetic_scratch_doubles(long long ncell) { return (size_t)5 * ncell + kSynthParts + 8; }

cudaError_t synthetic_correct(const StepArgs &a, const double h[3], const float *w, const float *e_in,
                              const float *e_out, float *Pr, double *scratch, double k_bulk, double dt, int max_cg,
                              double rel_tol, float *TL, cudaStream_t s, int *cg_iters) {
    const long long n = a.ncell;
    double *b = scratch, *x = b + n, *r = x + n, *p = r + n, *Ap = p + n, *part = Ap + n, *scal = part + kSynthParts;
    const unsigned nblk = (unsigned)((n + kThreads - 1) / kThreads);
    const dim3 g2(nblk, (unsigned)a.nb);
    k_eres_band<<<g2, kThreads, 0, s>>>(a, w, e_in, e_out, Pr);
    // b = -r / k_bulk with r = sum_k Pr / dt: L dT = b
    k_eres_rhs<<<nblk, kThreads, 0, s>>>(Pr, a.nb, n, 1.0 / (dt * k_bulk), b);
    Grid g;
    g.dim = a.dim;
    bool singular = true;
    for (int q = 0; q < 3; ++q) g.n[q] = a.n[q];
    for (int q = 0; q < 6; ++q) g.bc[q] = a.bc[q];
    for (int q = 0; q < a.dim; ++q)
        if (a.bc[2 * q] == kBcIsothermal || a.bc[2 * q + 1] == kBcIsothermal) singular = false;
    for (int q = 0; q < 3; ++q) g.ih2[q] = 1.0 / (h[q] * h[q]);
    if (a.dim == 1 && !singular && a.bc[0] != kBcPeriodic) {
        k_thomas_1d<<<1, 1, 0, s>>>(b, n, g.ih2[0], a.bc[0] == kBcIsothermal, a.bc[1] == kBcIsothermal, r, x);
        k_tl_correct<<<nblk, kThreads, 0, s>>>(x, scal, 0, n, TL);
        if (cg_iters) *cg_iters = 0;
        return cudaGetLastError();
    }
    if (singular) {
        k_partial_sum<<<kSynthParts, kThreads, 0, s>>>(b, nullptr, n, part);
        k_finish<<<1, kThreads, 0, s>>>(part, kSynthParts, scal, kMEAN, 1, n);
    }
    k_cg_init<<<nblk, kThreads, 0, s>>>(b, scal, singular ? 1 : 0, n, x, r, p);
    k_partial_sum<<<kSynthParts, kThreads, 0, s>>>(r, r, n, part);
    k_finish<<<1, kThreads, 0, s>>>(part, kSynthParts, scal, kRR, 0, n);
    double bb = 0.0;
    cudaError_t e = cudaMemcpyAsync(&bb, scal + kRR, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    int it = 0;
    if (bb > 0.0) {
        const double stop = rel_tol * rel_tol * bb;
        constexpr int kCheck = 16;
        while (it < max_cg) {
            for (int j = 0; j < kCheck && it < max_cg; ++j, ++it) {
                k_cg_matvec<<<nblk, kThreads, 0, s>>>(g, p, n, Ap);
                k_partial_sum<<<kSynthParts, kThreads, 0, s>>>(p, Ap, n, part);
                k_finish<<<1, kThreads, 0, s>>>(part, kSynthParts, scal, kPAP, 3, n);
                k_cg_update<<<nblk, kThreads, 0, s>>>(scal, n, p, Ap, x, r);
                k_partial_sum<<<kSynthParts, kThreads, 0, s>>>(r, r, n, part);
                k_finish<<<1, kThreads, 0, s>>>(part, kSynthParts, scal, kRR, 2, n);
                k_cg_dir<<<nblk, kThreads, 0, s>>>(scal, n, r, p);
            }
            double rr = 0.0;
            e = cudaMemcpyAsync(&rr, scal + kRR, sizeof(double), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) return e;
            if (!(rr > stop)) break;
        }
        if (singular) {
            k_partial_sum<<<kSynthParts, kThreads, 0, s>>>(x, nullptr, n, part);
            k_finish<<<1, kThreads, 0, s>>>(part, kSynthParts, scal, kMEAN, 1, n);
        }
        k_tl_correct<<<nblk, kThreads, 0, s>>>(x, scal, singular ? 1 : 0, n, TL);
    }
    if (cg_iters) *cg_iters = it;
    return cudaGetLastError();
}

}  // namespace bte
