// Host side of the C ABI declared in include/bte.h: validation, the directional and band
// tables (arXiv 2306.14181, Sec. 3.1-3.2), device buffers, and the step schedule of
// Algorithm 2 (transient solver).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/bte.h"
#include "bte_internal.h"
#include "bte_tiled.h"
#include "bte_adjoint.h"

using namespace bte;

static thread_local std::string g_create_error;

namespace bte {
int tiled_finalize_launches(const TiledPlan &plan, const int bc[6]);  // kernels launch_finalize_tiled launches
}  // namespace bte

struct bte_ctx {
    // problem
    int dim = 0, n[3] = {1, 1, 1};
    double h[3] = {1, 1, 1};
    double Tref = 0;
    int nb = 0, nd = 0;
    std::vector<double> C, v, tau, s, w;
    std::vector<int> mirror;  // [3][nd], -1 = none
    int bc[6] = {0, 0, 0, 0, 0, 0};
    double Tw[6] = {0, 0, 0, 0, 0, 0};
    double jump[3] = {0, 0, 0};  // temperature difference across each periodic pair (Sec. 2.2 (iv))
    bool has_jump = false;
    double dt = 0, T_scale = 1;
    int storage = 0, limiter = 0, rounding = 0, kernel = 0;
    uint64_t seed = 0;
    cudaStream_t stream = nullptr;
    int device = 0;
    double W = 0, sumC = 0, D = 0;
    long long ncell = 0, nelem = 0;
    size_t elem_bytes = 4, state_bytes = 0;
    // device state
    void *e[2] = {nullptr, nullptr};
    int cur = 0;
    float *TL = nullptr, *Q = nullptr, *P = nullptr;
    float *R = nullptr;  // code reference of the current state (16-bit storage): T_L of the step that wrote it
    int G = 0;
    void *ediff[2] = {nullptr, nullptr};
    int ecur = 0;
    int wc_max = 1;
    float inv_den[6] = {0, 0, 0, 0, 0, 0};
    // device tables
    float *nu = nullptr, *wmom = nullptr, *wdiff = nullptr, *iso = nullptr, *jmp = nullptr;
    int *mirror_d = nullptr;
    BandConst *band = nullptr;
    double *d_w = nullptr, *d_s = nullptr, *d_v = nullptr, *d_invtau = nullptr;
    // diagnostics scratch (allocated on first use)
    double *dg = nullptr;
    int *dflag = nullptr;
    double *rs = nullptr;  // residuals: T^n, |q|^n [2 ncell], block partials [4 kResidBlocks], results [4]
    // tiled-kernel plan
    TiledPlan plan;
    bool tiled = false;
    // persistent single-CTA path (small 1-D FP32 problems): per-call source amplitudes
    bool persist = false;
    float *d_amp = nullptr;
    size_t d_amp_n = 0;
    // pinned host staging (allocated on first use): the source field on its way up, with the
    // event that marks its upload read; the lattice temperature on its way down
    float *h_src = nullptr, *h_tl = nullptr;
    cudaEvent_t ev_src = nullptr;
    // source
    bool has_source = false, has_amp = false;
    std::vector<double> amp;
    long long step = 0;
    size_t device_bytes = 0;
    std::string err;
    // adjoint: direction weights (FP32) and, with tracing on, the last bte_adjoint's timing
    float *wf = nullptr;
    double adj_ms = 0, adj_recompute_ms = 0;
    long long adj_steps = 0, adj_recompute_steps = 0;
    // CUDA graph of kGraphSteps forward steps for long bte_step calls (see step_graphs), its
    // private stream and ordering events, and the context state it was captured from
    cudaStream_t gstream = nullptr;
    cudaGraphExec_t gexec = nullptr;
    cudaEvent_t gev[2] = {nullptr, nullptr};
    int gkey_cur = -1, gkey_ecur = -1, gkey_src = -1;
    const float *gkey_tl = nullptr;
    unsigned long long gkey_wait = 0;
    // steady solver's iterative scheme (Sec. 3.5): 0 sequential, 1 synthetic; the synthetic
    // scheme's scratch (allocated on first use) and the conjugate-gradient count of its last
    // correction
    int scheme = 0;
    bool tl_corrected = false;  // TL holds a synthetic correction, not the T_L of the state
    float *syn_pr = nullptr;
    double *syn_x = nullptr;
    int syn_cg = 0;
    // interface between two materials (Sec. 2.2 (v)): the wall created as BTE_BC_INTERFACE (-1:
    // none; the kernels treat it as diffuse), the coupled context, this side's plain diffuse
    // values at that wall [nb][wall cells] once mixed, and (side A only) the transmissions
    int iwall = -1;
    bte_ctx *peer = nullptr;
    bool iface_a = false;
    bool iface_pure = true;  // e_diff at iwall holds plain diffuse values (not the mixed ones)
    float *ipure = nullptr;
    float *ibeta = nullptr;  // [4][nb]: beta_ab, 1 - beta_ab, beta_ba, 1 - beta_ba
    cudaEvent_t iev = nullptr;
    // tracing: event triples (before forward, after forward, after finalize) per step
    bool prof = false;
    std::vector<cudaEvent_t> ev;
    size_t ev_used = 0;
};

// ------------------------------------------------------------------------------------------
// helpers
// ------------------------------------------------------------------------------------------
static bte_status fail(bte_ctx *c, bte_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    else g_create_error = buf;
    return st;
}

#define CU(ctx, call)                                                                                  \
    do {                                                                                               \
        cudaError_t e_ = (call);                                                                       \
        if (e_ != cudaSuccess)                                                                         \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? BTE_ENOMEM : BTE_ECUDA, "%s: %s (%s:%d)", \
                        #call, cudaGetErrorString(e_), __FILE__, __LINE__);                            \
    } while (0)

template <class T>
static bte_status dalloc(bte_ctx *c, T **p, size_t count) {
    const size_t bytes = count * sizeof(T);
    cudaError_t e = cudaMalloc((void **)p, bytes ? bytes : sizeof(T));
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return fail(c, BTE_ENOMEM, "cudaMalloc of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
    }
    c->device_bytes += bytes;
    return BTE_OK;
}

template <class T>
static bte_status upload(bte_ctx *c, T *dst, const T *src, size_t count) {
    CU(c, cudaMemcpy(dst, src, count * sizeof(T), cudaMemcpyHostToDevice));
    return BTE_OK;
}

#define TRY(x)                       \
    do {                             \
        bte_status st_ = (x);        \
        if (st_ != BTE_OK) return st_; \
    } while (0)

// Gauss-Legendre rule on [lo, hi] by Newton iteration on the Legendre polynomial P_n,
// evaluated with the three-term recurrence (j+1) P_{j+1} = (2j+1) x P_j - j P_{j-1}; the
// weights are 2 / ((1 - x^2) P_n'(x)^2).  Roots are found in pairs +-x so the rule is
// exactly symmetric.
static void gauss_legendre(int n, double lo, double hi, std::vector<double> &x, std::vector<double> &wt) {
    x.assign(n, 0.0);
    wt.assign(n, 0.0);
    const double pi = 3.14159265358979323846;
    for (int i = 0; i < (n + 1) / 2; ++i) {
        double z = std::cos(pi * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int j = 1; j < n; ++j) {
                const double p2 = ((2.0 * j + 1.0) * z * p1 - j * p0) / (j + 1.0);
                p0 = p1;
                p1 = p2;
            }
            if (n == 1) { p0 = 1.0; p1 = z; }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            const double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) {
                // derivative at the converged root
                double q0 = 1.0, q1 = z;
                for (int j = 1; j < n; ++j) {
                    const double q2 = ((2.0 * j + 1.0) * z * q1 - j * q0) / (j + 1.0);
                    q0 = q1;
                    q1 = q2;
                }
                if (n == 1) { q0 = 1.0; q1 = z; }
                dp = n * (z * q1 - q0) / (z * z - 1.0);
                break;
            }
        }
        if (2 * i + 1 == n) z = 0.0;
        const double wi = 2.0 / ((1.0 - z * z) * dp * dp);
        x[i] = -z;
        x[n - 1 - i] = z;
        wt[i] = wi;
        wt[n - 1 - i] = wi;
    }
    const double half = 0.5 * (hi - lo);
    for (int i = 0; i < n; ++i) {
        x[i] = lo + half * (x[i] + 1.0);
        wt[i] *= half;
    }
}

static bte_status build_quadrature(const bte_quadrature *q, int dim, bte_ctx *c) {
    const double pi = 3.14159265358979323846;
    c->s.clear();
    c->w.clear();
    if (q->kind == BTE_QUAD_GL1D_POLAR) {
        if (q->ntheta < 2 || q->ntheta > 1024) return fail(nullptr, BTE_EINVAL, "GL1D_POLAR needs 2..1024 nodes");
        std::vector<double> mu, wm;
        gauss_legendre(q->ntheta, -1.0, 1.0, mu, wm);
        for (int i = 0; i < q->ntheta; ++i) {
            c->s.push_back(mu[i]);
            c->s.push_back(0.0);
            c->s.push_back(0.0);
            c->w.push_back(2.0 * pi * wm[i]);
        }
    } else if (q->kind == BTE_QUAD_OCTANT) {
        if (q->ntheta < 1 || q->nphi < 1 || q->ntheta > 64 || q->nphi > 64)
            return fail(nullptr, BTE_EINVAL, "OCTANT needs 1..64 polar and azimuthal nodes");
        std::vector<double> mu, wm, ph, wp;
        gauss_legendre(q->ntheta, 0.0, 1.0, mu, wm);
        gauss_legendre(q->nphi, 0.0, 0.5 * pi, ph, wp);
        for (int o = 0; o < 8; ++o)
            for (int j = 0; j < q->ntheta; ++j)
                for (int l = 0; l < q->nphi; ++l) {
                    const double st = std::sqrt(1.0 - mu[j] * mu[j]);
                    const double sx = (o & 1) ? -1.0 : 1.0, sy = (o & 2) ? -1.0 : 1.0, sz = (o & 4) ? -1.0 : 1.0;
                    c->s.push_back(sx * st * std::cos(ph[l]));
                    c->s.push_back(sy * st * std::sin(ph[l]));
                    c->s.push_back(sz * mu[j]);
                    c->w.push_back(wm[j] * wp[l]);
                }
    } else if (q->kind == BTE_QUAD_EXPLICIT) {
        if (q->ndirs < 1 || !q->s || !q->w) return fail(nullptr, BTE_EINVAL, "EXPLICIT quadrature needs s, w, ndirs");
        for (int d = 0; d < q->ndirs; ++d) {
            for (int a = 0; a < 3; ++a) {
                if (!std::isfinite(q->s[3 * d + a])) return fail(nullptr, BTE_EINVAL, "non-finite direction");
                c->s.push_back(q->s[3 * d + a]);
            }
            if (!(q->w[d] > 0.0) || !std::isfinite(q->w[d])) return fail(nullptr, BTE_EINVAL, "weights must be > 0");
            c->w.push_back(q->w[d]);
        }
    } else {
        return fail(nullptr, BTE_EINVAL, "unknown quadrature kind %d", q->kind);
    }
    c->nd = (int)c->w.size();
    (void)dim;
    // mirror partners: direction with component a negated (same weight)
    c->mirror.assign(3 * c->nd, -1);
    for (int a = 0; a < 3; ++a)
        for (int d = 0; d < c->nd; ++d)
            for (int m = 0; m < c->nd; ++m) {
                bool ok = std::fabs(c->w[m] - c->w[d]) <= 1e-12 * c->w[d];
                for (int b = 0; b < 3 && ok; ++b) {
                    const double t = (b == a) ? -c->s[3 * d + b] : c->s[3 * d + b];
                    ok = std::fabs(c->s[3 * m + b] - t) <= 1e-12;
                }
                if (ok) {
                    c->mirror[a * c->nd + d] = m;
                    break;
                }
            }
    return BTE_OK;
}

static StepArgs make_args(const bte_ctx *c) {
    StepArgs a;
    memset(&a, 0, sizeof a);
    a.dim = c->dim;
    for (int i = 0; i < 3; ++i) a.n[i] = c->n[i];
    a.stride[0] = 1;
    a.stride[1] = c->n[0];
    a.stride[2] = (long long)c->n[0] * c->n[1];
    a.ncell = c->ncell;
    a.nb = c->nb;
    a.nd = c->nd;
    for (int i = 0; i < 6; ++i) {
        a.bc[i] = c->bc[i];
        a.inv_den[i] = c->inv_den[i];
    }
    a.wc_max = c->wc_max;
    a.amp = 0.f;
    a.invD = (float)(1.0 / c->D);
    a.nu = c->nu;
    a.wmom = c->wmom;
    a.wdiff = c->wdiff;
    a.mirror = c->mirror_d;
    a.band = c->band;
    a.iso = c->iso;
    a.jmp = c->jmp;
    a.TL = c->TL;
    a.R = c->R;
    a.invTs = (float)(1.0 / c->T_scale);
    a.sr = 0;
    a.srkey = 0;
    a.Q = c->has_source ? c->Q : nullptr;
    a.P = c->P;
    return a;
}

static double amplitude_at(const bte_ctx *c, long long n) {
    if (!c->has_amp) return 1.0;
    return n < (long long)c->amp.size() ? c->amp[n] : 0.0;
}

// T_L and the diffuse-wall values of the current state (after a fill or an upload).
static bte_status iface_mix(bte_ctx *c);

static bte_status refresh_moments(bte_ctx *c) {
    StepArgs a = make_args(c);
    a.e_in = c->e[c->cur];
    a.ediff_out = c->ediff[c->ecur ^ 1];
    CU(c, launch_moment_only(a, c->storage, c->stream));
    c->ecur ^= 1;
    CU(c, launch_finalize(a, c->nb, c->TL, c->stream));
    c->tl_corrected = false;
    c->iface_pure = true;
    if (c->peer) TRY(iface_mix(c));
    return BTE_OK;
}

// Interface values of a coupled pair from both sides' current states (Sec. 2.2 (v)).  The mix
// runs on side B's stream after the work queued on side A's, and side A's stream waits for it.
static bte_status iface_mix(bte_ctx *c) {
    bte_ctx *A = c->iface_a ? c : c->peer, *B = c->iface_a ? c->peer : c;
    const int ax = A->iwall >> 1;
    const int ncw = (int)(A->ncell / A->n[ax]);
    CU(A, cudaEventRecord(A->iev, A->stream));
    CU(B, cudaStreamWaitEvent(B->stream, A->iev, 0));
    float *eA = static_cast<float *>(A->ediff[A->ecur]) + (size_t)A->iwall * A->nb * A->wc_max;
    float *eB = static_cast<float *>(B->ediff[B->ecur]) + (size_t)B->iwall * B->nb * B->wc_max;
    CU(B, launch_iface_mix(eA, A->ipure, A->iface_pure, A->wc_max, eB, B->ipure, B->iface_pure, B->wc_max, A->ibeta,
                           A->nb, ncw, B->stream));
    CU(B, cudaEventRecord(B->iev, B->stream));
    CU(A, cudaStreamWaitEvent(A->stream, B->iev, 0));
    A->iface_pure = B->iface_pure = false;
    return BTE_OK;
}

static void free_all(bte_ctx *c) {
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    c->gexec = nullptr;
    for (cudaEvent_t &e : c->gev)
        if (e) cudaEventDestroy(e), e = nullptr;
    if (c->gstream) cudaStreamDestroy(c->gstream);
    c->gstream = nullptr;
    cudaFree(c->syn_pr);
    cudaFree(c->syn_x);
    c->syn_pr = nullptr;
    c->syn_x = nullptr;
    if (c->iev) cudaEventDestroy(c->iev);
    c->iev = nullptr;
    cudaFree(c->ipure);
    cudaFree(c->ibeta);
    c->ipure = c->ibeta = nullptr;
    void *ptrs[] = {c->d_amp, c->wf, c->e[0], c->e[1], c->TL, c->R, c->Q, c->P, c->ediff[0], c->ediff[1], c->nu, c->wmom, c->wdiff,
                    c->iso, c->jmp, c->mirror_d, c->band, c->d_w, c->d_s, c->d_v, c->d_invtau, c->dg, c->dflag,
                    c->rs};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    tiled_free(c->plan);
    for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
    c->ev.clear();
    if (c->h_src) cudaFreeHost(c->h_src);
    if (c->h_tl) cudaFreeHost(c->h_tl);
    if (c->ev_src) cudaEventDestroy(c->ev_src);
    c->h_src = c->h_tl = nullptr;
    c->ev_src = nullptr;
}

static bte_status prof_event(bte_ctx *c, cudaEvent_t *out) {
    if (c->ev_used == c->ev.size()) {
        cudaEvent_t e;
        CU(c, cudaEventCreate(&e));
        c->ev.push_back(e);
    }
    *out = c->ev[c->ev_used++];
    CU(c, cudaEventRecord(*out, c->stream));
    return BTE_OK;
}

// ------------------------------------------------------------------------------------------
// ABI
// ------------------------------------------------------------------------------------------
extern "C" bte_status bte_create(const bte_grid *grid, const bte_bands *bands, const bte_quadrature *quad,
                                 const bte_boundaries *walls, const bte_options *opts, bte_ctx **out) {
    if (!out) return fail(nullptr, BTE_EINVAL, "out is NULL");
    *out = nullptr;
    if (!grid || !bands || !quad || !walls || !opts) return fail(nullptr, BTE_EINVAL, "NULL argument");
    bte_ctx tmp;
    bte_ctx *c = &tmp;
    // grid
    if (grid->dim < 1 || grid->dim > 3) return fail(nullptr, BTE_EINVAL, "dim must be 1, 2 or 3");
    c->dim = grid->dim;
    c->n[0] = grid->nx;
    c->n[1] = grid->ny;
    c->n[2] = grid->nz;
    c->h[0] = grid->dx;
    c->h[1] = grid->dy;
    c->h[2] = grid->dz;
    c->Tref = grid->Tref;
    for (int a = 0; a < 3; ++a) {
        if (a < c->dim) {
            if (c->n[a] < 2) return fail(nullptr, BTE_EINVAL, "active extent %d is %d; must be >= 2", a, c->n[a]);
            if (!(c->h[a] > 0.0) || !std::isfinite(c->h[a])) return fail(nullptr, BTE_EINVAL, "cell size must be > 0");
        } else if (c->n[a] != 1) {
            return fail(nullptr, BTE_EINVAL, "extent of inactive axis %d must be 1", a);
        }
    }
    c->ncell = (long long)c->n[0] * c->n[1] * c->n[2];
    // bands
    if (bands->nbands < 1 || !bands->C || !bands->vabs || !bands->tau)
        return fail(nullptr, BTE_EINVAL, "bands need nbands >= 1 and C, vabs, tau");
    c->nb = bands->nbands;
    for (int k = 0; k < c->nb; ++k) {
        const double Ck = bands->C[k], vk = bands->vabs[k], tk = bands->tau[k];
        if (!(Ck > 0) || !(vk > 0) || !(tk > 0) || !std::isfinite(Ck) || !std::isfinite(vk) || !std::isfinite(tk))
            return fail(nullptr, BTE_EINVAL, "band %d: C, |v| and tau must be finite and > 0", k);
        c->C.push_back(Ck);
        c->v.push_back(vk);
        c->tau.push_back(tk);
    }
    // quadrature
    TRY(build_quadrature(quad, c->dim, c));
    if ((long long)c->nb * c->nd > 65535) return fail(nullptr, BTE_EINVAL, "nbands * ndirs must be <= 65535");
    // walls
    for (int wl = 0; wl < 6; ++wl) {
        const int t = walls->type[wl];
        if (t < BTE_BC_ISOTHERMAL || t > BTE_BC_INTERFACE) return fail(nullptr, BTE_EINVAL, "wall %d: bad type %d", wl, t);
        if (!std::isfinite(walls->T_wall[wl])) return fail(nullptr, BTE_EINVAL, "wall %d: non-finite T_wall", wl);
        c->bc[wl] = t;
        if (t == BTE_BC_INTERFACE) {
            // the kernels see a diffuse wall; bte_interface supplies its incoming values
            if (c->iwall >= 0) return fail(nullptr, BTE_EINVAL, "at most one interface wall a context");
            if ((wl >> 1) >= c->dim) return fail(nullptr, BTE_EINVAL, "wall %d: interface on an inactive axis", wl);
            c->iwall = wl;
            c->bc[wl] = BTE_BC_DIFFUSE;
        }
        c->Tw[wl] = walls->T_wall[wl];
    }
    for (int a = 0; a < 3; ++a) {
        if (a >= c->dim) {
            c->bc[2 * a] = c->bc[2 * a + 1] = BTE_BC_PERIODIC;  // unused
            if (walls->dT_jump[a] != 0.0) return fail(nullptr, BTE_EINVAL, "inactive axis %d: dT_jump must be 0", a);
            continue;
        }
        if ((c->bc[2 * a] == BTE_BC_PERIODIC) != (c->bc[2 * a + 1] == BTE_BC_PERIODIC))
            return fail(nullptr, BTE_EINVAL, "axis %d: a periodic wall needs a periodic partner", a);
        const double jp = walls->dT_jump[a];
        if (!std::isfinite(jp)) return fail(nullptr, BTE_EINVAL, "axis %d: non-finite dT_jump", a);
        if (jp != 0.0 && c->bc[2 * a] != BTE_BC_PERIODIC)
            return fail(nullptr, BTE_EINVAL, "axis %d: dT_jump needs a periodic pair", a);
        c->jump[a] = jp;
        if (jp != 0.0) c->has_jump = true;
        for (int side = 0; side < 2; ++side)
            if (c->bc[2 * a + side] == BTE_BC_SPECULAR)
                for (int d = 0; d < c->nd; ++d)
                    if (c->mirror[a * c->nd + d] < 0)
                        return fail(nullptr, BTE_EINVAL, "specular wall on axis %d: direction %d has no mirror", a, d);
    }
    // options
    if (!(opts->dt > 0.0) || !std::isfinite(opts->dt)) return fail(nullptr, BTE_EINVAL, "dt must be > 0");
    if (opts->storage < BTE_STORE_F32 || opts->storage > BTE_STORE_BF16) return fail(nullptr, BTE_EINVAL, "bad storage");
    if (opts->limiter < BTE_LIM_FIRST_ORDER || opts->limiter > BTE_LIM_VANALBADA)
        return fail(nullptr, BTE_EINVAL, "bad limiter");
    if (opts->kernel < BTE_KERNEL_AUTO || opts->kernel > BTE_KERNEL_PERSISTENT) return fail(nullptr, BTE_EINVAL, "bad kernel");
    if (opts->rounding != BTE_ROUND_NEAREST && opts->rounding != BTE_ROUND_STOCHASTIC)
        return fail(nullptr, BTE_EINVAL, "bad rounding");
    if (c->iwall >= 0 && opts->storage != BTE_STORE_F32)
        return fail(nullptr, BTE_EUNSUPPORTED, "interface walls need FP32 storage");
    c->dt = opts->dt;
    c->storage = opts->storage;
    c->limiter = opts->limiter;
    c->rounding = opts->rounding;
    c->kernel = opts->kernel;
    c->seed = opts->seed;
    c->T_scale = opts->T_scale > 0 ? opts->T_scale : 1.0;
    c->stream = (cudaStream_t)opts->stream;
    c->elem_bytes = c->storage == BTE_STORE_F32 ? 4 : 2;
    c->nelem = c->ncell * c->nb * c->nd;
    c->state_bytes = (size_t)c->nelem * c->elem_bytes;
    // derived sums (sequential order)
    c->W = 0;
    for (double x : c->w) c->W += x;
    c->sumC = 0;
    c->D = 0;
    for (int k = 0; k < c->nb; ++k) {
        c->sumC += c->C[k];
        c->D += c->C[k] / c->tau[k];
    }

    // the context proper
    bte_ctx *ctx = new (std::nothrow) bte_ctx(*c);
    if (!ctx) return fail(nullptr, BTE_ENOMEM, "host allocation failed");
    c = ctx;
    auto bail = [&](bte_status st) {
        g_create_error = c->err;
        free_all(c);
        delete c;
        return st;
    };
    if (cudaGetDevice(&c->device) != cudaSuccess) {
        cudaGetLastError();
        c->err = "no CUDA device";
        return bail(BTE_ECUDA);
    }
    const int nplanes = c->nb * c->nd;
    // kernel plan
    c->G = c->nb;
    {
        // a 1-D FP32 state that fits in one CTA's shared memory runs persistent
        const size_t np = (size_t)c->nb * c->nd;
        const size_t ps = (2 * np * c->n[0] + c->n[0] + 2 * c->nb + 5 * np + 8 * (size_t)c->n[0]) * sizeof(float);
        int dev = 0, optin = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
            cudaGetLastError();
            optin = 0;
        }
        const bool fits = c->dim == 1 && c->storage == BTE_STORE_F32 && ps <= (size_t)optin && !c->has_jump &&
                          c->iwall < 0;
        if (c->kernel == BTE_KERNEL_PERSISTENT && !fits) {
            c->err = "persistent kernel unavailable: it needs a 1-D FP32 state that fits in shared memory, no "
                     "periodic temperature jump and no interface wall";
            return bail(BTE_EUNSUPPORTED);
        }
        c->persist = fits && (c->kernel == BTE_KERNEL_AUTO || c->kernel == BTE_KERNEL_PERSISTENT);
    }
    if (c->kernel != BTE_KERNEL_GENERIC && !c->persist) {
        std::string why;
        // the tiled kernel takes periodic ghosts as plain wrapped rows (no jump offset)
        c->tiled = !c->has_jump && tiled_plan(c->dim, c->n, c->nb, c->nd, c->storage, c->limiter,
                                              c->rounding == BTE_ROUND_STOCHASTIC, c->bc, c->plan, why);
        if (c->has_jump) why = "a periodic temperature jump runs the generic kernel";
        if (!c->tiled && c->kernel == BTE_KERNEL_TILED) {
            c->err = "tiled kernel unavailable: " + why;
            return bail(BTE_EUNSUPPORTED);
        }
    }
    // wall-cell slots (a multiple of 8 elements keeps every e_diff row 16-byte aligned)
    c->wc_max = 1;
    for (int a = 0; a < c->dim; ++a) {
        long long m = c->ncell / c->n[a];
        if (m > c->wc_max) c->wc_max = (int)m;
    }
    c->wc_max = (c->wc_max + 7) / 8 * 8;
    // diffuse normalisers
    for (int wl = 0; wl < 2 * c->dim; ++wl) {
        const int a = wl >> 1;
        const double ns = (wl & 1) ? 1.0 : -1.0;
        double den = 0;
        for (int d = 0; d < c->nd; ++d) {
            const double sn = ns * c->s[3 * d + a];
            if (sn < 0) den += c->w[d] * (-sn);
        }
        c->inv_den[wl] = den > 0 ? (float)(1.0 / den) : 0.f;
        if (c->bc[wl] == BTE_BC_DIFFUSE && !(den > 0)) {
            c->err = "diffuse wall without incoming directions";
            return bail(BTE_EINVAL);
        }
    }
    // host tables
    std::vector<float> nu(3 * nplanes, 0.f), wmom(nplanes), wdiff(6 * c->nd, 0.f), iso(6 * c->nb, 0.f),
        jmp(3 * c->nb, 0.f);
    std::vector<BandConst> band(c->nb);
    for (int k = 0; k < c->nb; ++k) {
        BandConst &b = band[k];
        b.dtinv = (float)(c->dt / c->tau[k]);
        b.ck = (float)(c->C[k] / c->W);
        b.srck = (float)(c->dt * c->C[k] / (c->sumC * c->W));
        const double sc = c->storage == BTE_STORE_F32 ? 1.0 : c->C[k] * c->T_scale / c->W;
        b.scale = (float)sc;
        b.inv_scale = (float)(1.0 / (double)b.scale);
        b.wtau = (float)(1.0 / c->tau[k]);
        b.pad0 = b.pad1 = 0.f;
        for (int d = 0; d < c->nd; ++d) {
            const int p = k * c->nd + d;
            for (int a = 0; a < c->dim; ++a) nu[3 * p + a] = (float)(c->dt * c->v[k] * c->s[3 * d + a] / c->h[a]);
            wmom[p] = (float)(c->w[d] / c->tau[k]);
        }
        for (int wl = 0; wl < 2 * c->dim; ++wl)
            if (c->bc[wl] == BTE_BC_ISOTHERMAL) iso[wl * c->nb + k] = (float)(c->C[k] * c->Tw[wl] / c->W);
        for (int a = 0; a < 3; ++a) jmp[a * c->nb + k] = (float)(c->C[k] * c->jump[a] / c->W);
    }
    for (int wl = 0; wl < 2 * c->dim; ++wl) {
        const int a = wl >> 1;
        const double ns = (wl & 1) ? 1.0 : -1.0;
        for (int d = 0; d < c->nd; ++d) {
            const double sn = ns * c->s[3 * d + a];
            if (sn > 0) wdiff[wl * c->nd + d] = (float)(c->w[d] * sn);
        }
    }
    std::vector<double> invtau(c->nb);
    for (int k = 0; k < c->nb; ++k) invtau[k] = 1.0 / c->tau[k];
    std::vector<int> mir(c->mirror);
    for (auto &m : mir)
        if (m < 0) m = 0;  // never read: specular walls require a partner

    bte_status st;
    if ((st = dalloc(c, (char **)&c->e[0], c->state_bytes)) != BTE_OK) return bail(st);
    if ((st = dalloc(c, (char **)&c->e[1], c->state_bytes)) != BTE_OK) return bail(st);
    if ((st = dalloc(c, &c->TL, c->ncell)) != BTE_OK) return bail(st);
    if ((st = dalloc(c, &c->R, c->ncell)) != BTE_OK) return bail(st);
    if ((st = dalloc(c, &c->Q, c->ncell)) != BTE_OK) return bail(st);
    {
        // moment partials: band-major rows for the generic passes, segment rows for the tiled one
        size_t np = (size_t)c->nb * c->ncell;
        if (c->tiled) np = std::max(np, (size_t)c->plan.G * c->plan.tcells);
        if ((st = dalloc(c, &c->P, np)) != BTE_OK) return bail(st);
    }
    for (int i = 0; i < 2; ++i)
        // + 16 elements: the tiled kernel copies 16-byte aligned spans that may reach past the last slot
        if ((st = dalloc(c, (char **)&c->ediff[i], ((size_t)6 * c->nb * c->wc_max + 16) * c->elem_bytes)) != BTE_OK)
            return bail(st);
    if ((st = dalloc(c, &c->nu, nu.size())) != BTE_OK) return bail(st);
    if ((st = dalloc(c, &c->wmom, wmom.size())) != BTE_OK) return bail(st);
    if ((st = dalloc(c, &c->wdiff, wdiff.size())) != BTE_OK) return bail(st);
    if ((st = dalloc(c, &c->iso, iso.size())) != BTE_OK) return bail(st);
    if ((st = dalloc(c, &c->jmp, jmp.size())) != BTE_OK) return bail(st);
    if ((st = dalloc(c, &c->mirror_d, mir.size())) != BTE_OK) return bail(st);
    if ((st = dalloc(c, &c->band, band.size())) != BTE_OK) return bail(st);
    if ((st = dalloc(c, &c->d_w, c->w.size())) != BTE_OK) return bail(st);
    if ((st = dalloc(c, &c->wf, c->w.size())) != BTE_OK) return bail(st);
    if ((st = dalloc(c, &c->d_s, c->s.size())) != BTE_OK) return bail(st);
    if ((st = dalloc(c, &c->d_v, c->v.size())) != BTE_OK) return bail(st);
    if ((st = dalloc(c, &c->d_invtau, invtau.size())) != BTE_OK) return bail(st);
    if ((st = upload(c, c->nu, nu.data(), nu.size())) != BTE_OK) return bail(st);
    if ((st = upload(c, c->wmom, wmom.data(), wmom.size())) != BTE_OK) return bail(st);
    if ((st = upload(c, c->wdiff, wdiff.data(), wdiff.size())) != BTE_OK) return bail(st);
    if ((st = upload(c, c->iso, iso.data(), iso.size())) != BTE_OK) return bail(st);
    if ((st = upload(c, c->jmp, jmp.data(), jmp.size())) != BTE_OK) return bail(st);
    if ((st = upload(c, c->mirror_d, mir.data(), mir.size())) != BTE_OK) return bail(st);
    if ((st = upload(c, c->band, band.data(), band.size())) != BTE_OK) return bail(st);
    if ((st = upload(c, c->d_w, c->w.data(), c->w.size())) != BTE_OK) return bail(st);
    {
        std::vector<float> wf(c->w.begin(), c->w.end());
        if ((st = upload(c, c->wf, wf.data(), wf.size())) != BTE_OK) return bail(st);
    }
    if ((st = upload(c, c->d_s, c->s.data(), c->s.size())) != BTE_OK) return bail(st);
    if ((st = upload(c, c->d_v, c->v.data(), c->v.size())) != BTE_OK) return bail(st);
    if ((st = upload(c, c->d_invtau, invtau.data(), invtau.size())) != BTE_OK) return bail(st);
    if (cudaMemset(c->ediff[0], 0, c->elem_bytes * (6 * c->nb * c->wc_max + 16)) != cudaSuccess ||
        cudaMemset(c->ediff[1], 0, c->elem_bytes * (6 * c->nb * c->wc_max + 16)) != cudaSuccess) {
        c->err = "cudaMemset failed";
        return bail(BTE_ECUDA);
    }
    if (c->tiled) {
        std::string why;
        if (!tiled_setup(c->plan, make_args(c), why)) {
            c->err = "tiled kernel setup failed: " + why;
            return bail(BTE_ECUDA);
        }
    }
    if ((st = bte_init_temperature(c, nullptr)) != BTE_OK) return bail(st);
    if ((st = bte_synchronize(c)) != BTE_OK) return bail(st);
    *out = c;
    return BTE_OK;
}

extern "C" void bte_destroy(bte_ctx *ctx) {
    if (!ctx) return;
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    else cudaDeviceSynchronize();
    if (bte_ctx *p = ctx->peer) {
        // the partner keeps a plain diffuse wall: its diffuse values of the current state again
        if (p->stream) cudaStreamSynchronize(p->stream);
        p->peer = nullptr;
        ctx->peer = nullptr;
        refresh_moments(p);
    }
    free_all(ctx);
    delete ctx;
}

extern "C" const char *bte_last_error(const bte_ctx *ctx) {
    return ctx ? ctx->err.c_str() : g_create_error.c_str();
}

extern "C" bte_status bte_init_temperature(bte_ctx *c, const double *dT0) {
    if (!c) return fail(nullptr, BTE_EINVAL, "ctx is NULL");
    double *d = nullptr;
    if (dT0) {
        for (long long i = 0; i < c->ncell; ++i)
            if (!std::isfinite(dT0[i])) return fail(c, BTE_EINVAL, "dT0 holds a non-finite value at cell %lld", i);
        TRY(dalloc(c, &d, c->ncell));
        c->device_bytes -= c->ncell * sizeof(double);
        cudaError_t e = cudaMemcpyAsync(d, dT0, c->ncell * sizeof(double), cudaMemcpyHostToDevice, c->stream);
        if (e != cudaSuccess) {
            cudaFree(d);
            return fail(c, BTE_ECUDA, "upload of dT0: %s", cudaGetErrorString(e));
        }
    }
    StepArgs a = make_args(c);
    a.e_out = c->e[c->cur];
    cudaError_t e = launch_fill(a, c->storage, d, c->R, c->stream);
    if (d) {
        cudaStreamSynchronize(c->stream);
        cudaFree(d);
    }
    if (e != cudaSuccess) return fail(c, BTE_ECUDA, "equilibrium fill: %s", cudaGetErrorString(e));
    TRY(refresh_moments(c));
    c->step = 0;
    return BTE_OK;
}

extern "C" bte_status bte_set_source(bte_ctx *c, const float *Q, int on_device, const double *amp, int n_amp) {
    if (!c) return fail(nullptr, BTE_EINVAL, "ctx is NULL");
    if (n_amp < 0 || (n_amp > 0 && !amp)) return fail(c, BTE_EINVAL, "bad amplitude array");
    if (amp)
        for (int i = 0; i < n_amp; ++i)
            if (!std::isfinite(amp[i])) return fail(c, BTE_EINVAL, "amplitude %d is not finite", i);
    if (!Q) {
        c->has_source = false;
        c->has_amp = false;
        c->amp.clear();
        return BTE_OK;
    }
    if (on_device) {
        CU(c, cudaMemcpyAsync(c->Q, Q, c->ncell * sizeof(float), cudaMemcpyDeviceToDevice, c->stream));
    } else {
        // checked and copied in one pass into pinned staging (once the previous upload has read
        // it), then uploaded in stream order: the caller may free Q on return, and nothing
        // waits for the steps already queued
        if (!c->h_src) CU(c, cudaMallocHost((void **)&c->h_src, c->ncell * sizeof(float)));
        if (!c->ev_src) CU(c, cudaEventCreateWithFlags(&c->ev_src, cudaEventDisableTiming));
        else CU(c, cudaEventSynchronize(c->ev_src));  // the previous upload has read the staging
        // the exponent field all ones marks an infinity or a NaN; an integer test and no early
        // exit keep the loop vectorised
        uint32_t nonfinite = 0;
        const uint32_t *qb = reinterpret_cast<const uint32_t *>(Q);
        uint32_t *hb = reinterpret_cast<uint32_t *>(c->h_src);
        for (long long i = 0; i < c->ncell; ++i) {
            const uint32_t v = qb[i];
            nonfinite |= (uint32_t)((v & 0x7f800000u) == 0x7f800000u);
            hb[i] = v;
        }
        if (nonfinite) {
            for (long long i = 0; i < c->ncell; ++i)
                if (!std::isfinite(Q[i])) return fail(c, BTE_EINVAL, "Q holds a non-finite value at cell %lld", i);
        }
        CU(c, cudaMemcpyAsync(c->Q, c->h_src, c->ncell * sizeof(float), cudaMemcpyHostToDevice, c->stream));
        CU(c, cudaEventRecord(c->ev_src, c->stream));
    }
    c->has_source = true;
    c->has_amp = amp != nullptr;
    c->amp.assign(amp ? amp : (const double *)nullptr, amp ? amp + n_amp : (const double *)nullptr);
    return BTE_OK;
}

// All nsteps steps in one persistent single-CTA launch (1-D FP32 states in shared memory).
static bte_status step_persistent(bte_ctx *c, int nsteps) {
    if ((size_t)nsteps > c->d_amp_n) {
        if (c->d_amp) cudaFree(c->d_amp);
        c->d_amp = nullptr;
        c->d_amp_n = 0;
        CU(c, cudaMalloc((void **)&c->d_amp, (size_t)nsteps * sizeof(float)));
        c->d_amp_n = nsteps;
    }
    std::vector<float> amps(nsteps);
    for (int s = 0; s < nsteps; ++s) amps[s] = (float)amplitude_at(c, c->step + s);
    CU(c, cudaMemcpyAsync(c->d_amp, amps.data(), nsteps * sizeof(float), cudaMemcpyHostToDevice, c->stream));
    StepArgs a = make_args(c);
    cudaEvent_t ev;
    if (c->prof) TRY(prof_event(c, &ev));
    CU(c, launch_persist_1d(a, c->limiter, nsteps, c->d_amp, static_cast<float *>(c->e[c->cur]), c->TL,
                            static_cast<float *>(c->ediff[c->ecur]), c->stream));
    if (c->prof) {
        TRY(prof_event(c, &ev));
        TRY(prof_event(c, &ev));
    }
    // (a copy from pageable memory has left `amps` when cudaMemcpyAsync returns)
    c->step += nsteps;
    return BTE_OK;
}

static bte_status step_one(bte_ctx *c, cudaStream_t s);

// A long bte_step call replays a CUDA graph of kGraphSteps steps (an even number, so that the
// two state buffers, the two wall-value buffers and the T_L / code-reference pair are back where
// they were) instead of launching every kernel of every step.  That is exact when the steps differ
// only in those buffers: a constant source amplitude, no stochastic rounding (its key depends on
// the step index), no kernel tracing and no pending failure-detection test.  The graph runs on a
// private stream ordered after and before the context's stream by events; it is captured again
// when the buffers' parity, the source's presence or the wait limit differ from its capture.
constexpr int kGraphSteps = 32;

static bool graph_eligible(const bte_ctx *c) {
    const bool sr = c->rounding == BTE_ROUND_STOCHASTIC && c->storage != BTE_STORE_F32;
    return !c->persist && !c->has_amp && !sr && !c->prof && !(c->tiled && c->plan.stall);
}

static bte_status step_graphs(bte_ctx *c, int chunks) {
    const unsigned long long wait = c->tiled ? c->plan.wait_ns : 0ull;
    const int src = c->has_source ? 1 : 0;
    if (!c->gexec || c->gkey_cur != c->cur || c->gkey_ecur != c->ecur || c->gkey_tl != c->TL || c->gkey_src != src ||
        c->gkey_wait != wait) {
        if (c->gexec) cudaGraphExecDestroy(c->gexec);
        c->gexec = nullptr;
        if (!c->gstream) CU(c, cudaStreamCreateWithFlags(&c->gstream, cudaStreamNonBlocking));
        for (cudaEvent_t &e : c->gev)
            if (!e) CU(c, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        const int cur = c->cur, ecur = c->ecur;
        float *TL = c->TL, *R = c->R;
        const long long step = c->step;
        CU(c, cudaStreamBeginCapture(c->gstream, cudaStreamCaptureModeThreadLocal));
        bte_status st = BTE_OK;
        for (int i = 0; i < kGraphSteps && st == BTE_OK; ++i) st = step_one(c, c->gstream);
        cudaGraph_t graph = nullptr;
        const cudaError_t ec = cudaStreamEndCapture(c->gstream, &graph);
        c->cur = cur;
        c->ecur = ecur;
        c->TL = TL;
        c->R = R;
        c->step = step;
        if (st != BTE_OK) {
            if (graph) cudaGraphDestroy(graph);
            return st;
        }
        if (ec != cudaSuccess) return fail(c, BTE_ECUDA, "step graph capture: %s", cudaGetErrorString(ec));
        const cudaError_t ei = cudaGraphInstantiate(&c->gexec, graph, 0);
        cudaGraphDestroy(graph);
        if (ei != cudaSuccess) {
            c->gexec = nullptr;
            return fail(c, BTE_ECUDA, "step graph instantiation: %s", cudaGetErrorString(ei));
        }
        c->gkey_cur = cur;
        c->gkey_ecur = ecur;
        c->gkey_tl = TL;
        c->gkey_src = src;
        c->gkey_wait = wait;
    }
    CU(c, cudaEventRecord(c->gev[0], c->stream));
    CU(c, cudaStreamWaitEvent(c->gstream, c->gev[0], 0));
    for (int i = 0; i < chunks; ++i) {
        CU(c, cudaGraphLaunch(c->gexec, c->gstream));
        c->step += kGraphSteps;
    }
    CU(c, cudaEventRecord(c->gev[1], c->gstream));
    CU(c, cudaStreamWaitEvent(c->stream, c->gev[1], 0));
    return BTE_OK;
}

extern "C" bte_status bte_step(bte_ctx *c, int nsteps) {
    if (!c) return fail(nullptr, BTE_EINVAL, "ctx is NULL");
    if (nsteps < 0) return fail(c, BTE_EINVAL, "n must be >= 0");
    if (c->peer) return fail(c, BTE_ESTATE, "the context is coupled at an interface: it steps through bte_step_pair");
    // after synthetic iterations the step starts from the state's own T_L (Eq. BTE_get_e0)
    if (c->tl_corrected && nsteps > 0) TRY(refresh_moments(c));
    if (c->persist) return nsteps > 0 ? step_persistent(c, nsteps) : BTE_OK;
    int s = 0;
    if (nsteps >= 2 * kGraphSteps && graph_eligible(c)) {
        const int chunks = nsteps / kGraphSteps;
        TRY(step_graphs(c, chunks));
        s = chunks * kGraphSteps;
    }
    for (; s < nsteps; ++s) TRY(step_one(c, c->stream));
    return BTE_OK;
}

extern "C" bte_status bte_step_pair(bte_ctx *a, bte_ctx *b, int nsteps) {
    if (!a || !b) return fail(a ? a : b, BTE_EINVAL, "ctx is NULL");
    if (nsteps < 0) return fail(a, BTE_EINVAL, "n must be >= 0");
    if (a->peer != b || b->peer != a) return fail(a, BTE_ESTATE, "the two contexts are not coupled with each other");
    for (int s = 0; s < nsteps; ++s) {
        TRY(step_one(a, a->stream));
        TRY(step_one(b, b->stream));
        a->iface_pure = b->iface_pure = true;
        TRY(iface_mix(a));
    }
    return BTE_OK;
}

extern "C" bte_status bte_interface(bte_ctx *a, int wa, bte_ctx *b, int wb, const double *bab, const double *bba) {
    if (!a || !b) return fail(a ? a : b, BTE_EINVAL, "ctx is NULL");
    if (a == b) return fail(a, BTE_EINVAL, "an interface couples two contexts");
    if (!bab || !bba) return fail(a, BTE_EINVAL, "beta arrays are NULL");
    if (a->peer || b->peer) return fail(a, BTE_EINVAL, "a context is already coupled");
    if (wa < 0 || wa > 5 || wb < 0 || wb > 5 || a->iwall != wa || b->iwall != wb)
        return fail(a, BTE_EINVAL, "walls %d and %d are not the contexts' interface walls", wa, wb);
    if (a->dim != b->dim || a->nb != b->nb) return fail(a, BTE_EINVAL, "dimension or band count differ");
    const int ax = wa >> 1;
    if ((wb >> 1) != ax || (wa & 1) == (wb & 1))
        return fail(a, BTE_EINVAL, "the walls must lie on the same axis and on opposite sides");
    for (int x = 0; x < 3; ++x)
        if (x != ax && a->n[x] != b->n[x]) return fail(a, BTE_EINVAL, "cell counts across the interface differ (axis %d)", x);
    std::vector<float> beta(4 * (size_t)a->nb);
    for (int k = 0; k < a->nb; ++k) {
        if (!(bab[k] >= 0.0 && bab[k] <= 1.0) || !(bba[k] >= 0.0 && bba[k] <= 1.0))
            return fail(a, BTE_EINVAL, "band %d: transmissions must lie in [0, 1]", k);
        beta[k] = (float)bab[k];
        beta[a->nb + k] = (float)(1.0 - bab[k]);
        beta[2 * a->nb + k] = (float)bba[k];
        beta[3 * a->nb + k] = (float)(1.0 - bba[k]);
    }
    const size_t ncw = (size_t)(a->ncell / a->n[ax]);
    for (bte_ctx *c : {a, b}) {
        if (!c->ipure) TRY(dalloc(c, &c->ipure, (size_t)c->nb * ncw));
        if (!c->iev) CU(c, cudaEventCreateWithFlags(&c->iev, cudaEventDisableTiming));
    }
    if (!a->ibeta) TRY(dalloc(a, &a->ibeta, beta.size()));
    TRY(upload(a, a->ibeta, beta.data(), beta.size()));
    CU(a, cudaStreamSynchronize(a->stream));
    a->peer = b;
    b->peer = a;
    a->iface_a = true;
    b->iface_a = false;
    return iface_mix(a);
}

static bte_status step_one(bte_ctx *c, cudaStream_t strm) {
    {
        StepArgs a = make_args(c);
        a.amp = (float)amplitude_at(c, c->step);
        if (c->rounding == BTE_ROUND_STOCHASTIC && c->storage != BTE_STORE_F32) {
            // the step's rounding key: the seed's two halves and the step index, hashed
            a.sr = 1;
            a.srkey = mix32((uint32_t)c->seed ^ mix32((uint32_t)(c->seed >> 32) ^ mix32((uint32_t)c->step)));
        }
        a.e_in = c->e[c->cur];
        a.e_out = c->e[c->cur ^ 1];
        a.ediff_in = c->ediff[c->ecur];
        a.ediff_out = c->ediff[c->ecur ^ 1];
        cudaError_t e;
        cudaEvent_t ev;
        if (c->prof) TRY(prof_event(c, &ev));
        if (c->tiled) {
            e = launch_step_tiled(a, c->plan, strm);
            c->plan.stall = 0;
        } else {
            e = launch_step_generic(a, c->storage, c->limiter, strm);
        }
        if (e != cudaSuccess) return fail(c, BTE_ECUDA, "forward step launch: %s", cudaGetErrorString(e));
        if (c->prof) TRY(prof_event(c, &ev));
        // T_L^{n+1} goes to the buffer of the old code reference; T_L^n becomes the reference of
        // the new state
        float *TL_next = c->R;
        if (c->tiled) e = launch_finalize_tiled(a, c->plan, c->storage, TL_next, strm);
        else e = launch_finalize(a, c->G, TL_next, strm);
        if (e != cudaSuccess) return fail(c, BTE_ECUDA, "finalize launch: %s", cudaGetErrorString(e));
        if (c->prof) TRY(prof_event(c, &ev));
        c->R = c->TL;
        c->TL = TL_next;
        c->cur ^= 1;
        c->ecur ^= 1;
        ++c->step;
    }
    return BTE_OK;
}

// Bounded device waits of the tiled kernel report through a flag; a set flag means a step
// gave up (its output is invalid) and is returned as BTE_ETIMEOUT once.
static bte_status check_device_flags(bte_ctx *c) {
    if (!c->tiled || !c->plan.err) return BTE_OK;
    int flag = 0;
    CU(c, cudaMemcpyAsync(&flag, c->plan.err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CU(c, cudaStreamSynchronize(c->stream));
    if (flag) {
        CU(c, cudaMemsetAsync(c->plan.err, 0, sizeof(int), c->stream));
        return fail(c, BTE_ETIMEOUT, "a bounded wait in the tiled forward kernel gave up (flag %d)", flag);
    }
    return BTE_OK;
}

extern "C" bte_status bte_synchronize(bte_ctx *c) {
    if (!c) return fail(nullptr, BTE_EINVAL, "ctx is NULL");
    CU(c, cudaStreamSynchronize(c->stream));
    CU(c, cudaGetLastError());
    return check_device_flags(c);
}

extern "C" bte_status bte_set_wait_limit(bte_ctx *c, long long limit_ns, int stall_test) {
    if (!c) return fail(nullptr, BTE_EINVAL, "ctx is NULL");
    if (stall_test < 0 || stall_test > 3) return fail(c, BTE_EINVAL, "stall_test must be 0..3");
    c->plan.wait_ns = limit_ns > 0 ? (unsigned long long)limit_ns : 2000000000ull;
    c->plan.stall = stall_test;
    return BTE_OK;
}

extern "C" bte_status bte_lattice_temperature(bte_ctx *c, double *dTL) {
    if (!c || !dTL) return fail(c, BTE_EINVAL, "NULL argument");
    if (!c->h_tl) CU(c, cudaMallocHost((void **)&c->h_tl, c->ncell * sizeof(float)));  // pinned: a direct copy
    CU(c, cudaMemcpyAsync(c->h_tl, c->TL, c->ncell * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
    CU(c, cudaStreamSynchronize(c->stream));
    const float *t = c->h_tl;
    for (long long i = 0; i < c->ncell; ++i) dTL[i] = t[i];
    return BTE_OK;
}

static bte_status diag_buffers(bte_ctx *c) {
    if (!c->dg) {
        // T, TL, cellE: ncell each; q: 3 ncell; wall partials: 6 nb wc_max; sums: 1024 + 8
        const size_t n = (size_t)6 * c->ncell + (size_t)6 * c->nb * c->wc_max + 1032;
        TRY(dalloc(c, &c->dg, n));
        TRY(dalloc(c, &c->dflag, 1));
    }
    return BTE_OK;
}

static DiagOut diag_layout(bte_ctx *c) {
    DiagOut o;
    o.T = c->dg;
    o.TL = c->dg + c->ncell;
    o.cellE = c->dg + 2 * c->ncell;
    o.q = c->dg + 3 * c->ncell;
    o.wallpart = c->dg + 6 * c->ncell;
    o.nonfinite = c->dflag;
    return o;
}

extern "C" bte_status bte_moments(bte_ctx *c, double *dT, double *dTL, double *q) {
    if (!c) return fail(nullptr, BTE_EINVAL, "ctx is NULL");
    TRY(diag_buffers(c));
    DiagOut o = diag_layout(c);
    CU(c, cudaMemsetAsync(c->dflag, 0, sizeof(int), c->stream));
    StepArgs a = make_args(c);
    a.e_in = c->e[c->cur];
    CU(c, launch_moments64(a, c->storage, c->d_w, c->d_s, c->d_v, c->d_invtau, c->sumC, c->D, o, c->stream));
    int flag = 0;
    CU(c, cudaMemcpyAsync(&flag, c->dflag, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    if (dT) CU(c, cudaMemcpyAsync(dT, o.T, c->ncell * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    if (dTL) CU(c, cudaMemcpyAsync(dTL, o.TL, c->ncell * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    if (q) CU(c, cudaMemcpyAsync(q, o.q, 3 * c->ncell * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CU(c, cudaStreamSynchronize(c->stream));
    if (flag) return fail(c, BTE_ENONFINITE, "the state holds a non-finite value");
    return BTE_OK;
}

extern "C" bte_status bte_energy(bte_ctx *c, double *E_total, double wall_flux[6]) {
    if (!c) return fail(nullptr, BTE_EINVAL, "ctx is NULL");
    TRY(diag_buffers(c));
    DiagOut o = diag_layout(c);
    double *sums = c->dg + 6 * c->ncell + (size_t)6 * c->nb * c->wc_max;  // [1024 scratch][8 results]
    CU(c, cudaMemsetAsync(c->dflag, 0, sizeof(int), c->stream));
    CU(c, cudaMemsetAsync(o.wallpart, 0, sizeof(double) * 6 * c->nb * c->wc_max, c->stream));
    StepArgs a = make_args(c);
    a.e_in = c->e[c->cur];
    a.ediff_in = c->ediff[c->ecur];
    DiagOut o2 = o;
    o2.T = o2.TL = o2.q = nullptr;
    CU(c, launch_moments64(a, c->storage, c->d_w, c->d_s, c->d_v, c->d_invtau, c->sumC, c->D, o2, c->stream));
    CU(c, launch_sum64(o.cellE, c->ncell, sums, sums + 1024, c->stream));
    CU(c, launch_wallflux64(a, c->storage, c->limiter, c->d_w, c->d_s, c->d_v, o, c->stream));
    for (int wl = 0; wl < 6; ++wl)
        CU(c, launch_sum64(o.wallpart + (size_t)wl * c->nb * c->wc_max, (long long)c->nb * c->wc_max, sums,
                           sums + 1025 + wl, c->stream));
    double res[7];
    int flag = 0;
    CU(c, cudaMemcpyAsync(res, sums + 1024, 7 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CU(c, cudaMemcpyAsync(&flag, c->dflag, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CU(c, cudaStreamSynchronize(c->stream));
    double L[3];
    for (int ax = 0; ax < 3; ++ax) L[ax] = ax < c->dim ? c->h[ax] : 1.0;
    const double V = L[0] * L[1] * L[2];
    if (E_total) *E_total = V * res[0];
    if (wall_flux)
        for (int wl = 0; wl < 6; ++wl) wall_flux[wl] = (wl < 2 * c->dim) ? (V / L[wl >> 1]) * res[1 + wl] : 0.0;
    if (flag) return fail(c, BTE_ENONFINITE, "the state holds a non-finite value");
    return BTE_OK;
}

// T and q of the current state (Eq. getTQ, FP64) into the diagnostic buffers; the non-finite
// flag is cleared first and read by the caller.
static bte_status moments_on_device(bte_ctx *c, const DiagOut &o) {
    StepArgs a = make_args(c);
    a.e_in = c->e[c->cur];
    DiagOut o2 = o;
    o2.TL = nullptr;
    o2.cellE = nullptr;
    CU(c, launch_moments64(a, c->storage, c->d_w, c->d_s, c->d_v, c->d_invtau, c->sumC, c->D, o2, c->stream));
    return BTE_OK;
}

// One sequential iteration of the steady implicit DOM (Sec. 3.3-3.5): the forward step writes
// e^n + dt R, the sweep turns it into e^n + De, and T_L and the diffuse-wall values follow from
// the new state.
static bte_status sis_one(bte_ctx *c) {
    // a sequential iteration after synthetic ones relaxes towards the state's own T_L again
    if (c->tl_corrected && c->scheme != BTE_SCHEME_SYNTHETIC) TRY(refresh_moments(c));
    StepArgs a = make_args(c);
    a.amp = (float)amplitude_at(c, c->step);
    a.e_in = c->e[c->cur];
    a.e_out = c->e[c->cur ^ 1];
    a.ediff_in = c->ediff[c->ecur];
    a.ediff_out = c->ediff[c->ecur ^ 1];
    cudaError_t e;
    if (c->tiled) {
        e = launch_step_tiled(a, c->plan, c->stream);
        c->plan.stall = 0;
    } else {
        e = launch_step_generic(a, c->storage, c->limiter, c->stream);
    }
    if (e != cudaSuccess) return fail(c, BTE_ECUDA, "forward step launch: %s", cudaGetErrorString(e));
    CU(c, launch_sis_sweep(a, static_cast<const float *>(c->e[c->cur]), static_cast<float *>(c->e[c->cur ^ 1]),
                           c->stream));
    c->cur ^= 1;
    TRY(refresh_moments(c));
    if (c->scheme != BTE_SCHEME_SYNTHETIC) return BTE_OK;
    // synthetic scheme: the forward step of the new state (e0 of its own T_L) gives the energy
    // residual, and the macroscopic equation corrects the T_L the next sweep relaxes towards
    if (!c->syn_pr) TRY(dalloc(c, &c->syn_pr, (size_t)c->nb * c->ncell));
    if (!c->syn_x) TRY(dalloc(c, &c->syn_x, synthetic_scratch_doubles(c->ncell)));
    StepArgs b = make_args(c);
    b.amp = a.amp;
    b.e_in = c->e[c->cur];
    b.e_out = c->e[c->cur ^ 1];
    b.ediff_in = c->ediff[c->ecur];
    b.ediff_out = c->ediff[c->ecur ^ 1];
    if (c->tiled) {
        e = launch_step_tiled(b, c->plan, c->stream);
        c->plan.stall = 0;
    } else {
        e = launch_step_generic(b, c->storage, c->limiter, c->stream);
    }
    if (e != cudaSuccess) return fail(c, BTE_ECUDA, "forward step launch: %s", cudaGetErrorString(e));
    double kb = 0.0;
    for (int k = 0; k < c->nb; ++k) kb += c->C[k] * c->v[k] * c->v[k] * c->tau[k];
    kb /= 3.0;
    const int max_cg = 40 * (c->n[0] + c->n[1] + c->n[2]);
    CU(c, synthetic_correct(b, c->h, c->wf, static_cast<const float *>(c->e[c->cur]),
                            static_cast<const float *>(c->e[c->cur ^ 1]), c->syn_pr, c->syn_x, kb, c->dt, max_cg, 1e-8,
                            c->TL, c->stream, &c->syn_cg));
    c->tl_corrected = true;
    return BTE_OK;
}

extern "C" bte_status bte_set_steady_scheme(bte_ctx *c, int scheme) {
    if (!c) return fail(nullptr, BTE_EINVAL, "ctx is NULL");
    if (scheme != BTE_SCHEME_SEQUENTIAL && scheme != BTE_SCHEME_SYNTHETIC) return fail(c, BTE_EINVAL, "bad scheme");
    c->scheme = scheme;
    return BTE_OK;
}

static bte_status sis_check(bte_ctx *c) {
    if (c->storage != BTE_STORE_F32) return fail(c, BTE_EUNSUPPORTED, "the implicit iteration needs FP32 storage");
    if (c->peer) return fail(c, BTE_ESTATE, "the context is coupled at an interface");
    return BTE_OK;
}

extern "C" bte_status bte_sis_iterate(bte_ctx *c, int n) {
    if (!c) return fail(nullptr, BTE_EINVAL, "ctx is NULL");
    if (n < 0) return fail(c, BTE_EINVAL, "n must be >= 0");
    TRY(sis_check(c));
    for (int s = 0; s < n; ++s) TRY(sis_one(c));
    return BTE_OK;
}

// eps_T and eps_q of Algorithm 2's loop condition between the last two of n more steps (or
// implicit iterations).
static bte_status residuals_after(bte_ctx *c, int nsteps, bool implicit, double *eps_T, double *eps_q);

extern "C" bte_status bte_residuals(bte_ctx *c, int nsteps, double *eps_T, double *eps_q) {
    if (!c) return fail(nullptr, BTE_EINVAL, "ctx is NULL");
    return residuals_after(c, nsteps, false, eps_T, eps_q);
}

extern "C" bte_status bte_run_steady_implicit(bte_ctx *c, long long max_iters, int check_every, double tol_T,
                                              double tol_q, long long *iters, double *eps_T, double *eps_q) {
    if (!c) return fail(nullptr, BTE_EINVAL, "ctx is NULL");
    if (max_iters < 1 || check_every < 1) return fail(c, BTE_EINVAL, "max_iters and check_every must be >= 1");
    if (!(tol_T >= 0.0) || !(tol_q >= 0.0)) return fail(c, BTE_EINVAL, "tolerances must be >= 0");
    TRY(sis_check(c));
    long long done = 0;
    double eT = HUGE_VAL, eq = HUGE_VAL;
    while (done < max_iters) {
        const int n = (int)std::min<long long>(check_every, max_iters - done);
        TRY(residuals_after(c, n, true, &eT, &eq));
        done += n;
        if (eT < tol_T && eq < tol_q) break;
    }
    if (iters) *iters = done;
    if (eps_T) *eps_T = eT;
    if (eps_q) *eps_q = eq;
    return BTE_OK;
}

static bte_status residuals_after(bte_ctx *c, int nsteps, bool implicit, double *eps_T, double *eps_q) {
    if (nsteps < 1) return fail(c, BTE_EINVAL, "nsteps must be >= 1");
    TRY(diag_buffers(c));
    if (!c->rs) TRY(dalloc(c, &c->rs, (size_t)2 * c->ncell + 4 * kResidBlocks + 4));
    double *Tp = c->rs, *qp = c->rs + c->ncell, *part = c->rs + 2 * c->ncell, *res = part + 4 * kResidBlocks;
    const DiagOut o = diag_layout(c);
    TRY(implicit ? bte_sis_iterate(c, nsteps - 1) : bte_step(c, nsteps - 1));
    CU(c, cudaMemsetAsync(c->dflag, 0, sizeof(int), c->stream));
    TRY(moments_on_device(c, o));
    CU(c, launch_resid_keep(o.T, o.q, c->ncell, Tp, qp, c->stream));
    TRY(implicit ? bte_sis_iterate(c, 1) : bte_step(c, 1));
    TRY(moments_on_device(c, o));
    CU(c, launch_residuals(o.T, o.q, Tp, qp, c->ncell, c->Tref, part, res, c->stream));
    double r[4];
    int flag = 0;
    CU(c, cudaMemcpyAsync(r, res, sizeof r, cudaMemcpyDeviceToHost, c->stream));
    CU(c, cudaMemcpyAsync(&flag, c->dflag, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CU(c, cudaStreamSynchronize(c->stream));
    TRY(check_device_flags(c));
    if (flag) return fail(c, BTE_ENONFINITE, "the state holds a non-finite value");
    const double N = (double)c->ncell;
    auto ratio = [](double rms, double mx) { return rms == 0.0 ? 0.0 : (mx > 0.0 ? rms / mx : HUGE_VAL); };
    if (eps_T) *eps_T = ratio(std::sqrt(r[0] / N), r[2]);
    if (eps_q) *eps_q = ratio(std::sqrt(r[1] / N), r[3]);
    return BTE_OK;
}

extern "C" bte_status bte_run_steady(bte_ctx *c, long long max_steps, int check_every, double tol_T, double tol_q,
                                     long long *steps_done, double *eps_T, double *eps_q) {
    if (!c) return fail(nullptr, BTE_EINVAL, "ctx is NULL");
    if (max_steps < 1 || check_every < 1) return fail(c, BTE_EINVAL, "max_steps and check_every must be >= 1");
    if (!(tol_T >= 0.0) || !(tol_q >= 0.0)) return fail(c, BTE_EINVAL, "tolerances must be >= 0");
    long long done = 0;
    double eT = HUGE_VAL, eq = HUGE_VAL;
    while (done < max_steps) {
        const int n = (int)std::min<long long>(check_every, max_steps - done);
        TRY(bte_residuals(c, n, &eT, &eq));
        done += n;
        if (eT < tol_T && eq < tol_q) break;
    }
    if (steps_done) *steps_done = done;
    if (eps_T) *eps_T = eT;
    if (eps_q) *eps_q = eq;
    return BTE_OK;
}

extern "C" bte_status bte_get_state(bte_ctx *c, void *dst, size_t bytes, float *ref, int on_device) {
    if (!c || !dst) return fail(c, BTE_EINVAL, "NULL argument");
    if (bytes != c->state_bytes) return fail(c, BTE_EINVAL, "bytes %zu != state_bytes %zu", bytes, c->state_bytes);
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    CU(c, cudaMemcpyAsync(dst, c->e[c->cur], bytes, kind, c->stream));
    if (ref && c->storage != BTE_STORE_F32) CU(c, cudaMemcpyAsync(ref, c->R, c->ncell * sizeof(float), kind, c->stream));
    else if (ref && on_device) CU(c, cudaMemsetAsync(ref, 0, c->ncell * sizeof(float), c->stream));
    else if (ref) memset(ref, 0, c->ncell * sizeof(float));
    if (!on_device) CU(c, cudaStreamSynchronize(c->stream));
    return BTE_OK;
}

extern "C" bte_status bte_set_state(bte_ctx *c, const void *src, size_t bytes, const float *ref, int on_device,
                                    int keep_step) {
    if (!c || !src) return fail(c, BTE_EINVAL, "NULL argument");
    if (bytes != c->state_bytes) return fail(c, BTE_EINVAL, "bytes %zu != state_bytes %zu", bytes, c->state_bytes);
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (ref && !on_device)
        for (long long i = 0; i < c->ncell; ++i)
            if (!std::isfinite(ref[i])) return fail(c, BTE_EINVAL, "ref holds a non-finite value at cell %lld", i);
    CU(c, cudaMemcpyAsync(c->e[c->cur], src, bytes, kind, c->stream));
    if (ref) CU(c, cudaMemcpyAsync(c->R, ref, c->ncell * sizeof(float), kind, c->stream));
    else CU(c, cudaMemsetAsync(c->R, 0, c->ncell * sizeof(float), c->stream));
    if (!on_device) CU(c, cudaStreamSynchronize(c->stream));
    TRY(refresh_moments(c));
    if (!keep_step) c->step = 0;
    return BTE_OK;
}

extern "C" bte_status bte_get_values(bte_ctx *c, float *dst, int on_device) {
    if (!c || !dst) return fail(c, BTE_EINVAL, "NULL argument");
    StepArgs a = make_args(c);
    a.e_in = c->e[c->cur];
    float *out = dst;
    const size_t bytes = (size_t)c->nelem * sizeof(float);
    if (!on_device) CU(c, cudaMalloc((void **)&out, bytes));
    cudaError_t e = launch_decode(a, c->storage, out, c->stream);
    if (e == cudaSuccess && !on_device) e = cudaMemcpyAsync(dst, out, bytes, cudaMemcpyDeviceToHost, c->stream);
    if (!on_device) {
        const cudaError_t e2 = cudaStreamSynchronize(c->stream);
        if (e == cudaSuccess) e = e2;
        cudaFree(out);
    }
    if (e != cudaSuccess) return fail(c, BTE_ECUDA, "state decode: %s", cudaGetErrorString(e));
    return BTE_OK;
}

extern "C" bte_status bte_get_info(const bte_ctx *c, bte_info *info) {
    if (!c || !info) return fail(nullptr, BTE_EINVAL, "NULL argument");
    info->dim = c->dim;
    info->nx = c->n[0];
    info->ny = c->n[1];
    info->nz = c->n[2];
    info->nbands = c->nb;
    info->ndirs = c->nd;
    info->ncell = c->ncell;
    info->nelem = c->nelem;
    info->state_bytes = c->state_bytes;
    info->elem_bytes = (int)c->elem_bytes;
    info->storage = c->storage;
    info->limiter = c->limiter;
    info->kernel = c->persist ? BTE_KERNEL_PERSISTENT : (c->tiled ? BTE_KERNEL_TILED : BTE_KERNEL_GENERIC);
    info->dt = c->dt;
    info->W = c->W;
    info->step = c->step;
    info->device_bytes = c->device_bytes;
    // forward + finalize passes (the tiled finalize adds one for walls that need ghost values)
    info->launches_per_step = c->persist ? 1 : 1 + (c->tiled ? tiled_finalize_launches(c->plan, c->bc) : 1);
    return BTE_OK;
}

extern "C" bte_status bte_get_quadrature(const bte_ctx *c, double *s, double *w) {
    if (!c) return fail(nullptr, BTE_EINVAL, "ctx is NULL");
    if (s) memcpy(s, c->s.data(), c->s.size() * sizeof(double));
    if (w) memcpy(w, c->w.data(), c->w.size() * sizeof(double));
    return BTE_OK;
}

extern "C" bte_status bte_profile(bte_ctx *c, int enable) {
    if (!c) return fail(nullptr, BTE_EINVAL, "ctx is NULL");
    if (enable) {
        CU(c, cudaStreamSynchronize(c->stream));
        c->ev_used = 0;
    }
    c->prof = enable != 0;
    return BTE_OK;
}

extern "C" bte_status bte_profile_read(bte_ctx *c, double *fwd_ms, long long *fwd_launches, double *fin_ms,
                                       long long *fin_launches) {
    if (!c) return fail(nullptr, BTE_EINVAL, "ctx is NULL");
    CU(c, cudaStreamSynchronize(c->stream));
    double f = 0, g = 0;
    const size_t n = c->ev_used / 3;
    for (size_t i = 0; i < n; ++i) {
        float a = 0, b = 0;
        CU(c, cudaEventElapsedTime(&a, c->ev[3 * i], c->ev[3 * i + 1]));
        CU(c, cudaEventElapsedTime(&b, c->ev[3 * i + 1], c->ev[3 * i + 2]));
        f += a;
        g += b;
    }
    if (fwd_ms) *fwd_ms = f;
    if (fin_ms) *fin_ms = g;
    if (fwd_launches) *fwd_launches = (long long)n;
    if (fin_launches) *fin_launches = (long long)n;
    return BTE_OK;
}

extern "C" bte_status bte_energy_noalloc(bte_ctx *c, double *E_total, double wall_flux[6]) {
    if (!c) return fail(nullptr, BTE_EINVAL, "ctx is NULL");
    StepArgs a = make_args(c);
    a.e_in = c->e[c->cur];
    a.ediff_in = c->ediff[c->ecur];
    double res[7];
    int nonfinite = 0;
    cudaError_t e = cudaSuccess;
    const int rc = launch_energy_noalloc(a, c->storage, c->limiter, c->d_w, c->d_s, c->d_v, res, &nonfinite, c->stream, &e);
    if (rc == 1)
        return fail(c, BTE_EINVAL,
                    "grid too large for the allocation-free reduction: every reduction (cells, or wall cells x bands) "
                    "must have at most %lld items",
                    energy_noalloc_max_items());
    if (rc != 0) return fail(c, BTE_ECUDA, "allocation-free energy reduction: %s", cudaGetErrorString(e));
    double L[3];
    for (int ax = 0; ax < 3; ++ax) L[ax] = ax < c->dim ? c->h[ax] : 1.0;
    const double V = L[0] * L[1] * L[2];
    if (E_total) *E_total = V * res[0];
    if (wall_flux)
        for (int wl = 0; wl < 6; ++wl) wall_flux[wl] = (wl < 2 * c->dim) ? (V / L[wl >> 1]) * res[1 + wl] : 0.0;
    if (nonfinite) return fail(c, BTE_ENONFINITE, "the state holds a non-finite value");
    return BTE_OK;
}

// ------------------------------------------------------------------------------------------
// Discrete adjoint with checkpointing (kernels: bte_adjoint.cu)
// ------------------------------------------------------------------------------------------
namespace {

// Everything that resumes the forward step from a state: codes, their reference, T_L and
// the wall ghost tables of that state, and the step index (source amplitude, rounding key).
struct Snap {
    void *e = nullptr;
    float *R = nullptr, *TL = nullptr;
    void *ediff = nullptr;
    long long step = 0;
};

struct AdjWork {
    bte_ctx *c;
    size_t ediff_bytes = 0;
    std::vector<void *> blocks;  // every device allocation of the call
    ~AdjWork() {
        for (void *p : blocks) cudaFree(p);
    }
    bool alloc(void **p, size_t bytes) {
        if (cudaMalloc(p, bytes ? bytes : 16) != cudaSuccess) {
            cudaGetLastError();
            *p = nullptr;
            return false;
        }
        blocks.push_back(*p);
        return true;
    }
    bool snap(Snap &s) {
        return alloc(&s.e, c->state_bytes) && alloc((void **)&s.R, c->ncell * sizeof(float)) &&
               alloc((void **)&s.TL, c->ncell * sizeof(float)) && alloc(&s.ediff, ediff_bytes);
    }
};

}  // namespace

static bte_status snap_save(bte_ctx *c, Snap &s, size_t ediff_bytes) {
    CU(c, cudaMemcpyAsync(s.e, c->e[c->cur], c->state_bytes, cudaMemcpyDeviceToDevice, c->stream));
    CU(c, cudaMemcpyAsync(s.R, c->R, c->ncell * sizeof(float), cudaMemcpyDeviceToDevice, c->stream));
    CU(c, cudaMemcpyAsync(s.TL, c->TL, c->ncell * sizeof(float), cudaMemcpyDeviceToDevice, c->stream));
    CU(c, cudaMemcpyAsync(s.ediff, c->ediff[c->ecur], ediff_bytes, cudaMemcpyDeviceToDevice, c->stream));
    s.step = c->step;
    return BTE_OK;
}

static bte_status snap_restore(bte_ctx *c, const Snap &s, size_t ediff_bytes) {
    CU(c, cudaMemcpyAsync(c->e[c->cur], s.e, c->state_bytes, cudaMemcpyDeviceToDevice, c->stream));
    CU(c, cudaMemcpyAsync(c->R, s.R, c->ncell * sizeof(float), cudaMemcpyDeviceToDevice, c->stream));
    CU(c, cudaMemcpyAsync(c->TL, s.TL, c->ncell * sizeof(float), cudaMemcpyDeviceToDevice, c->stream));
    CU(c, cudaMemcpyAsync(c->ediff[c->ecur], s.ediff, ediff_bytes, cudaMemcpyDeviceToDevice, c->stream));
    c->step = s.step;
    return BTE_OK;
}

extern "C" bte_status bte_adjoint(bte_ctx *c, int nsteps, int ckpt_every, const double *probe, double *J,
                                  double *dJ_dQ, double *dJ_dlogtau) {
    if (!c) return fail(nullptr, BTE_EINVAL, "ctx is NULL");
    if (!probe) return fail(c, BTE_EINVAL, "probe is NULL");
    if (nsteps < 0) return fail(c, BTE_EINVAL, "nsteps must be >= 0");
    if (ckpt_every < 0) return fail(c, BTE_EINVAL, "ckpt_every must be >= 0");
    if (c->peer) return fail(c, BTE_ESTATE, "the context is coupled at an interface (no adjoint of the pair)");
    if (c->tl_corrected) TRY(refresh_moments(c));
    for (long long i = 0; i < c->ncell; ++i)
        if (!std::isfinite(probe[i])) return fail(c, BTE_EINVAL, "probe holds a non-finite value at cell %lld", i);
    const long long nc = c->ncell, nel = c->nelem;
    int K = ckpt_every > 0 ? ckpt_every : std::max(1, (int)std::ceil(std::sqrt((double)std::max(nsteps, 1))));
    K = std::max(1, std::min(K, std::max(nsteps, 1)));
    const int nseg = nsteps > 0 ? (nsteps + K - 1) / K : 0;
    AdjWork w;
    w.c = c;
    w.ediff_bytes = ((size_t)6 * c->nb * c->wc_max + 16) * c->elem_bytes;
    // adjoint state and partials
    float *lam[2], *mu[2], *pmu, *pq, *pt, *pr;
    double *gQ, *gt, *tpart;
    const int ntb = adj_tau_blocks(nc);
    if (!w.alloc((void **)&lam[0], nel * sizeof(float)) || !w.alloc((void **)&lam[1], nel * sizeof(float)) ||
        !w.alloc((void **)&mu[0], nc * sizeof(float)) || !w.alloc((void **)&mu[1], nc * sizeof(float)) ||
        !w.alloc((void **)&pmu, (size_t)c->nb * nc * sizeof(float)) ||
        !w.alloc((void **)&pq, (size_t)c->nb * nc * sizeof(float)) ||
        !w.alloc((void **)&pt, (size_t)c->nb * nc * sizeof(float)) || !w.alloc((void **)&pr, nc * sizeof(float)) ||
        !w.alloc((void **)&gQ, nc * sizeof(double)) || !w.alloc((void **)&gt, c->nb * sizeof(double)) ||
        !w.alloc((void **)&tpart, (size_t)c->nb * ntb * sizeof(double)))
        return fail(c, BTE_ENOMEM, "adjoint buffers do not fit in device memory");
    // checkpoints: one per segment, then within a segment either every state (when K states
    // fit in half of the free memory) or every K2 = ceil(sqrt K)-th state, its sub-segments
    // recomputed into K2 more snapshots
    const size_t snap_bytes = c->state_bytes + 2 * nc * sizeof(float) + w.ediff_bytes;
    size_t mfree = 0, mtot = 0;
    CU(c, cudaMemGetInfo(&mfree, &mtot));
    const size_t fixed = (size_t)(nseg + 1) * snap_bytes;
    int K2 = 1;
    if (fixed + (size_t)K * snap_bytes > mfree / 2) K2 = (int)std::ceil(std::sqrt((double)K));
    if (const char *env = std::getenv("BTE_ADJOINT_INNER_STRIDE")) {  // testing the two-level path
        const int v = std::atoi(env);
        if (v >= 1) K2 = std::min(v, K);
    }
    const int n2 = (K + K2 - 1) / K2;
    std::vector<Snap> L1(nseg), L2(n2), L3(K2 > 1 ? K2 : 0);
    Snap fin;
    for (auto &s : L1)
        if (!w.snap(s)) return fail(c, BTE_ENOMEM, "adjoint checkpoints do not fit in device memory");
    for (auto &s : L2)
        if (!w.snap(s)) return fail(c, BTE_ENOMEM, "adjoint checkpoints do not fit in device memory");
    for (auto &s : L3)
        if (!w.snap(s)) return fail(c, BTE_ENOMEM, "adjoint checkpoints do not fit in device memory");
    if (!w.snap(fin)) return fail(c, BTE_ENOMEM, "adjoint checkpoints do not fit in device memory");
    // tiled adjoint: segment partials, wall corrections, block partials of sum mu T_L
    float *Pm = nullptr, *Pq = nullptr, *Ps = nullptr, *corr[3] = {nullptr, nullptr, nullptr};
    double *mtp = nullptr;
    // the tiled adjoint takes rows that fill the forward kernel's row capacity exactly
    const bool tiled_adj = c->tiled && c->nd <= adj_walls_max_dirs() && c->plan.nx == c->n[0];
    float *wscr = nullptr;
    if (tiled_adj) {
        const size_t gt_rows = (size_t)std::max(1, c->plan.G);
        if (!w.alloc((void **)&Pm, gt_rows * c->plan.tcells * sizeof(float)) ||
            !w.alloc((void **)&Pq, gt_rows * c->plan.tcells * sizeof(float)) ||
            !w.alloc((void **)&Ps, 2 * gt_rows * sizeof(float)) ||
            !w.alloc((void **)&mtp, (size_t)((nc + 255) / 256) * sizeof(double)) ||
            !w.alloc((void **)&wscr, (size_t)std::max(1LL, adj_walls_scratch_floats(make_args(c))) * sizeof(float)))
            return fail(c, BTE_ENOMEM, "adjoint buffers do not fit in device memory");
        for (int ax = 0; ax < c->dim; ++ax) {
            if (c->bc[2 * ax] == BTE_BC_PERIODIC) continue;
            const long long lines = nc / c->n[ax];
            if (!w.alloc((void **)&corr[ax], (size_t)c->nb * 4 * lines * sizeof(float)))
                return fail(c, BTE_ENOMEM, "adjoint buffers do not fit in device memory");
        }
    }
    {
        std::vector<float> pf(probe, probe + nc);
        CU(c, cudaMemcpyAsync(pr, pf.data(), nc * sizeof(float), cudaMemcpyHostToDevice, c->stream));
        CU(c, cudaMemsetAsync(gQ, 0, nc * sizeof(double), c->stream));
        CU(c, cudaMemsetAsync(gt, 0, c->nb * sizeof(double), c->stream));
        CU(c, cudaStreamSynchronize(c->stream));
    }
    const bool prof = c->prof;
    c->prof = false;  // the forward steps of the adjoint are not traced as bte_step calls
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    double adj_ms = 0, rec_ms = 0;
    long long adj_n = 0, rec_n = 0;
    if (prof) {
        CU(c, cudaEventCreate(&ev0));
        CU(c, cudaEventCreate(&ev1));
    }
    auto timed_steps = [&](int n) -> bte_status {
        if (n <= 0) return BTE_OK;
        if (prof) CU(c, cudaEventRecord(ev0, c->stream));
        bte_status st = bte_step(c, n);
        if (st != BTE_OK) return st;
        if (prof) {
            float ms = 0;
            CU(c, cudaEventRecord(ev1, c->stream));
            CU(c, cudaEventSynchronize(ev1));
            CU(c, cudaEventElapsedTime(&ms, ev0, ev1));
            rec_ms += ms;
            rec_n += n;
        }
        return BTE_OK;
    };
    int cur = 0;
    long long base_step = c->step;
    AdjArgs g;
    g.w = c->wf;
    g.W = (float)c->W;
    g.pmu = pmu;
    g.pq = pq;
    g.pt = pt;
    auto adj_step = [&](const Snap &s) -> bte_status {
        StepArgs a = make_args(c);
        a.e_in = s.e;
        a.R = s.R;
        a.TL = s.TL;
        a.ediff_in = s.ediff;
        g.lam_in = lam[cur];
        g.lam_out = lam[cur ^ 1];
        g.mu_in = mu[cur];
        if (prof) CU(c, cudaEventRecord(ev0, c->stream));
        if (tiled_adj) {
            // interior and periodic faces on the tiles, then the faces next to each wall, then
            // mu^n, dJ/dQ (the q^n of lambda^n with the amplitude of step n-1) and dJ/dlog tau
            CU(c, launch_adj_tiled(a, c->plan, lam[cur], lam[cur ^ 1], mu[cur], Pm, Pq, Ps, c->wf, c->storage,
                                   c->limiter, c->stream));
            CU(c, launch_adj_walls(a, g, c->storage, c->limiter, lam[cur ^ 1], corr, wscr, c->stream));
            AdjTFinal f;
            f.tile_seg0 = c->plan.unit_seg0 + c->plan.U;
            f.seg_band = c->plan.seg_band;
            f.Pm = Pm;
            f.Pq = Pq;
            f.Ps = Ps;
            f.mu_in = mu[cur];
            for (int ax = 0; ax < 3; ++ax) f.corr[ax] = corr[ax];
            f.G = c->plan.G;
            f.tcells = c->plan.tcells;
            f.ty = c->plan.ty;
            f.tz = c->plan.tz;
            f.nty = c->plan.nty;
            const float amp_prev = s.step > base_step ? (float)amplitude_at(c, s.step - 1) : 0.f;
            CU(c, launch_adj_tfinal(a, f, amp_prev, mu[cur ^ 1], gQ, mtp, c->W, gt, c->stream));
        } else {
            CU(c, launch_adj_step(a, g, c->storage, c->limiter, c->stream));
            CU(c, launch_adj_reduce(a, g, (float)amplitude_at(c, s.step), mu[cur ^ 1], gQ, tpart, gt, c->stream));
        }
        if (prof) {
            float ms = 0;
            CU(c, cudaEventRecord(ev1, c->stream));
            CU(c, cudaEventSynchronize(ev1));
            CU(c, cudaEventElapsedTime(&ms, ev0, ev1));
            adj_ms += ms;
            ++adj_n;
        }
        cur ^= 1;
        return BTE_OK;
    };
    bte_status st = BTE_OK;
    auto run = [&]() -> bte_status {
        // forward sweep, keeping the segment checkpoints
        base_step = c->step;
        for (int s = 0; s < nseg; ++s) {
            TRY(snap_save(c, L1[s], w.ediff_bytes));
            TRY(timed_steps(std::min(K, nsteps - s * K)));
        }
        TRY(snap_save(c, fin, w.ediff_bytes));
        // J = sum p T_L^N and lambda^N
        {
            std::vector<float> tl(nc);
            CU(c, cudaMemcpyAsync(tl.data(), c->TL, nc * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
            CU(c, cudaStreamSynchronize(c->stream));
            double jv = 0;
            for (long long i = 0; i < nc; ++i) jv += probe[i] * (double)tl[i];
            if (J) *J = jv;
            StepArgs a = make_args(c);
            a.e_in = c->e[c->cur];
            g.lam_out = lam[cur];
            g.lam_in = nullptr;
            g.mu_in = nullptr;
            CU(c, launch_adj_init(a, g, c->storage, pr, c->stream));
            // the tiled path takes dJ/dQ of step N-1 from q^N here; the generic step kernel
            // takes it from lambda^{n+1} itself
            const float amp_last = tiled_adj && nsteps > 0 ? (float)amplitude_at(c, c->step - 1) : 0.f;
            CU(c, launch_adj_reduce(a, g, amp_last, mu[cur], gQ, tpart, gt, c->stream));
        }
        // reverse sweep, segment by segment
        for (int s = nseg - 1; s >= 0; --s) {
            const int n0 = s * K, n1 = std::min(nsteps, n0 + K);
            TRY(snap_restore(c, L1[s], w.ediff_bytes));
            const int ns2 = (n1 - n0 + K2 - 1) / K2;
            for (int m = n0; m < n1; ++m) {
                if ((m - n0) % K2 == 0) TRY(snap_save(c, L2[(m - n0) / K2], w.ediff_bytes));
                if ((m - n0) / K2 == ns2 - 1 && K2 > 1) break;  // the last sub-checkpoint is taken
                if (m < n1 - 1) TRY(timed_steps(1));
            }
            if (K2 == 1) {
                for (int m = n1 - 1; m >= n0; --m) TRY(adj_step(L2[m - n0]));
                continue;
            }
            for (int sub = ns2 - 1; sub >= 0; --sub) {
                const int m0 = n0 + sub * K2, m1 = std::min(n1, m0 + K2);
                TRY(snap_restore(c, L2[sub], w.ediff_bytes));
                for (int m = m0; m < m1; ++m) {
                    TRY(snap_save(c, L3[m - m0], w.ediff_bytes));
                    if (m < m1 - 1) TRY(timed_steps(1));
                }
                for (int m = m1 - 1; m >= m0; --m) TRY(adj_step(L3[m - m0]));
            }
        }
        TRY(snap_restore(c, fin, w.ediff_bytes));
        if (dJ_dQ) CU(c, cudaMemcpyAsync(dJ_dQ, gQ, nc * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        if (dJ_dlogtau) CU(c, cudaMemcpyAsync(dJ_dlogtau, gt, c->nb * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        CU(c, cudaStreamSynchronize(c->stream));
        return check_device_flags(c);
    };
    st = run();
    c->prof = prof;
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
    if (st == BTE_OK && prof) {
        c->adj_ms = adj_ms;
        c->adj_steps = adj_n;
        c->adj_recompute_ms = rec_ms;
        c->adj_recompute_steps = rec_n;
    }
    if (st != BTE_OK) cudaStreamSynchronize(c->stream);
    return st;
}

extern "C" bte_status bte_adjoint_profile_read(bte_ctx *c, double *adj_ms, long long *adj_steps, double *fwd_ms,
                                               long long *fwd_steps) {
    if (!c) return fail(nullptr, BTE_EINVAL, "ctx is NULL");
    if (adj_ms) *adj_ms = c->adj_ms;
    if (adj_steps) *adj_steps = c->adj_steps;
    if (fwd_ms) *fwd_ms = c->adj_recompute_ms;
    if (fwd_steps) *fwd_steps = c->adj_recompute_steps;
    return BTE_OK;
}
