// Internal declarations shared by the host side (bte_api.cu) and the kernels of the
// GB300 explicit DOM transient step.  Not part of the public ABI (include/bte.h).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

namespace bte {

constexpr int kBcIsothermal = 0, kBcDiffuse = 1, kBcSpecular = 2, kBcPeriodic = 3;
constexpr int kStoreF32 = 0, kStoreF16 = 1, kStoreBF16 = 2;
constexpr int kLimFirst = 0, kLimMinmod = 1, kLimVanAlbada = 2;

// Random bits of the stochastic rounding of element (plane, cell): the 32-bit integer hash
// lowbias32 (C. Wellons, "hash-prospector") applied to the cell index xor a per-plane key,
// itself the hash of the step key plus the plane index times the golden-ratio constant.
__host__ __device__ __forceinline__ uint32_t mix32(uint32_t x) {
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}
__host__ __device__ __forceinline__ uint32_t plane_key(uint32_t srkey, int plane) {
    return mix32(srkey + (uint32_t)plane * 0x9e3779b9u);
}

// Per-band FP32 constants of the update (index k).
struct BandConst {
    float dtinv;   // dt / tau_k
    float ck;      // C_k / W      (e0_k = ck * T_L)
    float srck;    // dt C_k / (sum C W)   (source per unit Q and amplitude)
    float scale;   // 16-bit storage scale s_k = C_k T_scale / W (1 for FP32)
    float inv_scale;
    float wtau;    // 1 / tau_k
    float pad0, pad1;
};

// Everything one forward-step launch reads.  Passed by value.
struct StepArgs {
    int dim;
    int n[3];          // nx, ny, nz
    long long stride[3];   // 1, nx, nx*ny
    long long ncell;
    int nb, nd;
    int bc[6];
    int wc_max;        // wall cells per wall slot in the e_diff buffers
    float inv_den[6];  // 1 / sum_{s.n<0} w |s.n| per diffuse wall
    float amp;         // source amplitude a(t_n)
    float invD;        // 1 / sum_k C_k / tau_k
    // tables (device)
    const float *nu;       // [plane][3]  dt v_k s_{d,a} / dx_a (signed; 0 on inactive axes)
    const float *wmom;     // [plane]     w_d / tau_k, the T_L moment weight
    const float *wdiff;    // [6][nd]     w_d (s_d.n) for directions leaving through the wall, else 0
    const int *mirror;     // [3][nd]
    const BandConst *band; // [nb]
    const float *iso;      // [6][nb]     C_k T_wall / W, rounded to a value the storage format holds
    const float *jmp;      // [3][nb]     C_k dT_jump[a] / W: offset of the -a wall's periodic ghosts (+a: minus it)
    // fields
    const void *e_in;
    void *e_out;
    const float *TL;       // [ncell] T_L^n; also the code reference of e_out (16-bit storage)
    const float *R;        // [ncell] code reference of e_in (16-bit storage: T_L of the step that wrote it)
    float invTs;           // 1 / T_scale
    int sr;                // 16-bit codes of e_out: 0 round to nearest, 1 stochastic rounding
    unsigned srkey;        // key of this step's rounding bits (from the seed and the step index)
    const float *Q;        // [ncell] or null
    const void *ediff_in;  // [6][nb][wc_max] wall ghost values of e^n: diffuse-wall values, and for
                           // 16-bit storage the thermalizing-wall emission (storage format, coded
                           // against the reference of the wall cell like the state)
    void *ediff_out;       // [6][nb][wc_max] the same for e^{n+1}
    float *P;              // moment partials [G][ncell]
};

// Launchers (bte_kernels.cu).  All return the launch error (cudaGetLastError()).
cudaError_t launch_fill(const StepArgs &a, int storage, const double *dT0, float *R_out, cudaStream_t s);
cudaError_t launch_moment_only(const StepArgs &a, int storage, cudaStream_t s);
cudaError_t launch_step_generic(const StepArgs &a, int storage, int limiter, cudaStream_t s);
cudaError_t launch_finalize(const StepArgs &a, int G, float *TL_out, cudaStream_t s);
// Persistent single-CTA run of nsteps steps of a 1-D FP32 problem (bte_persist.cu): e_io in
// place, T_L and the diffuse-wall values of the final state out; amps[s] the source amplitude
// of step s of the call.
size_t persist_1d_smem(const StepArgs &a);
cudaError_t launch_persist_1d(const StepArgs &a, int limiter, int nsteps, const float *amps, float *e_io,
                              float *tl_out, float *ediff_out, cudaStream_t s);
// Decoded state values e (FP32, [nb*nd][ncell]) of e_in into out (device).
cudaError_t launch_decode(const StepArgs &a, int storage, float *out, cudaStream_t s);

// FP64 diagnostics (bte_kernels.cu).
struct DiagOut {
    double *T, *TL, *q;       // [ncell], [ncell], [3][ncell] (device)
    double *cellE;            // [ncell] sum_k sum_d w e  per cell
    double *wallpart;         // [6][nb][wc_max] partial wall flows
    int *nonfinite;           // flag
};
cudaError_t launch_moments64(const StepArgs &a, int storage, const double *w, const double *sv, const double *v,
                             const double *invtau, double sumC, double D, DiagOut o, cudaStream_t s);
cudaError_t launch_wallflux64(const StepArgs &a, int storage, int limiter, const double *w, const double *sv,
                              const double *v, DiagOut o, cudaStream_t s);
// Deterministic FP64 sum of n values into *out (device); scratch holds >= 1024 doubles.
cudaError_t launch_sum64(const double *x, long long n, double *scratch, double *out, cudaStream_t s);
// Residuals of the transient loop condition (Algorithm 2) between two states: keep T^n, |q|^n
// (FP64, from launch_moments64's T and q) into Tp, qp; then out4 = {sum (T^n - T^{n+1})^2,
// sum (|q|^n - |q|^{n+1})^2, max (T_ref + T^{n+1}), max |q^{n+1}|}; scratch >= 4 kResidBlocks.
constexpr int kResidBlocks = 512;
cudaError_t launch_resid_keep(const double *T, const double *q, long long n, double *Tp, double *qp, cudaStream_t s);
cudaError_t launch_residuals(const double *T, const double *q, const double *Tp, const double *qp, long long n,
                             double Tref, double *scratch, double *out4, cudaStream_t s);
// Interface between two materials (Sec. 2.2 (v)): for every band k and interface cell j, with
// S_A, S_B the two sides' plain diffuse values (from eA / eB where pure_a / pure_b, else from the
// copies pa / pb an earlier call kept), writes S_A, S_B to pa, pb and the incoming values
// eA = beta_ba S_B + (1 - beta_ab) S_A, eB = beta_ab S_A + (1 - beta_ba) S_B.  eA, eB: the
// interface wall's rows of each side's e_diff (band stride sa / sb); pa, pb: [nb][ncw];
// beta: [4][nb] = beta_ab, 1 - beta_ab, beta_ba, 1 - beta_ba.
cudaError_t launch_iface_mix(float *eA, float *pa, int pure_a, int sa, float *eB, float *pb, int pure_b, int sb,
                             const float *beta, int nb, int ncw, cudaStream_t s);
// Steady implicit DOM, sequential iteration (Sec. 3.3-3.5): e_io holds the forward step's output
// e^n + dt R on entry and e^{n+1} = e^n + De on exit, De solving each plane's first-order upwind
// system (dt/tau + sum|nu_a|) De_i - sum_a |nu_a| De_{up_a(i)} = dt R_i (0 across walls).  FP32.
cudaError_t launch_sis_sweep(const StepArgs &a, const float *e_in, float *e_io, cudaStream_t s);
// Synthetic iterative scheme (Sec. 3.5): from e_in (the state) and e_out (the forward step's
// e_in + dt R, R with e0 of T_L(e_in)), the energy residual r = sum_k sum_d w_d R, then
// conjugate gradients on k_bulk L dT = -r (L: the cell Laplacian, thermalizing walls hold the
// temperature, reflecting walls pass no heat, periodic pairs wrap; mean-free when no wall is
// thermalizing), and TL += dT.  Pr: nb * ncell floats; scratch: synthetic_scratch_doubles(ncell).
// 1-D grids with a thermalizing wall and no periodic pair are solved directly (Thomas); else
// CG, synchronising the stream every 16 iterations to test |r_cg| <= rel_tol |b|.
constexpr int kSynthParts = 304;
size_t synthetic_scratch_doubles(long long ncell);
cudaError_t synthetic_correct(const StepArgs &a, const double h[3], const float *w, const float *e_in,
                              const float *e_out, float *Pr, double *scratch, double k_bulk, double dt, int max_cg,
                              double rel_tol, float *TL, cudaStream_t s, int *cg_iters);
// Energy and wall flows into host7[7] with no device allocation (file-scope device scratch).
// Returns 0, 1 (grid larger than the scratch covers) or 2 (CUDA error in *err).
int launch_energy_noalloc(const StepArgs &a, int storage, int limiter, const double *w, const double *sv,
                          const double *v, double *host7, int *nonfinite, cudaStream_t s, cudaError_t *err);
long long energy_noalloc_max_items();

}  // namespace bte
