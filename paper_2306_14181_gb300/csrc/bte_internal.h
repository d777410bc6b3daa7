// Internal declarations shared by the host side (bte_api.cu) and the kernels of the
// GB300 explicit DOM transient step.  Not part of the public ABI (include/bte.h).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

namespace bte {

constexpr int kBcIsothermal = 0, kBcDiffuse = 1, kBcSpecular = 2, kBcPeriodic = 3;
constexpr int kStoreF32 = 0, kStoreF16 = 1, kStoreBF16 = 2;
constexpr int kLimFirst = 0, kLimMinmod = 1, kLimVanAlbada = 2;

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
    // fields
    const void *e_in;
    void *e_out;
    const float *TL;       // [ncell] T_L^n
    const float *Q;        // [ncell] or null
    const void *ediff_in;  // [6][nb][wc_max] diffuse-wall incoming values from e^n (storage format)
    void *ediff_out;       // [6][nb][wc_max] from e^{n+1} (storage format)
    float *P;              // moment partials [G][ncell]
};

// Launchers (bte_kernels.cu).  All return the launch error (cudaGetLastError()).
cudaError_t launch_fill(const StepArgs &a, int storage, const double *dT0, cudaStream_t s);
cudaError_t launch_moment_only(const StepArgs &a, int storage, cudaStream_t s);
cudaError_t launch_step_generic(const StepArgs &a, int storage, int limiter, cudaStream_t s);
cudaError_t launch_finalize(const StepArgs &a, int G, float *TL_out, cudaStream_t s);

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
// Energy and wall flows into host7[7] with no device allocation (file-scope device scratch).
// Returns 0, 1 (grid larger than the scratch covers) or 2 (CUDA error in *err).
int launch_energy_noalloc(const StepArgs &a, int storage, int limiter, const double *w, const double *sv,
                          const double *v, double *host7, int *nonfinite, cudaStream_t s, cudaError_t *err);
long long energy_noalloc_max_items();

}  // namespace bte
