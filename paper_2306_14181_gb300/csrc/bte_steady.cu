// Steady state by the implicit discrete-ordinates method, sequential iterative scheme
// (Sec. 3.3-3.5 of arXiv 2306.14181, Eq. disretized_BTE in delta form).
//
// One iteration: the forward step computes e^n + dt R (R: the steady equation's right-hand side
// with the step's limited second-order faces, walls and source), then this sweep solves, for
// every band k and direction d, the first-order upwind system of the increment
//     (dt/tau_k + sum_a |nu_a|) De_i - sum_a |nu_a| De_{up_a(i)} = dt R_i,
// nu_a = dt v_k s_{d,a} / h_a being the step's own Courant numbers and up_a(i) the upwind
// neighbour of cell i along axis a; across a wall (periodic pairs included) the upwind De is 0,
// so each plane's system is lower triangular in upwind order and one sweep solves it:
// z, y and x each run from the upwind side.
//
// One warp a plane.  A row is cut into chunks of 128 cells in upwind order, 4 consecutive cells
// a lane.  Along x the recurrence De_u = a_u + b De_{u-1} (b = |nu_x| / diag, a_u the cell's
// right-hand side with its y and z upwind terms, over diag) is a composition of affine maps:
// each lane folds its 4 cells into one map, a warp scan of maps (Kogge-Stone, 5 shuffle steps)
// gives every lane the De entering its cells, and the lanes then run their 4 cells again.  The
// y and z upwind De are read back from the row and slice the same lane wrote before (e_io -
// e_in at the same x), so a lane only ever reads its own stores.
#include <cuda_runtime.h>

#include "bte_internal.h"

namespace bte {
namespace {

constexpr int kSweepWarps = 4;
constexpr int kCellsPerLane = 4;

__global__ void __launch_bounds__(kSweepWarps * 32) k_sis_sweep(const StepArgs a, const float *__restrict__ e_in,
                                                                 float *e_io) {
    const int lane = threadIdx.x & 31;
    const long long plane = (long long)blockIdx.x * kSweepWarps + (threadIdx.x >> 5);
    if (plane >= (long long)a.nb * a.nd) return;
    const int k = (int)(plane / a.nd);
    const int nx = a.n[0], ny = a.n[1], nz = a.n[2];
    const float nux = fabsf(a.nu[3 * plane]), nuy = fabsf(a.nu[3 * plane + 1]), nuz = fabsf(a.nu[3 * plane + 2]);
    const int sx = a.nu[3 * plane] >= 0.f ? 1 : -1;
    const int sy = a.nu[3 * plane + 1] >= 0.f ? 1 : -1;
    const int sz = a.nu[3 * plane + 2] >= 0.f ? 1 : -1;
    const float diag = a.band[k].dtinv + nux + nuy + nuz;
    const float inv = 1.f / diag;
    const float b = nux * inv;
    const float *ei = e_in + plane * a.ncell;
    float *eo = e_io + plane * a.ncell;
    const long long dyg = (long long)sy * nx, dzg = (long long)sz * nx * ny;
    for (int uz = 0; uz < nz; ++uz) {
        const int z = sz > 0 ? uz : nz - 1 - uz;
        for (int uy = 0; uy < ny; ++uy) {
            const int y = sy > 0 ? uy : ny - 1 - uy;
            const long long row = ((long long)z * ny + y) * nx;
            float carry = 0.f;  // De of the cell before the chunk (0 at the upwind wall)
            for (int u0 = 0; u0 < nx; u0 += 32 * kCellsPerLane) {
                float av[kCellsPerLane];
                long long ix[kCellsPerLane];
                int nv = 0;
                #pragma unroll
                for (int v = 0; v < kCellsPerLane; ++v) {
                    const int u = u0 + lane * kCellsPerLane + v;
                    av[v] = 0.f;
                    ix[v] = -1;
                    if (u < nx) {
                        const int x = sx > 0 ? u : nx - 1 - u;
                        const long long i = row + x;
                        float r = eo[i] - ei[i];  // dt R
                        if (uy > 0) r = fmaf(nuy, eo[i - dyg] - ei[i - dyg], r);
                        if (uz > 0) r = fmaf(nuz, eo[i - dzg] - ei[i - dzg], r);
                        av[v] = r * inv;
                        ix[v] = i;
                        ++nv;
                    }
                }
                // the lane's map De_out = A + B De_in over its valid cells
                float A = 0.f, B = 1.f;
                #pragma unroll
                for (int v = 0; v < kCellsPerLane; ++v)
                    if (v < nv) {
                        A = fmaf(b, A, av[v]);
                        B *= b;
                    }
                // inclusive scan of the maps over the lanes: lane l composes lanes 0..l
                #pragma unroll
                for (int off = 1; off < 32; off <<= 1) {
                    const float Au = __shfl_up_sync(0xffffffffu, A, off);
                    const float Bu = __shfl_up_sync(0xffffffffu, B, off);
                    if (lane >= off) {
                        A = fmaf(B, Au, A);
                        B *= Bu;
                    }
                }
                const float Ain = __shfl_up_sync(0xffffffffu, A, 1);
                const float Bin = __shfl_up_sync(0xffffffffu, B, 1);
                float d = lane == 0 ? carry : fmaf(Bin, carry, Ain);
                #pragma unroll
                for (int v = 0; v < kCellsPerLane; ++v)
                    if (v < nv) {
                        d = fmaf(b, d, av[v]);
                        eo[ix[v]] = ei[ix[v]] + d;
                    }
                // De of the chunk's last cell: the composed map of all 32 lanes applied to carry
                carry = __shfl_sync(0xffffffffu, fmaf(B, carry, A), 31);
            }
        }
    }
}

}  // namespace

cudaError_t launch_sis_sweep(const StepArgs &a, const float *e_in, float *e_io, cudaStream_t s) {
    const long long planes = (long long)a.nb * a.nd;
    const unsigned blocks = (unsigned)((planes + kSweepWarps - 1) / kSweepWarps);
    k_sis_sweep<<<blocks, kSweepWarps * 32, 0, s>>>(a, e_in, e_io);
    return cudaGetLastError();
}

}  // namespace bte
