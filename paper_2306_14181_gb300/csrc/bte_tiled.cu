// Shared-memory tiled forward kernel of the explicit DOM transient step (arXiv 2306.14181,
// Sec. 4, Eq. disretized_transientBTE), written for sm_103a.
//
// Work unit: a plane-tile = one (band k, direction d) plane restricted to a spatial tile of full
// x-rows (nx = 32 * VX cells) by TY rows (by TZ slices in 3-D).  Persistent CTAs take equal,
// contiguous ranges of the tile-major list of plane-tiles.  In each CTA one producer warp (of a
// producer warpgroup that hands its spare registers to the consumers) moves every box row the
// stencil needs into a ring of shared-memory stages with TMA bulk copies (cp.async.bulk,
// completion counted on an mbarrier): the tile with its upwind-oriented halo (two rows upwind,
// one downwind per axis) and, for rows outside the domain, the ghost rows of Sec. 2.2 - the
// wrapped row (periodic), the mirrored direction's row (specular), the wall row itself
// (outgoing directions), the diffuse-wall value row, or a constant (thermalizing wall).
// Consumer warps (16 in 2-D, 12 in 3-D) own 4 rows of VL = 3 or 4 cells a lane (two warps per
// 256-cell row), take the x-stencil from warp shuffles, stream y in registers and read z from
// shared memory, store e^{n+1} straight to global memory, and keep the T_L moment partials and
// the per-cell source terms in shared memory for a whole segment (one tile and one band).  A
// segment's partials go to one row of P (and of PW for diffuse walls); the finalize passes sum
// a tile's segments in a fixed order, so the reduction is deterministic without atomics.  Every
// mbarrier wait is bounded.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "bte_tiled_kernel.cuh"

namespace bte {

namespace tiled {

// ---- finalize passes ---------------------------------------------------------------------
// T_L_i = (sum over the segments of i's tile, in order) / sum_k C_k / tau_k
__global__ void __launch_bounds__(256) k_finalize_tiled(const StepArgs a, const TiledArgs p, float *TL) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.ncell) return;
    const int nx = a.n[0], ny = a.n[1];
    const int x = (int)(i % nx), y = (int)((i / nx) % ny), z = (int)(i / ((long long)nx * ny));
    const int ty = y / p.ty, tz = z / p.tz;
    const int tile = tz * p.nty + ty;
    // the tile arrays keep rows of p.nxt cells (the kernel's row capacity, >= nx)
    const int li = ((z - tz * p.tz) * p.ty + (y - ty * p.ty)) * p.nxt + x;
    // the tile's segments: its units in part order, each unit's bands in order
    const int g0 = p.tile_seg0[tile], g1 = p.tile_seg0[tile + 1];
    const float *P = a.P + li;
    float s = 0.f;
    #pragma unroll 8
    for (int g = g0; g < g1; ++g) s += P[(size_t)g * p.tcells];
    TL[i] = s * a.invD;
}

// Wall ghost values of e^{n+1} for the next step.  Diffuse wall: e_diff[w][k][wall cell] =
// (sum over the band-k segments of the cell's tile) / sum_in w|s.n|.  With 16-bit storage the
// value is coded against the wall cell's new reference rho = T_L^n / T_scale, and thermalizing
// y/z walls get their emission C_k T_w / W coded the same way.
struct WallList {
    int w[6];
};

template <int S>
__global__ void __launch_bounds__(256) k_ediff_tiled(const StepArgs a, const TiledArgs p, const WallList wls) {
    using T = typename St<S>::T;
    const int wall = wls.w[blockIdx.z];
    const int ax = wall >> 1, side = wall & 1;
    const int nx = a.n[0], ny = a.n[1], nz = a.n[2];
    const int n0 = ax == 0 ? ny : nx;            // fastest wall-cell coordinate extent
    const int n1 = ax == 2 ? ny : nz;
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int k = blockIdx.y;
    if (j >= (long long)n0 * n1) return;
    const int ja = (int)(j % n0), jb = (int)(j / n0);
    int x, y, z;
    if (ax == 0) { x = side ? nx - 1 : 0; y = ja; z = jb; }
    else if (ax == 1) { x = ja; y = side ? ny - 1 : 0; z = jb; }
    else { x = ja; y = jb; z = side ? nz - 1 : 0; }
    const BandConst b = a.band[k];
    float v;
    if (a.bc[wall] == kBcIsothermal) {
        v = a.iso[wall * a.nb + k];
    } else {
        const int ty = y / p.ty, tz = z / p.tz;
        const int tile = tz * p.nty + ty;
        const int yl = y - ty * p.ty, zl = z - tz * p.tz;
        const int slot = ax == 0 ? zl * p.ty + yl : (ax == 1 ? zl * p.nxt + x : yl * p.nxt + x);
        float s = 0.f;
        for (int jj = 0; jj < p.J; ++jj) {
            const int u = jj * p.ntiles + tile;
            const int p0 = part_begin(p, jj), p1 = part_begin(p, jj + 1);
            if (p0 >= p1) continue;
            const int b0 = p0 / a.nd, b1 = (p1 - 1) / a.nd;
            if (k < b0 || k > b1) continue;
            s += p.PW[((size_t)(p.unit_seg0[u] + k - b0) * p.nwd + p.wslot[wall]) * p.tw + slot];
        }
        v = s * a.inv_den[wall];
    }
    T *out = static_cast<T *>(a.ediff_out) + ((long long)wall * a.nb + k) * a.wc_max + j;
    if constexpr (St<S>::kRef) {
        const uint32_t c = St<S>::enc(fmaf(v, b.inv_scale, -a.TL[((long long)z * ny + y) * nx + x] * a.invTs));
        *reinterpret_cast<unsigned short *>(out) = (unsigned short)c;
    } else {
        *out = v;
    }
}

// Per-plane constants the producer copies into each stage:
// [nu_x, nu_y, nu_z, w/tau, dt/tau, s_k, 1/s_k, iso(-x), iso(+x), wdiff(w=0..5), 0]
// (with 16-bit storage the two x-wall emissions in units of s_k, as the kernel computes in them)
__global__ void k_build_headers(const StepArgs a, float *hdr, int scaled) {
    const int pl = blockIdx.x * blockDim.x + threadIdx.x;
    if (pl >= a.nb * a.nd) return;
    const int k = pl / a.nd, d = pl % a.nd;
    const BandConst b = a.band[k];
    float *h = hdr + (size_t)pl * kHdrFloats;
    h[0] = a.nu[3 * pl];
    h[1] = a.nu[3 * pl + 1];
    h[2] = a.nu[3 * pl + 2];
    h[3] = a.wmom[pl];
    h[4] = b.dtinv;
    h[5] = b.scale;
    h[6] = b.inv_scale;
    h[7] = scaled ? a.iso[0 * a.nb + k] * b.inv_scale : a.iso[0 * a.nb + k];
    h[8] = scaled ? a.iso[1 * a.nb + k] * b.inv_scale : a.iso[1 * a.nb + k];
    for (int w = 0; w < 6; ++w) h[9 + w] = (w < 2 * a.dim && a.bc[w] == kBcDiffuse) ? a.wdiff[w * a.nd + d] : 0.f;
    h[15] = 0.f;
}

// Rows of the thermalizing-wall emission C_k T_w / W (FP32 storage).
__global__ void k_fill_isorows(const StepArgs a, int nx, float *rows) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;  // over 6 * nb * nx
    if (i >= 6 * a.nb * nx) return;
    rows[i] = a.iso[i / nx];
}

// ---- dispatch -------------------------------------------------------------------------------
StepKernel pick(int storage, int lim, int nx, int dim, bool sr) {
    if (storage == kStoreF32) return dim == 2 ? pick_f32_2d(lim, nx) : pick_f32_3d(lim, nx);
    if (storage == kStoreF16) return dim == 2 ? pick_f16_2d(lim, nx, sr) : pick_f16_3d(lim, nx, sr);
    return dim == 2 ? pick_bf16_2d(lim, nx, sr) : pick_bf16_3d(lim, nx, sr);
}

template <class V>
bool upload_vec(V **dst, const std::vector<V> &v, std::string &why) {
    if (cudaMalloc((void **)dst, std::max<size_t>(1, v.size()) * sizeof(V)) != cudaSuccess) {
        cudaGetLastError();
        why = "cudaMalloc failed";
        return false;
    }
    if (!v.empty() && cudaMemcpy(*dst, v.data(), v.size() * sizeof(V), cudaMemcpyHostToDevice) != cudaSuccess) {
        why = "cudaMemcpy failed";
        return false;
    }
    return true;
}

}  // namespace tiled

using namespace tiled;

// ------------------------------------------------------------------------------------------
// host side
// ------------------------------------------------------------------------------------------
bool tiled_plan(int dim, const int n[3], int nb, int nd, int storage, int limiter, bool sr, const int bc[6],
                TiledPlan &plan, std::string &why) {
    plan = TiledPlan();
    if (dim != 2 && dim != 3) {
        why = "the tiled kernel covers 2-D and 3-D grids";
        return false;
    }
    // Row capacity NX of the kernel instance: the smallest of 64, 96, 128 and (2-D) 256 cells that
    // holds the grid's rows, such that a row is a whole number of 16-byte units (its bulk copies
    // start and end on 16-byte boundaries), a whole number of lanes (VL = NX / 32 / warps per row
    // cells a lane), and every warp of the row keeps at least two lanes of cells.
    const int gxn = n[0];
    const int esz = storage == kStoreF32 ? 4 : 2;
    int nx = 0;
    {
        const int caps[4] = {64, 96, 128, 256};
        for (int cap : caps) {
            if (cap == 256 && dim != 2) continue;
            const int w = cap == 256 ? 2 : 1, vl = cap / (32 * w);
            const int lo = w == 2 ? 128 + 2 * vl : 2 * vl;
            if (gxn <= cap && gxn >= lo && gxn % vl == 0 && (gxn * esz) % 16 == 0) {
                nx = cap;
                break;
            }
        }
    }
    if (nx == 0) {
        why = "the tiled kernel needs rows of a multiple of 16 bytes and of the cells a lane holds, at most 256 "
              "(2-D) or 128 (3-D) cells";
        return false;
    }
    const int wpr = nx == 256 ? 2 : 1;
    const int ncw = dim == 2 ? Geo<2, 1>::NCW : Geo<3, 1>::NCW;
    const int TZ = dim == 2 ? Geo<2, 1>::TZ : Geo<3, 1>::TZ;
    const int TY = dim == 3 ? Geo<3, 1>::TY : (wpr == 2 ? Geo<2, 2>::TY : Geo<2, 1>::TY);
    plan.vx = nx / 32;
    plan.dim = dim;
    plan.storage = storage;
    plan.nx = nx;
    // rows per bulk copy of a box slice (BTE_TILED_CHUNK overrides, for tuning runs)
    plan.chunk = 16;
    if (const char *env = std::getenv("BTE_TILED_CHUNK")) {
        const int c = std::atoi(env);
        if (c >= 1 && c <= 1024) plan.chunk = c;
    }
    // rows shorter than the capacity lie at another stride in global memory than in the box:
    // one bulk copy a row
    if (gxn != nx) plan.chunk = 1;
    plan.ty = TY;
    plan.tz = TZ;
    plan.threads = (ncw + kProducerWarps) * 32;
    plan.nty = (n[1] + TY - 1) / TY;
    plan.ntz = dim == 3 ? (n[2] + TZ - 1) / TZ : 1;
    plan.ntiles = plan.nty * plan.ntz;
    plan.tcells = nx * TY * TZ;
    plan.tw = std::max(std::max(TY * TZ, nx * TZ), dim == 3 ? nx * TY : 0);
    const size_t box = (size_t)(TY + 3) * (dim == 3 ? TZ + 3 : 1) * nx * esz;
    const int V = 16 / esz;  // elements in 16 bytes
    const size_t side_bytes = ((size_t)2 * TZ * TY * V + (size_t)2 * TZ * (TY + V)) * esz;
    plan.side_off = (int)((box + 127) / 128 * 128);
    plan.hdr_off = plan.side_off + (int)((side_bytes + 15) / 16 * 16);
    plan.stage_bytes = (int)((plan.hdr_off + kHdrFloats * sizeof(float) + 127) / 128 * 128);
    plan.stage0 = 128;  // 2 ns mbarriers (ns <= 6) and the abort word at byte kAbortOff
    static_assert(kStallOff >= 2 * 6 * 8 && kAbortOff >= kStallOff + 8 && kAbortOff + 4 <= 128,
                  "test barrier and abort word after the stage barriers");
    const size_t budget = 227 * 1024;
    for (int w = 0; w < 2 * dim; ++w)
        if (bc[w] == kBcDiffuse) plan.wslot[w] = plan.nwd++;
    const size_t wall_bytes = (size_t)std::max(1, plan.nwd) * plan.tw * sizeof(float);
    const size_t bt_bytes = (size_t)plan.tcells * sizeof(float);
    const size_t acc_bytes = dim == 3 ? 0 : bt_bytes;  // 3-D consumers keep the moment partials in registers
    // 16-bit storage: the code references of the tile and its two-cell halo, one float per cell
    const size_t rho_bytes = storage == kStoreF32 ? 0 : (size_t)(TY + 4) * (dim == 3 ? TZ + 4 : 1) * nx * sizeof(float);
    plan.ns = 0;
    for (int ns = 6; ns >= 2; --ns)
        if (plan.stage0 + (size_t)ns * plan.stage_bytes + wall_bytes + bt_bytes + acc_bytes + rho_bytes + 128 <= budget) {
            plan.ns = ns;
            break;
        }
    if (plan.ns == 0) {
        why = "tile does not fit in shared memory";
        return false;
    }
    plan.wall_off = (int)(plan.stage0 + (size_t)plan.ns * plan.stage_bytes);
    plan.bt_off = plan.wall_off + (int)((wall_bytes + 127) / 128 * 128);
    plan.acc_off = plan.bt_off + (int)((bt_bytes + 127) / 128 * 128);
    plan.rho_off = plan.acc_off + (int)((acc_bytes + 127) / 128 * 128);
    plan.smem = plan.rho_off + (int)rho_bytes;
    plan.kernel = (void *)pick(storage, limiter, nx, dim, sr && storage != kStoreF32);
    if (!plan.kernel) {
        why = "no kernel instance";
        return false;
    }
    // persistent grid: SMs x resident CTAs
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        why = "no CUDA device";
        return false;
    }
    StepKernel kf = (StepKernel)plan.kernel;
    // The dynamic shared-memory cap is an attribute of the kernel instance, shared by every context
    // that runs it, so it is set to the device's opt-in limit (not to this plan's size, which a
    // later context with a smaller plan would lower below ours).
    int optin = 0;
    cudaFuncAttributes fa;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
        cudaFuncGetAttributes(&fa, kf) != cudaSuccess) {
        cudaGetLastError();
        why = "kernel attributes unavailable";
        return false;
    }
    const int smem_cap = optin - (int)fa.sharedSizeBytes;
    if (plan.smem > smem_cap ||
        cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_cap) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kf, plan.threads, plan.smem) != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        why = "kernel does not fit on an SM";
        return false;
    }
    plan.nctas = sms * per_sm;
    // plane-synchronous schedule: J parts per tile, units dealt round-robin to the CTAs
    const long long npl = (long long)nb * nd;
    if (npl * plan.ntiles > 0x7fffffffLL) {
        why = "too many plane-tiles";
        return false;
    }
    int g = plan.ntiles, hcf = plan.nctas;
    while (g) { const int r = hcf % g; hcf = g; g = r; }
    plan.np = (int)npl;
    plan.J = std::min(plan.nctas / hcf, plan.np);
    plan.U = plan.ntiles * plan.J;
    if (plan.nctas > plan.U) plan.nctas = plan.U;
    // segment rows numbered tile by tile: [U] first row of each unit, then [ntiles + 1] tile starts
    plan.h_unit_seg0.assign(plan.U + plan.ntiles + 1, 0);
    int nsg = 0;
    for (int t = 0; t < plan.ntiles; ++t) {
        plan.h_unit_seg0[plan.U + t] = nsg;
        for (int j = 0; j < plan.J; ++j) {
            const long long p0 = (long long)j * plan.np / plan.J, p1 = (long long)(j + 1) * plan.np / plan.J;
            const int nseg = p1 > p0 ? (int)((p1 - 1) / nd - p0 / nd + 1) : 0;
            plan.h_unit_seg0[j * plan.ntiles + t] = nsg;
            nsg += nseg;
        }
    }
    plan.h_unit_seg0[plan.U + plan.ntiles] = nsg;
    plan.G = nsg;
    plan.valid = 1;
    return true;
}

bool tiled_setup(TiledPlan &plan, const StepArgs &a, std::string &why) {
    if (!upload_vec(&plan.unit_seg0, plan.h_unit_seg0, why)) return false;
    // band of every segment row (the adjoint's per-band sums)
    {
        std::vector<int> sb(std::max(1, plan.G), 0);
        for (int u = 0; u < plan.U; ++u) {
            const int j = u / plan.ntiles;
            const long long p0 = (long long)j * plan.np / plan.J, p1 = (long long)(j + 1) * plan.np / plan.J;
            if (p1 <= p0) continue;
            const int b0 = (int)(p0 / a.nd), b1 = (int)((p1 - 1) / a.nd);
            for (int k = b0; k <= b1; ++k) sb[plan.h_unit_seg0[u] + k - b0] = k;
        }
        if (!upload_vec(&plan.seg_band, sb, why)) return false;
    }
    const size_t npw = std::max<size_t>(1, (size_t)plan.G * plan.nwd * plan.tw);
    if (cudaMalloc((void **)&plan.PW, npw * sizeof(float)) != cudaSuccess ||
        cudaMemset(plan.PW, 0, npw * sizeof(float)) != cudaSuccess ||
        cudaMalloc((void **)&plan.err, sizeof(int)) != cudaSuccess || cudaMemset(plan.err, 0, sizeof(int)) != cudaSuccess ||
        cudaMalloc((void **)&plan.hdr, (size_t)a.nb * a.nd * kHdrFloats * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        why = "cudaMalloc failed";
        return false;
    }
    k_build_headers<<<(a.nb * a.nd + 127) / 128, 128>>>(a, plan.hdr, plan.storage != kStoreF32);
    if (plan.storage == kStoreF32) {
        const int nrow = 6 * a.nb * plan.nx;
        if (cudaMalloc(&plan.isorow, (size_t)nrow * sizeof(float)) != cudaSuccess) {
            cudaGetLastError();
            why = "cudaMalloc failed";
            return false;
        }
        k_fill_isorows<<<(nrow + 255) / 256, 256>>>(a, plan.nx, static_cast<float *>(plan.isorow));
    }
    if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) {
        why = "header build failed";
        return false;
    }
    return true;
}

void tiled_free(TiledPlan &plan) {
    void *ptrs[] = {plan.unit_seg0, plan.seg_band, plan.PW, plan.err, plan.hdr, plan.isorow};
    for (void *q : ptrs)
        if (q) cudaFree(q);
    plan.unit_seg0 = nullptr;
    plan.seg_band = nullptr;
    plan.isorow = nullptr;
    plan.PW = nullptr;
    plan.err = nullptr;
    plan.hdr = nullptr;
}

TiledArgs tiled_device_args(const TiledPlan &plan) {
    TiledArgs t;
    memset(&t, 0, sizeof t);
    t.unit_seg0 = plan.unit_seg0;
    t.tile_seg0 = plan.unit_seg0 + plan.U;
    t.U = plan.U;
    t.J = plan.J;
    t.np = plan.np;
    t.ntiles = plan.ntiles;
    t.PW = plan.PW;
    t.hdr = plan.hdr;
    t.isorow = plan.isorow;
    t.err = plan.err;
    t.tw = plan.tw;
    t.nwd = plan.nwd;
    for (int w = 0; w < 6; ++w) t.wslot[w] = plan.wslot[w];
    t.bt_off = plan.bt_off;
    t.acc_off = plan.acc_off;
    t.rho_off = plan.rho_off;
    t.nty = plan.nty;
    t.ntz = plan.ntz;
    t.ns = plan.ns;
    t.stage0 = plan.stage0;
    t.stage_bytes = plan.stage_bytes;
    t.side_off = plan.side_off;
    t.hdr_off = plan.hdr_off;
    t.ty = plan.ty;
    t.tz = plan.tz;
    t.wall_off = plan.wall_off;
    t.tcells = plan.tcells;
    t.chunk = plan.chunk;
    t.wait_ns = plan.wait_ns;
    t.stall = plan.stall;
    t.nxt = plan.nx;
    return t;
}

cudaError_t launch_step_tiled(const StepArgs &a, const TiledPlan &plan, cudaStream_t s) {
    StepKernel kf = (StepKernel)plan.kernel;
    kf<<<plan.nctas, plan.threads, plan.smem, s>>>(a, tiled_device_args(plan));
    return cudaGetLastError();
}

// Walls whose ghost values the finalize pass writes: diffuse walls, and with 16-bit storage the
// thermalizing y/z walls (x walls use a per-plane constant).
static bool tiled_wall_pass(const TiledPlan &plan, const int bc[6], int w) {
    return bc[w] == kBcDiffuse || (plan.storage != kStoreF32 && bc[w] == kBcIsothermal && (w >> 1) > 0);
}

cudaError_t launch_finalize_tiled(const StepArgs &a, const TiledPlan &plan, int storage, float *TL_out,
                                  cudaStream_t s) {
    const TiledArgs t = tiled_device_args(plan);
    const unsigned nblk = (unsigned)((a.ncell + 255) / 256);
    k_finalize_tiled<<<nblk, 256, 0, s>>>(a, t, TL_out);
    // every wall that needs ghost values in one launch (z: the wall), x covering its cells
    WallList wl;
    int nw = 0;
    long long nwc = 0;
    for (int w = 0; w < 2 * plan.dim; ++w) {
        if (!tiled_wall_pass(plan, a.bc, w)) continue;
        const int ax = w >> 1;
        const long long m = ax == 0 ? (long long)a.n[1] * a.n[2]
                                    : (ax == 1 ? (long long)a.n[0] * a.n[2] : (long long)a.n[0] * a.n[1]);
        nwc = std::max(nwc, m);
        wl.w[nw++] = w;
    }
    if (nw > 0) {
        const dim3 g((unsigned)((nwc + 255) / 256), (unsigned)a.nb, (unsigned)nw);
        if (storage == kStoreF32) k_ediff_tiled<kStoreF32><<<g, 256, 0, s>>>(a, t, wl);
        else if (storage == kStoreF16) k_ediff_tiled<kStoreF16><<<g, 256, 0, s>>>(a, t, wl);
        else k_ediff_tiled<kStoreBF16><<<g, 256, 0, s>>>(a, t, wl);
    }
    return cudaGetLastError();
}

int tiled_finalize_launches(const TiledPlan &plan, const int bc[6]) {
    for (int w = 0; w < 2 * plan.dim; ++w)
        if (tiled_wall_pass(plan, bc, w)) return 2;
    return 1;
}

}  // namespace bte
