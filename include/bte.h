/*
 * bte.h - C ABI of the GB300 explicit discrete-ordinates (DOM) transient step of the
 * non-gray phonon Boltzmann transport equation (BTE) in the energy form of
 * arXiv 2306.14181 (GiftBTE), Sec. 4.
 *
 * The library (libbte_gb300.so) advances, on one GPU, the deviational energy density
 * e[k][d][z][y][x] (band k, direction d, Cartesian cell) with the forward-Euler finite-volume
 * update of Eq. (disretized_transientBTE):
 *
 *   e^{n+1} = e^n - sum_a (dt/dx_a) v_k s_{d,a} (e_{i+1/2} - e_{i-1/2})
 *                 + dt [ (C_k T_L^n / W - e^n) / tau_k + a(t_n) Q_i C_k / (sum_k C_k W) ]
 *
 * with the face value e_ij = e_m + grad(e_m).l taken at the upwind cell m (Sec. 4.1) through
 * a slope limiter, the lattice temperature T_L of Eq. (BTE_get_e0) formed from the new state
 * in the same pass, and the four wall types of Sec. 2.2 (thermalizing, diffusely and
 * specularly reflecting, periodic).  W = sum_d w_d is the discrete total solid angle (4 pi).
 *
 * Conventions for every call:
 *   - Temperatures are offsets from T_ref (K): T_wall, dT0, and the dT / dTL outputs.
 *   - The caller owns every pointer it passes; input arrays are copied or consumed before
 *     the call returns, output arrays are written before it returns.
 *   - Host arrays are plain C arrays; "device" pointers are CUDA device addresses on the
 *     device that was current when bte_create ran.
 *   - Work is issued on options.stream (NULL: the CUDA default stream) in call order.  Calls
 *     that return data to host memory synchronise that stream; the others do not block.
 *   - Nothing throws or aborts across the ABI.  Every call returns a bte_status; on failure
 *     bte_last_error() gives a one-line reason and the context is left unchanged where the
 *     failure was detected before any work was issued.
 *   - A context is not thread safe: use one context per host thread (or serialise calls).
 */
#ifndef BTE_GB300_H
#define BTE_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    BTE_OK = 0,
    BTE_EINVAL = 1,        /* an argument is out of range or inconsistent */
    BTE_ENOMEM = 2,        /* device or host allocation failed */
    BTE_ECUDA = 3,         /* a CUDA runtime call failed (message in bte_last_error) */
    BTE_ESTATE = 4,        /* call not valid in the context's current state */
    BTE_ENONFINITE = 5,    /* a non-finite value was found in the state or an output */
    BTE_ETIMEOUT = 6,      /* a bounded device wait gave up (see bte_set_wait_limit) */
    BTE_EUNSUPPORTED = 7   /* valid request this build does not implement */
} bte_status;

/* Directional discretisation (Sec. 3.2, Eq. directiondis). */
enum {
    BTE_QUAD_GL1D_POLAR = 0, /* 1-D geometries: Gauss-Legendre in mu = cos(theta) on [-1, 1],
                                s = (mu, 0, 0), w = 2 pi w_mu; ntheta = number of nodes */
    BTE_QUAD_OCTANT = 1,     /* ntheta Gauss-Legendre nodes in mu on [0, 1] times nphi nodes in
                                phi on [0, pi/2], w = w_mu w_phi, mirrored into 8 octants:
                                ndirs = 8 ntheta nphi.  Order: octant-major, then mu, then phi;
                                octant bit a set = component a negative */
    BTE_QUAD_EXPLICIT = 2    /* caller-given s[3*ndirs] and w[ndirs] */
};

/* Wall types (Sec. 2.2).  Walls are indexed -x, +x, -y, +y, -z, +z. */
enum {
    BTE_BC_ISOTHERMAL = 0, /* thermalizing wall, Eq. (thermal): emits C_k T_wall / W */
    BTE_BC_DIFFUSE = 1,    /* diffusely reflecting wall, Eq. (diff_bound) */
    BTE_BC_SPECULAR = 2,   /* specularly reflecting wall, Sec. 2.2 (ii) */
    BTE_BC_PERIODIC = 3,   /* periodic pair, Eq. (periodic); both walls of the axis */
    BTE_BC_INTERFACE = 4   /* one side of an interface between two materials, Sec. 2.2 (v): the
                              wall faces a wall of another context (see bte_interface) */
};

/* Storage of e in device memory.  All arithmetic is FP32 in every mode. */
enum {
    BTE_STORE_F32 = 0,
    BTE_STORE_F16 = 1,  /* e = s_k (h + R / T_scale), h binary16, s_k = C_k T_scale / W (see bte_get_state) */
    BTE_STORE_BF16 = 2  /* the same with h bfloat16 */
};

/* Slope limiter L(a, b) of the one-sided differences at the upwind cell; e_face = e_m + L/2.
 * The paper's least-squares gradient on a uniform grid is the unlimited central slope, which
 * forward Euler makes unstable for ballistic bands; a limiter keeps the step bounded. */
enum {
    BTE_LIM_FIRST_ORDER = 0, /* L = 0 */
    BTE_LIM_MINMOD = 1,      /* the smaller of a, b in magnitude if ab > 0, else 0 */
    BTE_LIM_VANALBADA = 2    /* ab(a+b)/(a^2+b^2) if ab > 0, else 0 (default) */
};

/* Rounding of the 16-bit codes the forward step writes.  Round to nearest loses every
 * per-step change below half a code step, so a slowly drifting state stalls; stochastic
 * rounding rounds up with probability equal to the fraction of a code step, unbiased, with
 * the random bits a counter-based hash of (seed, step index, plane k*ndirs+d, cell): the same
 * seed and inputs give bitwise the same run. */
enum { BTE_ROUND_NEAREST = 0, BTE_ROUND_STOCHASTIC = 1 };

/* Which forward kernel to run. */
enum {
    BTE_KERNEL_AUTO = 0,       /* persistent for small 1-D FP32 problems, else tiled where its shape
                                  limits allow, else generic */
    BTE_KERNEL_GENERIC = 1,    /* one thread per (cell, band); any grid shape */
    BTE_KERNEL_TILED = 2,      /* shared-memory tiled kernel; BTE_EUNSUPPORTED if the grid does not fit */
    BTE_KERNEL_PERSISTENT = 3  /* 1-D, FP32 storage, state in one CTA's shared memory for all the steps
                                  of a bte_step call (two block barriers a step, one launch a call);
                                  BTE_EUNSUPPORTED otherwise */
};

typedef struct bte_ctx bte_ctx;

/* Cartesian finite-volume grid (Sec. 4.1).  dim 1: nx cells (ny = nz = 1); dim 2: nx*ny
 * (nz = 1); dim 3: nx*ny*nz.  Cell sizes in metres; every active extent must be >= 2.
 * Axes beyond dim have unit length in volumes and face areas. */
typedef struct {
    int dim;
    int nx, ny, nz;
    double dx, dy, dz;
    double Tref; /* reference temperature (K); reported back, not used in the arithmetic */
} bte_grid;

/* Phonon bands (Sec. 3.1, Eq. banddis): heat capacity C_k (J/m^3/K), group speed |v_k| (m/s),
 * relaxation time tau_k (s), all > 0.  Host arrays of length nbands, copied. */
typedef struct {
    int nbands;
    const double *C;
    const double *vabs;
    const double *tau;
} bte_bands;

/* Directions (Sec. 3.2).  For BTE_QUAD_EXPLICIT, s (3*ndirs, unit vectors or, in 1-D, their
 * x projections) and w (ndirs, > 0) are host arrays, copied; ntheta/nphi are ignored.  Walls
 * of type specular need, for every direction, the one with the normal component negated. */
typedef struct {
    int kind;
    int ntheta;
    int nphi;
    int ndirs;
    const double *s;
    const double *w;
} bte_quadrature;

/* Wall types and thermalizing-wall temperatures (offsets from T_ref, K).
 * dT_jump[a]: temperature difference (K) across the periodic pair of axis a, Sec. 2.2 (iv):
 * the ghost values of the -a wall are the wrapped values plus C_k dT_jump[a] / W and those of
 * the +a wall the wrapped values minus it (every direction, both ghost layers), so that a
 * uniform gradient dT_jump[a] / L_a along +a is represented exactly; dT_jump[a] > 0 means the -a
 * side is the warmer one and heat flows towards +a.  Must be 0 on an axis that is not periodic
 * (BTE_EINVAL otherwise).  A non-zero jump runs the generic kernels (bte_info.kernel says so);
 * BTE_EUNSUPPORTED when options.kernel asks for the tiled or persistent kernel. */
typedef struct {
    int type[6];
    double T_wall[6];
    double dT_jump[3];
} bte_boundaries;

typedef struct {
    double dt;        /* time step (s), > 0 (Sec. 4.1: dt = beta dx_min / v) */
    int storage;      /* BTE_STORE_* */
    int limiter;      /* BTE_LIM_* */
    double T_scale;   /* K; 16-bit storage scale s_k = C_k T_scale / W.  <= 0: 1 K.  The codes hold
                         departures from local equilibrium in units of T_scale: for binary16 pick
                         T_scale near the expected temperature rise (subnormals below 6e-5) */
    int rounding;     /* BTE_ROUND_*; only meaningful for 16-bit storage */
    void *stream;     /* cudaStream_t; NULL = CUDA default stream */
    uint64_t seed;    /* key of the stochastic-rounding hash (BTE_ROUND_STOCHASTIC) */
    int kernel;       /* BTE_KERNEL_* */
} bte_options;

/* Sizes and settings of a context. */
typedef struct {
    int dim, nx, ny, nz;
    int nbands, ndirs;
    long long ncell;        /* nx*ny*nz */
    long long nelem;        /* nbands * ndirs * ncell, the updates per step */
    size_t state_bytes;     /* nelem * element size; the size bte_get_state/bte_set_state take */
    int elem_bytes;         /* 4 (FP32) or 2 (16-bit) */
    int storage, limiter, kernel; /* kernel actually used: BTE_KERNEL_GENERIC or _TILED */
    double dt;
    double W;               /* sum_d w_d */
    long long step;         /* steps taken since bte_init_temperature / bte_set_state */
    size_t device_bytes;    /* device memory held by the context */
    int launches_per_step;  /* kernel launches of one step (bte_step(ctx, 1)); the persistent 1-D
                               kernel launches once per bte_step call, whatever n */
} bte_info;

/* Create a context: validate, build the quadrature, band tables and mirror maps on the host,
 * allocate the device state and set it to equilibrium at dT = 0 (Algorithm 2, "Initial e").
 * On success *out owns device memory until bte_destroy.  Errors: BTE_EINVAL (bad sizes,
 * non-positive band data or dt, a periodic wall without its partner, a specular wall on a
 * quadrature without mirror partners), BTE_EUNSUPPORTED (kernel = TILED on a grid it cannot
 * tile), BTE_ENOMEM, BTE_ECUDA.  The reason of a failed create is returned by
 * bte_last_error(NULL) on the same thread. */
bte_status bte_create(const bte_grid *grid, const bte_bands *bands, const bte_quadrature *quad,
                      const bte_boundaries *walls, const bte_options *opts, bte_ctx **out);

/* Release every resource of the context (NULL is ignored).  Synchronises its stream first. */
void bte_destroy(bte_ctx *ctx);

/* One-line reason of the last failure on ctx (NULL: of the last failed bte_create on this
 * thread).  The string stays valid until the next call on the same context. */
const char *bte_last_error(const bte_ctx *ctx);

/* Equilibrium start (Algorithm 2; Sec. 4.2): e_{k,d,i} = C_k dT0_i / W for every band and
 * direction, T_L = dT0.  dT0: host array of ncell doubles (cell order x fastest), or NULL for
 * dT0 = 0.  Resets the step counter to 0. */
bte_status bte_init_temperature(bte_ctx *ctx, const double *dT0);

/* Volumetric heat source (Eq. BTE_origin, Q-dot): Q_i in W/m^3 per cell (ncell floats, host
 * or device per on_device), split over bands in proportion to C_k and uniformly over
 * directions.  amp[n] (host, n_amp doubles) scales the source at step n (t_n = n dt); steps
 * n >= n_amp get amplitude 0.  amp = NULL means amplitude 1 at every step.  Q = NULL removes
 * the source.  A host Q is checked (BTE_EINVAL on a non-finite value, nothing changed) and
 * copied into the context's pinned staging before the call returns, so the caller may reuse
 * or free it at once; the upload itself is stream ordered and the call does not wait for
 * steps already queued.  A device Q is copied in stream order and must stay valid until then. */
bte_status bte_set_source(bte_ctx *ctx, const float *Q, int on_device, const double *amp, int n_amp);

/* Advance n >= 0 steps of Eq. (disretized_transientBTE).  Each step is one fused pass of the
 * forward kernel over all (band, direction, cell) (flux, relaxation, source, walls, moment
 * partials), then one short pass that finishes T_L and the diffuse-wall values.  Stream
 * ordered, non-blocking.  A call of 64 steps or more replays a captured CUDA graph of 32 steps
 * (on a private stream ordered after and before the context's stream) when the steps differ only
 * in the ping-pong buffers: no source amplitudes, no stochastic rounding, no tracing; the result
 * is bitwise that of single steps. */
bte_status bte_step(bte_ctx *ctx, int n);

/* The lattice temperature the last step formed (FP32 on the device), as doubles into dTL
 * (host, ncell).  Synchronises (the copy goes through the context's pinned staging). */
bte_status bte_lattice_temperature(bte_ctx *ctx, double *dTL);

/* FP64 moments of the current state (Eq. getTQ and Eq. BTE_get_e0): dT (ncell), dTL (ncell)
 * and q (3*ncell, component-major: qx for all cells, then qy, then qz; W/m^2).  Host arrays;
 * any may be NULL.  Synchronises.  BTE_ENONFINITE if the state holds a non-finite value. */
bte_status bte_moments(bte_ctx *ctx, double *dT, double *dTL, double *q);

/* FP64 global energy-balance reductions of the current state: E_total = V sum_i sum_k sum_d
 * w_d e (J per unit length/area for dim < 3) and the outward heat flow through each wall,
 * wall_flux[6] = S_wall sum sum sum w_d v_k (s_d.n) e_face with e_face the wall-face value
 * the step uses.  One step then obeys E^{n+1} - E^n = dt (V a_n sum_i Q_i - sum wall_flux^n).
 * Host outputs; synchronises.  BTE_ENONFINITE on a non-finite state. */
bte_status bte_energy(bte_ctx *ctx, double *E_total, double wall_flux[6]);

/* The reductions of bte_energy without any device allocation.  The paper has no counterpart:
 * this entry point exists for callers that must not allocate device memory after set-up, for
 * example a host application that hands all device memory to its own pool, or code that runs
 * where a cudaMalloc would block or is not permitted.  bte_energy allocates its diagnostic
 * buffers on first use; this variant instead keeps its block partials, its seven results and a
 * non-finite flag in one fixed array of the library (2048 partial slots per reduction, about
 * 112 KB of device memory, held by every device that loads the library until the process
 * exits).  It calls no cudaMalloc, cudaFree or allocating library routine.
 *   - Inputs and outputs as for bte_energy (the context's current state; host E_total and
 *     wall_flux[6], either may be NULL).  Results equal bte_energy's up to FP64 rounding order.
 *   - Limit: each reduction - the cells, and each wall's (wall cells x bands) - may have at most
 *     2048 * 4096 = 8,388,608 items; larger grids return BTE_EINVAL and nothing is launched.
 *   - The first call made on a device looks up the array's device address (once per device,
 *     with that device current); make that first call before any stream capture.
 *   - Every call overwrites what it reads and clears the flag first, so nothing carries over
 *     between calls.  All calls in the process share the one array: calls that overlap on the
 *     GPU (other streams, contexts or host threads) race and must be serialised by the caller.
 * Synchronises the context's stream.  BTE_ENONFINITE on a non-finite state. */
bte_status bte_energy_noalloc(bte_ctx *ctx, double *E_total, double wall_flux[6]);

/* Copy the stored state out / in, in its storage format, layout e[k][d][z][y][x].  FP32
 * storage holds e.  16-bit storage holds codes h with
 *     e_{k,d,i} = s_k (h_{k,d,i} + R_i / T_scale),   s_k = C_k T_scale / W,
 * against a per-cell reference temperature R (the T_L the step that wrote the state relaxed
 * towards, Eq. BTE_get_e0), so h is the departure from the band's local equilibrium.
 * ref (ncell floats, K; same memory space as the state; may be NULL) receives R from
 * bte_get_state and supplies it to bte_set_state (NULL there: R = 0, i.e. e = s_k h).  FP32
 * storage ignores ref on input and returns zeros.  bytes must equal bte_info.state_bytes.
 * bte_set_state recomputes T_L and the wall ghost values from the new state and resets the
 * step counter to 0 unless keep_step is non-zero; BTE_EINVAL on a non-finite host ref. */
bte_status bte_get_state(bte_ctx *ctx, void *dst, size_t bytes, float *ref, int on_device);
bte_status bte_set_state(bte_ctx *ctx, const void *src, size_t bytes, const float *ref, int on_device, int keep_step);

/* The decoded state e (FP32, nbands*ndirs*ncell values, layout as above) into dst (host, or
 * device memory of the context's device when on_device is non-zero).  A host dst uses a
 * temporary device buffer of the same size; the context's stream is synchronised. */
bte_status bte_get_values(bte_ctx *ctx, float *dst, int on_device);

/* Residuals of the transient solver's loop condition (Sec. 4.1, Algorithm 2).  bte_residuals
 * runs nsteps >= 1 steps and returns, for the last two states n and n+1 of the call,
 *   eps_T = sqrt(sum_i (T_i^n - T_i^{n+1})^2 / N) / T_max,
 *   eps_q = sqrt(sum_i (|q|_i^n - |q|_i^{n+1})^2 / N) / |q|_max,
 * with T and q of Eq. (getTQ) formed in FP64 on the device, N the number of cells,
 * T_max = max_i (T_ref + T_i^{n+1}) (absolute temperature, as the paper's solver works in) and
 * |q|_max = max_i |q_i^{n+1}|; a ratio whose numerator is 0 is 0.  Outputs are host doubles (may
 * be NULL); the stream is synchronised.  Diagnostic buffers are allocated on first use.
 * bte_run_steady repeats bte_residuals(check_every) until eps_T < tol_T and eps_q < tol_q, or
 * until max_steps steps have run (the last stretch may be shorter); it returns the steps it ran
 * and the last residuals.  Both report BTE_ENONFINITE for a non-finite state and BTE_ETIMEOUT
 * as bte_synchronize does. */
bte_status bte_residuals(bte_ctx *ctx, int nsteps, double *eps_T, double *eps_q);
bte_status bte_run_steady(bte_ctx *ctx, long long max_steps, int check_every, double tol_T, double tol_q,
                          long long *steps_done, double *eps_T, double *eps_q);

/* Discrete adjoint (the exact transpose of the step; the paper has no adjoint) of
 *     J = sum_i probe_i T_L,i   after nsteps steps from the context's current state,
 * T_L of Eq. (BTE_get_e0).  Runs the nsteps forward steps (the context ends in the state
 * bte_step(ctx, nsteps) leaves), then the adjoint steps backward in time:
 *     lambda^N = dT_L/de^T probe,  lambda^n = J_n^T lambda^{n+1}
 * with J_n the step's Jacobian at e^n (limited upwind flux with the limiter's Jacobian,
 * transposed wall ghosts, relaxation and the T_L coupling).  States are recomputed from
 * checkpoints taken every ckpt_every steps (0: about sqrt(nsteps)); within a segment every
 * state is kept when it fits in half the free device memory, else every ceil(sqrt)-th and
 * the rest recomputed again.  Outputs (host, each may be NULL): J; dJ_dQ[ncell] =
 * dJ/dQ_i (K m^3/W per cell of the source field Q of bte_set_source, Q taken as 0 when none
 * is set); dJ_dlogtau[nbands] = dJ/d(log tau_k).  Temporary device memory is allocated and
 * freed inside the call; BTE_ENOMEM when it does not fit.  probe: host, ncell values. */
bte_status bte_adjoint(bte_ctx *ctx, int nsteps, int ckpt_every, const double *probe, double *J, double *dJ_dQ,
                       double *dJ_dlogtau);

/* With tracing on (bte_profile), the last bte_adjoint's device time of its adjoint steps
 * (transposed step plus its reductions, adj_steps of them) and of its forward steps
 * (the first sweep and the recomputations, fwd_steps of them).  Any pointer may be NULL. */
bte_status bte_adjoint_profile_read(bte_ctx *ctx, double *adj_ms, long long *adj_steps, double *fwd_ms,
                                    long long *fwd_steps);

/* Sizes and settings; the quadrature the context built (s: 3*ndirs, w: ndirs, host). */
bte_status bte_get_info(const bte_ctx *ctx, bte_info *info);
bte_status bte_get_quadrature(const bte_ctx *ctx, double *s, double *w);

/* Wait for all work issued on the context's stream.  Returns BTE_ETIMEOUT (once) when a
 * bounded device wait of a step issued since the last such report gave up. */
bte_status bte_synchronize(bte_ctx *ctx);

/* Time limit of the bounded waits in the tiled forward kernel (a control of this library; the
 * paper has no counterpart).  Each warp of that kernel waits on shared-memory barriers for its
 * data (consumers) or for a free stage (producer); a wait that lasts longer than limit_ns
 * nanoseconds gives up, the CTA stops its arithmetic but finishes its schedule, every bulk copy
 * it issued is waited for (2 s at most) before it exits, and the launch ends.  That step's
 * output is invalid: the next call that synchronises the stream (bte_synchronize, or a call
 * returning data to the host) returns BTE_ETIMEOUT once and clears the flag, and the context
 * stays usable (bte_set_state or bte_init_temperature gives a valid state again).
 * limit_ns <= 0 restores the default of 2 s.  Takes effect at the next bte_step; other kernels
 * hold no such waits.
 * stall_test (failure-detection test, normally 0): 1 makes every consumer warp's first wait of
 * the next tiled forward launch wait on a barrier that nothing completes, 2 does the same for
 * the producer warp (3: both); that wait gives up after limit_ns and the launch ends as above.
 * It applies to one launch only and is then cleared.  BTE_EINVAL for stall_test outside 0..3. */
bte_status bte_set_wait_limit(bte_ctx *ctx, long long limit_ns, int stall_test);

/* Steady state by the implicit discrete-ordinates method with the sequential iterative scheme
 * (Sec. 3.3-3.5, Eq. disretized_BTE in delta form).  One iteration forms the steady equation's
 * right-hand side R of the current state with the forward step's own faces (second order,
 * limited), walls and source (at the current step's amplitude), then solves for every band k and
 * direction d the first-order upwind system of the increment
 *   (1/tau_k + sum_a v_k |s_a| / h_a) De_i - sum_a (v_k |s_a| / h_a) De_{upwind neighbour along a} = R_i
 * by one sweep from the upwind corner (the upwind De across a wall, periodic pairs included, is
 * 0: the boundary values move at the next iteration), sets e = e + De, and forms T_L and the
 * diffuse-wall values of the new state.  A fixed point solves the steady discrete equation of
 * bte_step exactly.  bte_sis_iterate runs n >= 0 iterations (stream ordered, non-blocking; the
 * step counter is not advanced).  FP32 storage only (BTE_EUNSUPPORTED otherwise); BTE_ESTATE on
 * a context coupled at an interface. */
bte_status bte_sis_iterate(bte_ctx *ctx, int n);

/* Iterative scheme of bte_sis_iterate and bte_run_steady_implicit (Sec. 3.5). */
enum {
    BTE_SCHEME_SEQUENTIAL = 0, /* the lattice temperature of each sweep is that of the state (default) */
    BTE_SCHEME_SYNTHETIC = 1   /* after each sweep the lattice temperature is corrected by the macroscopic
                                  (diffusion-type) equation of Eq. disretized_macro: with the scheme's own face
                                  fluxes for q its right-hand side is k_bulk L T_L(e) - r(e), so the next sweep
                                  relaxes towards T_L(e) + dT with k_bulk L dT = -r, r_i = sum_k sum_d w_d R the
                                  energy residual of the new state, k_bulk = sum_k C_k v_k^2 tau_k / 3, L the cell
                                  Laplacian (thermalizing walls hold the temperature, reflecting walls pass no
                                  heat, periodic pairs wrap; the mean-free solution when no wall is thermalizing),
                                  solved in FP64 (1-D with a thermalizing wall: the Thomas algorithm; else
                                  conjugate gradients to a relative residual of 1e-8).  Its fixed point is the
                                  sequential scheme's; it converges in far fewer iterations near the diffusive
                                  limit.  An iteration costs a second forward step and the solve */
};

/* Select the scheme of the steady implicit iterations (BTE_EINVAL for another value).  After a
 * synthetic iteration bte_lattice_temperature returns the corrected lattice temperature the next
 * sweep uses; bte_moments' dTL is always that of the state, and bte_step, bte_adjoint and a
 * sequential iteration that follow start from the state's own T_L again. */
bte_status bte_set_steady_scheme(bte_ctx *ctx, int scheme);

/* Iterate until the loop condition of Sec. 3.5 holds between consecutive iterates, eps_T <
 * tol_T and eps_q < tol_q (as bte_residuals defines them), checked every check_every iterations,
 * or max_iters iterations have run.  Outputs (any may be NULL): the iterations run and the last
 * eps_T, eps_q.  Synchronises at every check. */
bte_status bte_run_steady_implicit(bte_ctx *ctx, long long max_iters, int check_every, double tol_T, double tol_q,
                                   long long *iters, double *eps_T, double *eps_q);

/* Interface between two materials (Sec. 2.2 (v), diffuse mismatch).  Wall wall_a of ctx_a (the
 * material-A side) and wall wall_b of ctx_b (material B) must both have been created as
 * BTE_BC_INTERFACE, on the same axis and opposite sides (A's +x against B's -x, say), with the
 * same cell counts along the other two axes (wall cells correspond one to one, same coordinates
 * across) and the same number of bands.  beta_ab[k] (host, nbands doubles in [0, 1]) is the
 * probability that a band-k phonon reaching the interface from A is transmitted into B,
 * beta_ba[k] the same from B into A; the rest is reflected diffusely.  At every interface cell
 * the incoming value of band k (every direction entering the material) is
 *   A: beta_ba S_B + (1 - beta_ab) S_A,     B: beta_ab S_A + (1 - beta_ba) S_B,
 * S_X being what a diffuse wall (Eq. diff_bound) would return on side X: the sum of w_d |s_d.n| e
 * over X's directions reaching the interface over the sum of w_d |s_d.n| over the others.  A
 * uniform temperature is stationary when beta_ba C_B = beta_ab C_A band by band (detailed
 * balance); with equal group speeds the heat that leaves one side enters the other.
 * Both contexts need FP32 storage (their interface walls are refused at bte_create otherwise), a
 * context has at most one interface wall, and ctx_a != ctx_b.  The pair then advances only
 * through bte_step_pair: bte_step, bte_residuals, bte_run_steady, bte_sis_iterate,
 * bte_run_steady_implicit and bte_adjoint on either context return BTE_ESTATE.  Before the
 * coupling (and after the partner's destruction) an interface wall is a diffuse wall.  bte_init_temperature and bte_set_state of either context keep the
 * coupling (the interface values are formed again from both current states).  bte_energy's flow
 * through the interface wall is the heat crossing the interface, outward from that side.  The
 * coupling holds until either context is destroyed; a context that is destroyed leaves its
 * partner uncoupled (its interface wall then behaves as a diffuse wall of Eq. diff_bound).
 * Stream ordered with respect to both contexts' streams.  BTE_EINVAL on any mismatch. */
bte_status bte_interface(bte_ctx *ctx_a, int wall_a, bte_ctx *ctx_b, int wall_b, const double *beta_ab,
                         const double *beta_ba);

/* Advance both contexts of an interface n >= 0 steps together: per step, one forward step of
 * each (as bte_step, on each context's own stream), then one short kernel that forms both
 * sides' interface values of the new states.  BTE_ESTATE unless ctx_a and ctx_b are coupled
 * with each other.  Non-blocking. */
bte_status bte_step_pair(bte_ctx *ctx_a, bte_ctx *ctx_b, int n);

/* Kernel tracing with CUDA events on the context's stream.  bte_profile(ctx, 1) clears the
 * counters and starts recording an event pair around every forward-step launch and every
 * finalize launch of bte_step; bte_profile(ctx, 0) stops.  bte_profile_read synchronises and
 * returns the summed device time (ms) and the launch counts since the last start.  Any output
 * pointer may be NULL. */
bte_status bte_profile(bte_ctx *ctx, int enable);
bte_status bte_profile_read(bte_ctx *ctx, double *fwd_ms, long long *fwd_launches, double *fin_ms,
                            long long *fin_launches);

#ifdef __cplusplus
}
#endif

#endif /* BTE_GB300_H */
