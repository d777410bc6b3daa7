/*
 * FP64 oracle for the explicit discrete-ordinates (DOM) transient step of the
 * non-gray phonon BTE (arXiv 2306.14181, Sec. 4).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is a plain, slow, deliberately unoptimised
 * restatement of the paper's equations.  It is loaded by the test-suite, by the
 * smoke check and by the benchmark's CPU-baseline leg; the product library never
 * links, loads or calls it, and it shares no code, header or table with it.
 *
 * Notation (paper Sec. 3.1-3.3, Sec. 4.1):
 *   k  band index (paper: lambda), d  direction index (paper: alpha),
 *   i  cell index, i = (z*ny + y)*nx + x;  state e[k][d][i] (deviational energy
 *   density per unit solid angle, relative to T_ref).
 *   C_k, v_k = |v_k|, tau_k  band heat capacity, group speed and relaxation time.
 *   s_d, w_d  direction unit vector and weight;  W = sum_d w_d  (= 4 pi).
 *
 * Readings of the paper taken here (each one is listed in the design notes):
 *   - Eq. (disretized_transientBTE): the relaxation and source terms are not
 *     multiplied by V_i; on a Cartesian cell the flux sum over faces divided by
 *     V_i becomes (dt/dx_a) v s_a (e_{i+1/2} - e_{i-1/2}) per axis a.
 *   - Eq. (BTE_get_e0): T_L = sum_k sum_d w_d e/tau_k / sum_k C_k/tau_k (no 1/4pi),
 *     e0_k = C_k T_L / W with W the discrete total weight.
 *   - The face value e_ij = e_m + grad(e_m).l (Sec. 4.1) is evaluated with a slope
 *     limiter L(a, b) of the two one-sided differences at the upwind cell m:
 *     e_face = e_m + L/2.  FIRST_ORDER: L = 0; MINMOD; VANALBADA: ab(a+b)/(a^2+b^2).
 *     With L = (a+b)/2 this is the unlimited central (least-squares) gradient.
 *   - Boundaries (Sec. 2.2) are imposed through two ghost layers per wall.
 *   - The volumetric source is split over bands and directions in proportion to
 *     the heat capacity and uniformly in angle: Qdot_{k,d,i} = a(t_n) Q_i C_k/(sum C W).
 *   - A periodic pair may carry a temperature difference dT (Sec. 2.2 (iv)): the
 *     ghosts of the -a wall hold the wrapped values plus C_k dT/W, those of the +a
 *     wall the wrapped values minus C_k dT/W (every direction and both ghost layers:
 *     the ghost region is the periodic image of the domain shifted by the jump, so a
 *     uniform gradient is represented exactly).  dT > 0: the -a side is warmer.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_BC_ISOTHERMAL 0
#define ORC_BC_DIFFUSE 1
#define ORC_BC_SPECULAR 2
#define ORC_BC_PERIODIC 3

#define ORC_LIM_FIRST_ORDER 0
#define ORC_LIM_MINMOD 1
#define ORC_LIM_VANALBADA 2

typedef struct {
    int dim, nx, ny, nz;
    double dx, dy, dz;
    int nb, nd;
    const double *C, *v, *tau; /* [nb] */
    const double *s;           /* [nd][3] */
    const double *w;           /* [nd] */
    const int *mirror;         /* [3][nd]: direction with component a negated */
    int bc[6];                 /* walls -x,+x,-y,+y,-z,+z */
    double Tw[6];              /* isothermal wall temperature minus T_ref (K) */
    double dt;
    int limiter;
    double jump[3];            /* temperature difference across each periodic pair (K), Sec. 2.2 (iv) */
} orc_problem;

/* ------------------------------------------------------------------------- */
/* small helpers                                                              */
/* ------------------------------------------------------------------------- */

static long ncell_of(const orc_problem *P) { return (long)P->nx * P->ny * P->nz; }

static int extent(const orc_problem *P, int a) { return a == 0 ? P->nx : (a == 1 ? P->ny : P->nz); }

static double spacing(const orc_problem *P, int a) { return a == 0 ? P->dx : (a == 1 ? P->dy : P->dz); }

/* Cell volume and wall face areas.  Axes that are not active (dim < 3) have unit length. */
static double length_of(const orc_problem *P, int a) { return a < P->dim ? spacing(P, a) : 1.0; }

static double cell_volume(const orc_problem *P) { return length_of(P, 0) * length_of(P, 1) * length_of(P, 2); }

static long cidx(const orc_problem *P, const int c[3]) { return ((long)c[2] * P->ny + c[1]) * P->nx + c[0]; }

static double total_weight(const orc_problem *P) {
    double W = 0.0;
    for (int d = 0; d < P->nd; ++d) W += P->w[d];
    return W;
}

static double sum_C(const orc_problem *P) {
    double S = 0.0;
    for (int k = 0; k < P->nb; ++k) S += P->C[k];
    return S;
}

/* D = sum_k C_k / tau_k, the denominator of T_L in Eq. (BTE_get_e0). */
static double sum_C_over_tau(const orc_problem *P) {
    double D = 0.0;
    for (int k = 0; k < P->nb; ++k) D += P->C[k] / P->tau[k];
    return D;
}

#define EIDX(P, k, d, i) ((((long)(k) * (P)->nd + (d)) * ncell_of(P)) + (i))

/* Offset of a periodic ghost of band k on the side `side` of axis a, Sec. 2.2 (iv):
 * e(r_B1) = e(r_B2) + C dT / 4 pi with 4 pi -> W; B1 = the -a wall. */
static double periodic_jump(const orc_problem *P, int k, int a, int side) {
    const double off = P->C[k] * P->jump[a] / total_weight(P);
    return side == 0 ? off : -off;
}

/* Slope limiter of the two one-sided differences a (upwind side) and b (downwind side). */
static double limiter(int kind, double a, double b) {
    if (kind == ORC_LIM_FIRST_ORDER) return 0.0;
    if (a * b <= 0.0) return 0.0;
    if (kind == ORC_LIM_MINMOD) return fabs(a) < fabs(b) ? a : b;
    return a * b * (a + b) / (a * a + b * b); /* van Albada */
}

/* ------------------------------------------------------------------------- */
/* Lattice temperature, Eq. (BTE_get_e0):                                     */
/*   T_L,i = sum_k sum_d w_d e_{k,d,i} / tau_k  /  sum_k C_k / tau_k          */
/* ------------------------------------------------------------------------- */
void orc_lattice_temperature(const orc_problem *P, const double *e, double *TL) {
    const long nc = ncell_of(P);
    const double D = sum_C_over_tau(P);
    #pragma omp parallel for schedule(static)
    for (long i = 0; i < nc; ++i) {
        double acc = 0.0;
        for (int k = 0; k < P->nb; ++k) {
            double sk = 0.0;
            for (int d = 0; d < P->nd; ++d) sk += P->w[d] * e[EIDX(P, k, d, i)];
            acc += sk / P->tau[k];
        }
        TL[i] = acc / D;
    }
}

/* Local temperature and heat flux, Eq. (getTQ):
 *   T_i = sum_d sum_k w_d e / sum_k C_k,   q_i = sum_d sum_k w_d v_k s_d e.            */
void orc_moments(const orc_problem *P, const double *e, double *T, double *TL, double *q) {
    const long nc = ncell_of(P);
    const double SC = sum_C(P);
    if (TL) orc_lattice_temperature(P, e, TL);
    #pragma omp parallel for schedule(static)
    for (long i = 0; i < nc; ++i) {
        double et = 0.0, qx = 0.0, qy = 0.0, qz = 0.0;
        for (int k = 0; k < P->nb; ++k)
            for (int d = 0; d < P->nd; ++d) {
                const double ed = e[EIDX(P, k, d, i)];
                et += P->w[d] * ed;
                qx += P->w[d] * P->v[k] * P->s[3 * d + 0] * ed;
                qy += P->w[d] * P->v[k] * P->s[3 * d + 1] * ed;
                qz += P->w[d] * P->v[k] * P->s[3 * d + 2] * ed;
            }
        if (T) T[i] = et / SC;
        if (q) { q[i] = qx; q[nc + i] = qy; q[2 * nc + i] = qz; }
    }
}

/* ------------------------------------------------------------------------- */
/* Diffusely reflecting wall, Eq. (diff_bound), with the discrete normaliser: */
/*   e_in = sum_{s.n>0} w (s.n) e(s)  /  sum_{s.n<0} w |s.n|                  */
/* evaluated at the wall-adjacent cell of every wall of type DIFFUSE.         */
/* ediff layout: [wall][k][cell]  (only wall-adjacent cells are filled).      */
/* ------------------------------------------------------------------------- */
static void diffuse_wall_values(const orc_problem *P, const double *e, double *ediff) {
    const long nc = ncell_of(P);
    for (int a = 0; a < P->dim; ++a)
        for (int side = 0; side < 2; ++side) {
            const int wall = 2 * a + side;
            if (P->bc[wall] != ORC_BC_DIFFUSE) continue;
            const double nsign = side == 0 ? -1.0 : 1.0; /* outward normal = nsign * unit vector a */
            double den = 0.0;
            for (int d = 0; d < P->nd; ++d) {
                const double sn = nsign * P->s[3 * d + a];
                if (sn < 0.0) den += P->w[d] * (-sn);
            }
            const int n = extent(P, a);
            for (int z = 0; z < P->nz; ++z)
                for (int y = 0; y < P->ny; ++y)
                    for (int x = 0; x < P->nx; ++x) {
                        int c[3] = {x, y, z};
                        if (c[a] != (side == 0 ? 0 : n - 1)) continue;
                        const long i = cidx(P, c);
                        for (int k = 0; k < P->nb; ++k) {
                            double num = 0.0;
                            for (int d = 0; d < P->nd; ++d) {
                                const double sn = nsign * P->s[3 * d + a];
                                if (sn > 0.0) num += P->w[d] * sn * e[EIDX(P, k, d, i)];
                            }
                            ediff[((long)wall * P->nb + k) * nc + i] = num / den;
                        }
                    }
        }
}

/* ------------------------------------------------------------------------- */
/* Value of field (k,d) at integer position p along axis a through cell c.    */
/* Positions -2,-1 and n,n+1 are ghosts; the boundary conditions of Sec. 2.2  */
/* fill them:                                                                 */
/*   PERIODIC   (Eq. periodic)   wrap around the axis;                        */
/*   ISOTHERMAL (Eq. thermal)    incoming: C_k T_w / W;  outgoing: wall cell; */
/*   DIFFUSE    (Eq. diff_bound) incoming: e_diff;       outgoing: wall cell; */
/*   SPECULAR   (Sec. 2.2 (ii))  mirrored direction at the mirrored cell, so  */
/*              the wall behaves exactly like the mirror image of the domain. */
/* "Incoming" means s.n < 0 with n the outward normal of the wall.            */
/* ------------------------------------------------------------------------- */
static double ext_value(const orc_problem *P, const double *e, const double *ediff, int k, int d, int a,
                        const int c[3], int p) {
    const int n = extent(P, a);
    int cc[3] = {c[0], c[1], c[2]};
    if (p >= 0 && p < n) {
        cc[a] = p;
        return e[EIDX(P, k, d, cidx(P, cc))];
    }
    const int side = p < 0 ? 0 : 1;
    const int layer = p < 0 ? -p : p - n + 1; /* 1 = next to the wall, 2 = second ghost */
    const int wall = 2 * a + side;
    const double sa = P->s[3 * d + a];
    const int incoming = side == 0 ? (sa > 0.0) : (sa < 0.0);
    const int wallpos = side == 0 ? 0 : n - 1;
    switch (P->bc[wall]) {
    case ORC_BC_PERIODIC:
        cc[a] = ((p % n) + n) % n;
        return e[EIDX(P, k, d, cidx(P, cc))] + periodic_jump(P, k, a, side);
    case ORC_BC_ISOTHERMAL:
        if (incoming) return P->C[k] * P->Tw[wall] / total_weight(P);
        cc[a] = wallpos;
        return e[EIDX(P, k, d, cidx(P, cc))];
    case ORC_BC_DIFFUSE:
        cc[a] = wallpos;
        if (incoming) return ediff[((long)wall * P->nb + k) * ncell_of(P) + cidx(P, cc)];
        return e[EIDX(P, k, d, cidx(P, cc))];
    case ORC_BC_SPECULAR:
    default:
        cc[a] = side == 0 ? layer - 1 : n - layer;
        return e[EIDX(P, k, P->mirror[a * P->nd + d], cidx(P, cc))];
    }
}

/* Face value e_ij = e_m + grad(e_m).l_{m,ij} (Sec. 4.1) at the face between positions
 * p and p+1 along axis a, m being the upwind cell for the sign of s_a.                 */
static double face_value(const orc_problem *P, const double *e, const double *ediff, int k, int d, int a,
                         const int c[3], int p) {
    const double sa = P->s[3 * d + a];
    if (sa > 0.0) {
        const double um = ext_value(P, e, ediff, k, d, a, c, p);
        const double ul = ext_value(P, e, ediff, k, d, a, c, p - 1);
        const double ur = ext_value(P, e, ediff, k, d, a, c, p + 1);
        return um + 0.5 * limiter(P->limiter, um - ul, ur - um);
    } else {
        const double um = ext_value(P, e, ediff, k, d, a, c, p + 1);
        const double ul = ext_value(P, e, ediff, k, d, a, c, p + 2);
        const double ur = ext_value(P, e, ediff, k, d, a, c, p);
        return um + 0.5 * limiter(P->limiter, um - ul, ur - um);
    }
}

/* One element of Eq. (disretized_transientBTE):
 *   e^{n+1} = e^n - sum_a (dt/dx_a) v_k s_a (e_{i+1/2} - e_{i-1/2})
 *             + dt [ (C_k T_L/W - e^n)/tau_k + amp Q_i C_k/(sum C W) ]                  */
static double step_element(const orc_problem *P, const double *e, const double *ediff, double TLi,
                           const float *Q, double amp, double W, double SC, int k, int d, const int c[3]) {
    const long i = cidx(P, c);
    const double en = e[EIDX(P, k, d, i)];
    double div = 0.0;
    for (int a = 0; a < P->dim; ++a) {
        const double sa = P->s[3 * d + a];
        if (sa == 0.0) continue;
        const double nu = P->dt * P->v[k] * sa / spacing(P, a);
        const double fr = face_value(P, e, ediff, k, d, a, c, c[a]);     /* face i+1/2 */
        const double fl = face_value(P, e, ediff, k, d, a, c, c[a] - 1); /* face i-1/2 */
        div += nu * (fr - fl);
    }
    const double e0 = P->C[k] * TLi / W;
    const double src = Q ? amp * (double)Q[i] * P->C[k] / (SC * W) : 0.0;
    return en - div + P->dt * ((e0 - en) / P->tau[k] + src);
}

/* ------------------------------------------------------------------------- */
/* One forward-Euler step, e_in (time n) -> e_out (time n+1), Algorithm 2.    */
/* T_L^n and the diffuse-wall values are formed from e^n first.              */
/* Q may be NULL (no source).                                                  */
/* ------------------------------------------------------------------------- */
static void step_with(const orc_problem *P, const double *e_in, const double *ediff, double *e_out, const float *Q,
                      double amp) {
    const long nc = ncell_of(P);
    const double W = total_weight(P), SC = sum_C(P);
    double *TL = (double *)malloc(sizeof(double) * nc);
    orc_lattice_temperature(P, e_in, TL);
    const long nplanes = (long)P->nb * P->nd;
    #pragma omp parallel for schedule(static)
    for (long pl = 0; pl < nplanes; ++pl) {
        const int k = (int)(pl / P->nd), d = (int)(pl % P->nd);
        for (int z = 0; z < P->nz; ++z)
            for (int y = 0; y < P->ny; ++y)
                for (int x = 0; x < P->nx; ++x) {
                    const int c[3] = {x, y, z};
                    e_out[EIDX(P, k, d, cidx(P, c))] = step_element(P, e_in, ediff, TL[cidx(P, c)], Q, amp, W, SC, k, d, c);
                }
    }
    free(TL);
}

void orc_step(const orc_problem *P, const double *e_in, double *e_out, const float *Q, double amp) {
    double *ediff = (double *)calloc((size_t)6 * P->nb * ncell_of(P), sizeof(double));
    diffuse_wall_values(P, e_in, ediff);
    step_with(P, e_in, ediff, e_out, Q, amp);
    free(ediff);
}

/* nsteps forward steps in place; amp[n] is the source amplitude at step n (NULL: 1). */
void orc_run(const orc_problem *P, double *e, const float *Q, const double *amp, int namp, long n0, int nsteps) {
    const long total = (long)P->nb * P->nd * ncell_of(P);
    double *tmp = (double *)malloc(sizeof(double) * total);
    for (int s = 0; s < nsteps; ++s) {
        const long n = n0 + s;
        const double a = amp ? (n < namp ? amp[n] : 0.0) : 1.0;
        orc_step(P, e, tmp, Q, a);
        memcpy(e, tmp, sizeof(double) * total);
    }
    free(tmp);
}

/* Selected elements of e^{n+1}: pts[3*j] = k, pts[3*j+1] = d, pts[3*j+2] = cell index.
 * Only the T_L and diffuse-wall values those elements need are formed.              */
void orc_step_points(const orc_problem *P, const double *e_in, const float *Q, double amp, long npts,
                     const long *pts, double *out) {
    const long nc = ncell_of(P);
    const double W = total_weight(P), SC = sum_C(P), D = sum_C_over_tau(P);
    double *ediff = (double *)calloc((size_t)6 * P->nb * nc, sizeof(double));
    diffuse_wall_values(P, e_in, ediff);
    #pragma omp parallel for schedule(dynamic, 64)
    for (long j = 0; j < npts; ++j) {
        const int k = (int)pts[3 * j], d = (int)pts[3 * j + 1];
        const long i = pts[3 * j + 2];
        const int c[3] = {(int)(i % P->nx), (int)((i / P->nx) % P->ny), (int)(i / ((long)P->nx * P->ny))};
        /* T_L at this one cell, Eq. (BTE_get_e0) */
        double acc = 0.0;
        for (int kk = 0; kk < P->nb; ++kk) {
            double sk = 0.0;
            for (int dd = 0; dd < P->nd; ++dd) sk += P->w[dd] * e_in[EIDX(P, kk, dd, i)];
            acc += sk / P->tau[kk];
        }
        out[j] = step_element(P, e_in, ediff, acc / D, Q, amp, W, SC, k, d, c);
    }
    free(ediff);
}

/* ------------------------------------------------------------------------- */
/* Global energy and wall heat flow (the energy-balance reductions).          */
/*   E = V sum_i sum_k sum_d w_d e                                            */
/*   F_wall = S_wall sum_{wall cells} sum_k sum_d w_d v_k (s_d.n) e_face       */
/* with e_face the wall-face value the step uses.  For one step,              */
/*   E^{n+1} - E^n = dt ( V amp sum_i Q_i - sum_walls F_wall^n ).             */
/* ------------------------------------------------------------------------- */
static void energy_with(const orc_problem *P, const double *e, const double *ediff, double *E_total,
                        double *wall_flux) {
    const long nc = ncell_of(P);
    const double V = cell_volume(P);
    double E = 0.0;
    for (int k = 0; k < P->nb; ++k)
        for (int d = 0; d < P->nd; ++d)
            for (long i = 0; i < nc; ++i) E += P->w[d] * e[EIDX(P, k, d, i)];
    *E_total = V * E;
    for (int wall = 0; wall < 6; ++wall) wall_flux[wall] = 0.0;
    for (int a = 0; a < P->dim; ++a) {
        const double S = V / length_of(P, a);
        const int n = extent(P, a);
        for (int side = 0; side < 2; ++side) {
            const int wall = 2 * a + side;
            const double nsign = side == 0 ? -1.0 : 1.0;
            double F = 0.0;
            for (int z = 0; z < P->nz; ++z)
                for (int y = 0; y < P->ny; ++y)
                    for (int x = 0; x < P->nx; ++x) {
                        int c[3] = {x, y, z};
                        if (c[a] != (side == 0 ? 0 : n - 1)) continue;
                        const int pface = side == 0 ? -1 : n - 1; /* face between pface and pface+1 */
                        for (int k = 0; k < P->nb; ++k)
                            for (int d = 0; d < P->nd; ++d) {
                                const double sa = P->s[3 * d + a];
                                if (sa == 0.0) continue;
                                const double ef = face_value(P, e, ediff, k, d, a, c, pface);
                                F += P->w[d] * P->v[k] * nsign * sa * ef;
                            }
                    }
            wall_flux[wall] = S * F;
        }
    }
}

void orc_energy(const orc_problem *P, const double *e, double *E_total, double *wall_flux) {
    double *ediff = (double *)calloc((size_t)6 * P->nb * ncell_of(P), sizeof(double));
    diffuse_wall_values(P, e, ediff);
    energy_with(P, e, ediff, E_total, wall_flux);
    free(ediff);
}

/* ------------------------------------------------------------------------- */
/* Steady state by the implicit DOM, sequential iterative scheme (Sec. 3.3-   */
/* 3.5, Eq. disretized_BTE in delta form).  One iteration updates every band  */
/* and direction from the current e^n and its T_L:                             */
/*   (1/tau_k + sum_a c_a) De_i - sum_a c_a De_{up_a(i)} = R_i,               */
/*   c_a = v_k |s_a| / h_a,  up_a(i) the upwind neighbour of i along axis a,   */
/* the left side with first-order upwind faces, the right side                */
/*   R_i = -sum_a (v_k s_a / h_a)(e_{i+1/2} - e_{i-1/2}) - (e_i - C_k T_L/W)/tau_k */
/*         + Q_i C_k / (sum C W)                                               */
/* with the transient step's face values and walls (second order, limited).  */
/* Across a wall (periodic pairs included) the upwind De is taken as 0: the   */
/* boundary values are those of e^n and move at the next iteration.  Each     */
/* (k, d) system is then lower triangular in upwind order and is solved by    */
/* one sweep: z, y and x each run from the upwind side.  e_out = e_in + De.   */
/* ------------------------------------------------------------------------- */
static double residual_element(const orc_problem *P, const double *e, const double *ediff, double TLi,
                               const float *Q, double amp, double W, double SC, int k, int d, const int c[3]) {
    const long i = cidx(P, c);
    const double en = e[EIDX(P, k, d, i)];
    double div = 0.0;
    for (int a = 0; a < P->dim; ++a) {
        const double sa = P->s[3 * d + a];
        if (sa == 0.0) continue;
        const double fr = face_value(P, e, ediff, k, d, a, c, c[a]);
        const double fl = face_value(P, e, ediff, k, d, a, c, c[a] - 1);
        div += P->v[k] * sa / spacing(P, a) * (fr - fl);
    }
    const double e0 = P->C[k] * TLi / W;
    const double src = Q ? amp * (double)Q[i] * P->C[k] / (SC * W) : 0.0;
    return -div + (e0 - en) / P->tau[k] + src;
}

/* The same iteration with the equilibrium e0 = C_k TL / W of a given lattice temperature TL (the
 * synthetic scheme of Sec. 3.5 corrects T_L between iterations). */
void orc_sis_iteration_tl(const orc_problem *P, const double *e_in, const double *TL, double *e_out, const float *Q,
                          double amp) {
    const long nc = ncell_of(P);
    const double W = total_weight(P), SC = sum_C(P);
    double *ediff = (double *)calloc((size_t)6 * P->nb * nc, sizeof(double));
    diffuse_wall_values(P, e_in, ediff);
    const long nplanes = (long)P->nb * P->nd;
    #pragma omp parallel for schedule(dynamic, 1)
    for (long pl = 0; pl < nplanes; ++pl) {
        const int k = (int)(pl / P->nd), d = (int)(pl % P->nd);
        double *De = (double *)malloc(sizeof(double) * nc);
        double cf[3] = {0, 0, 0}, diag = 1.0 / P->tau[k];
        int sg[3] = {1, 1, 1};
        for (int a = 0; a < P->dim; ++a) {
            const double sa = P->s[3 * d + a];
            cf[a] = P->v[k] * fabs(sa) / spacing(P, a);
            diag += cf[a];
            sg[a] = sa >= 0.0 ? 1 : -1;
        }
        for (int uz = 0; uz < P->nz; ++uz)
            for (int uy = 0; uy < P->ny; ++uy)
                for (int ux = 0; ux < P->nx; ++ux) {
                    const int c[3] = {sg[0] > 0 ? ux : P->nx - 1 - ux, sg[1] > 0 ? uy : P->ny - 1 - uy,
                                      sg[2] > 0 ? uz : P->nz - 1 - uz};
                    const long i = cidx(P, c);
                    double rhs = residual_element(P, e_in, ediff, TL[i], Q, amp, W, SC, k, d, c);
                    for (int a = 0; a < P->dim; ++a) {
                        if (cf[a] == 0.0) continue;
                        int cu[3] = {c[0], c[1], c[2]};
                        cu[a] -= sg[a];
                        if (cu[a] < 0 || cu[a] >= extent(P, a)) continue; /* across a wall: 0 */
                        rhs += cf[a] * De[cidx(P, cu)];
                    }
                    De[i] = rhs / diag;
                    e_out[EIDX(P, k, d, i)] = e_in[EIDX(P, k, d, i)] + De[i];
                }
        free(De);
    }
    free(ediff);
}

void orc_sis_iteration(const orc_problem *P, const double *e_in, double *e_out, const float *Q, double amp) {
    double *TL = (double *)malloc(sizeof(double) * ncell_of(P));
    orc_lattice_temperature(P, e_in, TL);
    orc_sis_iteration_tl(P, e_in, TL, e_out, Q, amp);
    free(TL);
}

/* ------------------------------------------------------------------------- */
/* Interface between two materials, Sec. 2.2 (v): wall wa of problem A (the   */
/* material-A side) faces wall wb of problem B, both declared DIFFUSE, with   */
/* the same axis, opposite sides and the same cells along the other two axes. */
/* A phonon of band k reaching the interface from A is transmitted into B     */
/* with probability bAB[k] and diffusely reflected otherwise; from B,         */
/* bBA[k].  The incoming value at each interface cell is therefore            */
/*   e_in,A = bBA S_B + (1 - bAB) S_A,   e_in,B = bAB S_A + (1 - bBA) S_B,     */
/* with S_X the diffuse value of side X's outgoing directions at its cell     */
/* (the integral of e |s.n| over the directions reaching the interface over   */
/* the integral of |s.n| over the other half, Eq. (diff_bound)'s discrete     */
/* normaliser: the 1/pi of the paper's formula).  Transmitted energy is taken */
/* with |s.n|; the paper's integral over B's directions carries s.n < 0.      */
/* ediffA, ediffB: [6][nb][ncell] of each problem, filled at every DIFFUSE    */
/* wall (plain diffuse values) and then mixed at the interface cells.         */
/* ------------------------------------------------------------------------- */
static int interface_ok(const orc_problem *A, int wa, const orc_problem *B, int wb) {
    if (A->dim != B->dim || A->nb != B->nb || wa < 0 || wb < 0 || wa >= 2 * A->dim || wb >= 2 * B->dim) return 0;
    if ((wa >> 1) != (wb >> 1) || (wa & 1) == (wb & 1)) return 0;
    if (A->bc[wa] != ORC_BC_DIFFUSE || B->bc[wb] != ORC_BC_DIFFUSE) return 0;
    for (int a = 0; a < 3; ++a)
        if (a != (wa >> 1) && extent(A, a) != extent(B, a)) return 0;
    return 1;
}

int orc_interface_values(const orc_problem *A, const double *eA, int wa, const orc_problem *B, const double *eB, int wb,
                         const double *bAB, const double *bBA, double *ediffA, double *ediffB) {
    if (!interface_ok(A, wa, B, wb)) return 1;
    const long ncA = ncell_of(A), ncB = ncell_of(B);
    diffuse_wall_values(A, eA, ediffA);
    diffuse_wall_values(B, eB, ediffB);
    const int a = wa >> 1;
    const int posA = (wa & 1) ? extent(A, a) - 1 : 0, posB = (wb & 1) ? extent(B, a) - 1 : 0;
    for (int z = 0; z < A->nz; ++z)
        for (int y = 0; y < A->ny; ++y)
            for (int x = 0; x < A->nx; ++x) {
                int c[3] = {x, y, z};
                if (c[a] != posA) continue;
                const long iA = cidx(A, c);
                c[a] = posB;
                const long iB = cidx(B, c);
                for (int k = 0; k < A->nb; ++k) {
                    double *pa = &ediffA[((long)wa * A->nb + k) * ncA + iA];
                    double *pb = &ediffB[((long)wb * B->nb + k) * ncB + iB];
                    const double SA = *pa, SB = *pb;
                    *pa = bBA[k] * SB + (1.0 - bAB[k]) * SA;
                    *pb = bAB[k] * SA + (1.0 - bBA[k]) * SB;
                }
            }
    return 0;
}

/* One step of both materials (Algorithm 2 for each, with the interface values above). */
int orc_interface_step(const orc_problem *A, const double *eA, double *eA_out, const float *QA, double ampA, int wa,
                       const orc_problem *B, const double *eB, double *eB_out, const float *QB, double ampB, int wb,
                       const double *bAB, const double *bBA) {
    double *ediffA = (double *)calloc((size_t)6 * A->nb * ncell_of(A), sizeof(double));
    double *ediffB = (double *)calloc((size_t)6 * B->nb * ncell_of(B), sizeof(double));
    const int rc = orc_interface_values(A, eA, wa, B, eB, wb, bAB, bBA, ediffA, ediffB);
    if (rc == 0) {
        step_with(A, eA, ediffA, eA_out, QA, ampA);
        step_with(B, eB, ediffB, eB_out, QB, ampB);
    }
    free(ediffA);
    free(ediffB);
    return rc;
}

/* Energy and wall heat flows of both materials; the flows through wa and wb are the */
/* interface heat flows (outward from each side).                                    */
int orc_interface_energy(const orc_problem *A, const double *eA, int wa, const orc_problem *B, const double *eB, int wb,
                         const double *bAB, const double *bBA, double *EA, double *fluxA, double *EB, double *fluxB) {
    double *ediffA = (double *)calloc((size_t)6 * A->nb * ncell_of(A), sizeof(double));
    double *ediffB = (double *)calloc((size_t)6 * B->nb * ncell_of(B), sizeof(double));
    const int rc = orc_interface_values(A, eA, wa, B, eB, wb, bAB, bBA, ediffA, ediffB);
    if (rc == 0) {
        energy_with(A, eA, ediffA, EA, fluxA);
        energy_with(B, eB, ediffB, EB, fluxB);
    }
    free(ediffA);
    free(ediffB);
    return rc;
}

/* ========================================================================= */
/* Discrete adjoint of the step (not in the paper; the exact transpose of    */
/* the forward step above, derived by hand).                                  */
/*                                                                           */
/* One step is e^{n+1} = F(e^n, T_L(e^n)) with T_L linear in e.  Its          */
/* Jacobian J = dF/de + dF/dT_L dT_L/de.  For a functional                    */
/*   J_obj = sum_i p_i T_L,i(e^N)                                             */
/* the adjoint lambda^N = dT_L/de^T p, lambda^n = J(e^n)^T lambda^{n+1}, and  */
/*   dJ/dQ_i      = sum_n dt a_n sum_{k,d} lambda^{n+1}_{k,d,i} C_k/(sum C W)  */
/*   dJ/dlog tau_k = sum_n [ sum_{d,i} lambda^{n+1} (-dt/tau_k)(C_k T_L/W - e) */
/*                  + sum_i mu_i dT_L,i/dlog tau_k ] + sum_i p_i dT_L^N/dlog tau_k */
/* with mu_i = sum_{k,d} lambda^{n+1}_{k,d,i} dt C_k/(W tau_k) and            */
/*   dT_L,i/dlog tau_k = (C_k T_L,i - sum_d w_d e_{k,d,i}) / (tau_k D).       */
/* Two independent codings of J are given: a forward (tangent) one and a      */
/* reverse (transpose) one, so that <lambda, J de> = <J^T lambda, de> checks  */
/* both.                                                                      */
/* ========================================================================= */

/* Partial derivatives La = dL/da, Lb = dL/db of the slope limiter (0 where ab <= 0). */
static void limiter_grad(int kind, double a, double b, double *La, double *Lb) {
    *La = *Lb = 0.0;
    if (kind == ORC_LIM_FIRST_ORDER || a * b <= 0.0) return;
    if (kind == ORC_LIM_MINMOD) {
        if (fabs(a) < fabs(b)) *La = 1.0;
        else *Lb = 1.0;
        return;
    }
    /* L = ab(a+b)/(a^2+b^2): dL/da = b^2 (2ab + b^2 - a^2)/(a^2+b^2)^2, symmetric in b */
    const double q = a * a + b * b;
    *La = b * b * (2.0 * a * b + b * b - a * a) / (q * q);
    *Lb = a * a * (2.0 * a * b + a * a - b * b) / (q * q);
}

/* Positions (along axis a) of the upwind-left, upwind and downwind-right values a face
 * reads, for the face between p and p+1 (same orientation as face_value). */
static void face_positions(const orc_problem *P, int d, int a, int p, int pos[3]) {
    if (P->s[3 * d + a] > 0.0) { pos[0] = p - 1; pos[1] = p; pos[2] = p + 1; }
    else { pos[0] = p + 2; pos[1] = p + 1; pos[2] = p; }
}

/* d(face)/d(u_l), d(face)/d(u_m), d(face)/d(u_r) of e_face = u_m + L(u_m-u_l, u_r-u_m)/2. */
static void face_grad(const orc_problem *P, const double *e, const double *ediff, int k, int d, int a,
                      const int c[3], int p, double g[3]) {
    int pos[3];
    face_positions(P, d, a, p, pos);
    const double ul = ext_value(P, e, ediff, k, d, a, c, pos[0]);
    const double um = ext_value(P, e, ediff, k, d, a, c, pos[1]);
    const double ur = ext_value(P, e, ediff, k, d, a, c, pos[2]);
    double La, Lb;
    limiter_grad(P->limiter, um - ul, ur - um, &La, &Lb);
    g[0] = -0.5 * La;
    g[1] = 1.0 + 0.5 * (La - Lb);
    g[2] = 0.5 * Lb;
}

/* The elements an extended value (ext_value) depends on, with their coefficients:
 * ext = sum_j coef[j] e[idx[j]] + (constant of a thermalizing wall).  Returns the count
 * (at most nd). */
static int ext_deps(const orc_problem *P, int k, int d, int a, const int c[3], int p, long *idx, double *coef) {
    const int n = extent(P, a);
    int cc[3] = {c[0], c[1], c[2]};
    if (p >= 0 && p < n) {
        cc[a] = p;
        idx[0] = EIDX(P, k, d, cidx(P, cc));
        coef[0] = 1.0;
        return 1;
    }
    const int side = p < 0 ? 0 : 1;
    const int layer = p < 0 ? -p : p - n + 1;
    const int wall = 2 * a + side;
    const double sa = P->s[3 * d + a];
    const int incoming = side == 0 ? (sa > 0.0) : (sa < 0.0);
    const int wallpos = side == 0 ? 0 : n - 1;
    switch (P->bc[wall]) {
    case ORC_BC_PERIODIC:
        cc[a] = ((p % n) + n) % n;
        idx[0] = EIDX(P, k, d, cidx(P, cc));
        coef[0] = 1.0;
        return 1;
    case ORC_BC_ISOTHERMAL:
        if (incoming) return 0;
        cc[a] = wallpos;
        idx[0] = EIDX(P, k, d, cidx(P, cc));
        coef[0] = 1.0;
        return 1;
    case ORC_BC_DIFFUSE: {
        cc[a] = wallpos;
        const long i = cidx(P, cc);
        if (!incoming) {
            idx[0] = EIDX(P, k, d, i);
            coef[0] = 1.0;
            return 1;
        }
        /* e_diff = sum_{s.n>0} w (s.n) e / sum_{s.n<0} w |s.n| at the wall cell */
        const double nsign = side == 0 ? -1.0 : 1.0;
        double den = 0.0;
        for (int dd = 0; dd < P->nd; ++dd) {
            const double sn = nsign * P->s[3 * dd + a];
            if (sn < 0.0) den += P->w[dd] * (-sn);
        }
        int m = 0;
        for (int dd = 0; dd < P->nd; ++dd) {
            const double sn = nsign * P->s[3 * dd + a];
            if (sn > 0.0) {
                idx[m] = EIDX(P, k, dd, i);
                coef[m] = P->w[dd] * sn / den;
                ++m;
            }
        }
        return m;
    }
    case ORC_BC_SPECULAR:
    default:
        cc[a] = side == 0 ? layer - 1 : n - layer;
        idx[0] = EIDX(P, k, P->mirror[a * P->nd + d], cidx(P, cc));
        coef[0] = 1.0;
        return 1;
    }
}

/* Homogeneous part of an extended value of a perturbation de (thermalizing-wall
 * emission and the periodic jump are constants, so their perturbation is 0). */
static double ext_value_lin(const orc_problem *P, const double *de, const double *dediff, int k, int d, int a,
                            const int c[3], int p) {
    const int n = extent(P, a);
    if (p < 0 || p >= n) {
        const int side = p < 0 ? 0 : 1;
        const int wall = 2 * a + side;
        const double sa = P->s[3 * d + a];
        const int incoming = side == 0 ? (sa > 0.0) : (sa < 0.0);
        if (P->bc[wall] == ORC_BC_ISOTHERMAL && incoming) return 0.0;
        if (P->bc[wall] == ORC_BC_PERIODIC) return ext_value(P, de, dediff, k, d, a, c, p) - periodic_jump(P, k, a, side);
    }
    return ext_value(P, de, dediff, k, d, a, c, p);
}

/* Tangent (forward-mode) step: dout = J(e) de, T_L coupling included. */
void orc_step_tangent(const orc_problem *P, const double *e, const double *de, double *dout) {
    const long nc = ncell_of(P);
    const double W = total_weight(P);
    double *dTL = (double *)malloc(sizeof(double) * nc);
    double *ediff = (double *)calloc((size_t)6 * P->nb * nc, sizeof(double));
    double *dediff = (double *)calloc((size_t)6 * P->nb * nc, sizeof(double));
    orc_lattice_temperature(P, de, dTL);
    diffuse_wall_values(P, e, ediff);
    diffuse_wall_values(P, de, dediff);
    for (int k = 0; k < P->nb; ++k)
        for (int d = 0; d < P->nd; ++d)
            for (int z = 0; z < P->nz; ++z)
                for (int y = 0; y < P->ny; ++y)
                    for (int x = 0; x < P->nx; ++x) {
                        const int c[3] = {x, y, z};
                        const long i = cidx(P, c);
                        double ddiv = 0.0;
                        for (int a = 0; a < P->dim; ++a) {
                            const double sa = P->s[3 * d + a];
                            if (sa == 0.0) continue;
                            const double nu = P->dt * P->v[k] * sa / spacing(P, a);
                            double dface[2];
                            for (int f = 0; f < 2; ++f) { /* face i+1/2 (p = c[a]) and i-1/2 (p = c[a]-1) */
                                const int p = c[a] - f;
                                int pos[3];
                                double g[3];
                                face_positions(P, d, a, p, pos);
                                face_grad(P, e, ediff, k, d, a, c, p, g);
                                dface[f] = 0.0;
                                for (int r = 0; r < 3; ++r)
                                    dface[f] += g[r] * ext_value_lin(P, de, dediff, k, d, a, c, pos[r]);
                            }
                            ddiv += nu * (dface[0] - dface[1]);
                        }
                        const double den = de[EIDX(P, k, d, i)];
                        dout[EIDX(P, k, d, i)] = den - ddiv + P->dt * (P->C[k] * dTL[i] / W - den) / P->tau[k];
                    }
    free(dTL);
    free(ediff);
    free(dediff);
}

/* Transposed (reverse-mode) step: lam_out = J(e)^T lam_in.  Every forward element scatters
 * its adjoint into the elements it read, through the ghost rules. */
void orc_adjoint_step(const orc_problem *P, const double *e, const double *lam_in, double *lam_out) {
    const long nc = ncell_of(P);
    const long total = (long)P->nb * P->nd * nc;
    const double W = total_weight(P), D = sum_C_over_tau(P);
    double *ediff = (double *)calloc((size_t)6 * P->nb * nc, sizeof(double));
    double *mu = (double *)calloc((size_t)nc, sizeof(double));
    diffuse_wall_values(P, e, ediff);
    memset(lam_out, 0, sizeof(double) * total);
    /* T_L coupling: d e^{n+1}_{k,d,i}/d T_L,i = dt C_k/(W tau_k) */
    #pragma omp parallel for schedule(static)
    for (long i = 0; i < nc; ++i)
        for (int k = 0; k < P->nb; ++k)
            for (int d = 0; d < P->nd; ++d) mu[i] += lam_in[EIDX(P, k, d, i)] * P->dt * P->C[k] / (W * P->tau[k]);
    /* Every element of band k scatters only into band k (the ghost rules never leave a band),
     * so the bands run in parallel and each element sums its terms in the serial order. */
    #pragma omp parallel for schedule(dynamic, 1)
    for (int k = 0; k < P->nb; ++k) {
        long *idx = (long *)malloc(sizeof(long) * (P->nd + 1));
        double *coef = (double *)malloc(sizeof(double) * (P->nd + 1));
        for (int d = 0; d < P->nd; ++d)
            for (int z = 0; z < P->nz; ++z)
                for (int y = 0; y < P->ny; ++y)
                    for (int x = 0; x < P->nx; ++x) {
                        const int c[3] = {x, y, z};
                        const long i = cidx(P, c);
                        const double lam = lam_in[EIDX(P, k, d, i)];
                        /* e^n and the relaxation -dt/tau e^n */
                        lam_out[EIDX(P, k, d, i)] += lam * (1.0 - P->dt / P->tau[k]);
                        /* T_L,i = sum w e / tau / D */
                        lam_out[EIDX(P, k, d, i)] += mu[i] * P->w[d] / (P->tau[k] * D);
                        /* flux: - nu (face(i+1/2) - face(i-1/2)) */
                        for (int a = 0; a < P->dim; ++a) {
                            const double sa = P->s[3 * d + a];
                            if (sa == 0.0) continue;
                            const double nu = P->dt * P->v[k] * sa / spacing(P, a);
                            for (int f = 0; f < 2; ++f) {
                                const int p = c[a] - f;
                                const double sgn = f == 0 ? -nu : nu;
                                int pos[3];
                                double g[3];
                                face_positions(P, d, a, p, pos);
                                face_grad(P, e, ediff, k, d, a, c, p, g);
                                for (int r = 0; r < 3; ++r) {
                                    const int m = ext_deps(P, k, d, a, c, pos[r], idx, coef);
                                    for (int j = 0; j < m; ++j) lam_out[idx[j]] += sgn * lam * g[r] * coef[j];
                                }
                            }
                        }
                    }
        free(idx);
        free(coef);
    }
    free(ediff);
    free(mu);
}

/* Adjoint of a whole run: J = sum_i p_i T_L,i after nsteps steps from e0 (steps n0 ..
 * n0+nsteps-1, source amplitude amp[n], 1 when amp is NULL, 0 past namp).  States are kept
 * at every ckpt-th step (ckpt <= 0: every state); the reverse sweep recomputes each segment
 * from its checkpoint before stepping back through it, which gives the same states bitwise
 * (the forward step is deterministic).  Memory: nsteps/ckpt + ckpt + 1 states.  Outputs J,
 * dJ/dQ (ncell) and dJ/dlog tau (nb).  Returns 0, or 1 when out of memory. */
int orc_adjoint(const orc_problem *P, const double *e0, const float *Q, const double *amp, int namp, long n0,
                int nsteps, const double *probe, double *J, double *gQ, double *gtau, int ckpt) {
    const long nc = ncell_of(P);
    const long total = (long)P->nb * P->nd * nc;
    const double W = total_weight(P), SC = sum_C(P), D = sum_C_over_tau(P);
    const int K = (ckpt > 0 && ckpt < nsteps) ? ckpt : (nsteps > 0 ? nsteps : 1);
    const int nseg = nsteps > 0 ? (nsteps + K - 1) / K : 0;
    double *cps = (double *)malloc(sizeof(double) * total * (size_t)(nseg > 0 ? nseg : 1));
    double *traj = (double *)malloc(sizeof(double) * total * (size_t)(K + 1)); /* a segment's states, then e^N */
    double *lam = (double *)malloc(sizeof(double) * total);
    double *lam2 = (double *)malloc(sizeof(double) * total);
    double *TL = (double *)malloc(sizeof(double) * nc);
    double *mu = (double *)malloc(sizeof(double) * nc);
    if (!cps || !traj || !lam || !lam2 || !TL || !mu) {
        free(cps); free(traj); free(lam); free(lam2); free(TL); free(mu);
        return 1;
    }
    /* forward sweep: checkpoints at steps 0, K, 2K, ..., e^N in the last slot of traj */
    memcpy(traj, e0, sizeof(double) * total);
    for (int s = 0; s < nsteps; ++s) {
        const long n = n0 + s;
        const double a = amp ? (n < namp ? amp[n] : 0.0) : 1.0;
        if (s % K == 0) memcpy(cps + (size_t)(s / K) * total, traj, sizeof(double) * total);
        orc_step(P, traj, traj + (size_t)K * total, Q, a);
        memcpy(traj, traj + (size_t)K * total, sizeof(double) * total);
    }
    memcpy(traj + (size_t)K * total, traj, sizeof(double) * total);
    for (long i = 0; i < nc; ++i) gQ[i] = 0.0;
    for (int k = 0; k < P->nb; ++k) gtau[k] = 0.0;
    /* J and lambda^N = dT_L/de^T p; the final T_L's own tau dependence */
    const double *eN = traj + (size_t)K * total;
    orc_lattice_temperature(P, eN, TL);
    double Jv = 0.0;
    for (long i = 0; i < nc; ++i) Jv += probe[i] * TL[i];
    *J = Jv;
    for (int k = 0; k < P->nb; ++k)
        for (int d = 0; d < P->nd; ++d)
            for (long i = 0; i < nc; ++i) lam[EIDX(P, k, d, i)] = probe[i] * P->w[d] / (P->tau[k] * D);
    for (int k = 0; k < P->nb; ++k)
        for (long i = 0; i < nc; ++i) {
            double S = 0.0;
            for (int d = 0; d < P->nd; ++d) S += P->w[d] * eN[EIDX(P, k, d, i)];
            gtau[k] += probe[i] * (P->C[k] * TL[i] - S) / (P->tau[k] * D);
        }
    for (int s = nsteps - 1; s >= 0; --s) {
        const long n = n0 + s;
        const double a = amp ? (n < namp ? amp[n] : 0.0) : 1.0;
        const int s0 = (s / K) * K;
        if (s == nsteps - 1 || s % K == K - 1) {
            /* entering segment [s0, s]: its states from the checkpoint */
            memcpy(traj, cps + (size_t)(s / K) * total, sizeof(double) * total);
            for (int m = s0; m < s; ++m) {
                const long nm = n0 + m;
                const double am = amp ? (nm < namp ? amp[nm] : 0.0) : 1.0;
                orc_step(P, traj + (size_t)(m - s0) * total, traj + (size_t)(m - s0 + 1) * total, Q, am);
            }
        }
        const double *en = traj + (size_t)(s - s0) * total;
        orc_lattice_temperature(P, en, TL);
        for (long i = 0; i < nc; ++i) mu[i] = 0.0;
        for (int k = 0; k < P->nb; ++k)
            for (int d = 0; d < P->nd; ++d)
                for (long i = 0; i < nc; ++i) {
                    const double l = lam[EIDX(P, k, d, i)];
                    gQ[i] += P->dt * a * l * P->C[k] / (SC * W);
                    mu[i] += l * P->dt * P->C[k] / (W * P->tau[k]);
                    gtau[k] += l * (-P->dt / P->tau[k]) * (P->C[k] * TL[i] / W - en[EIDX(P, k, d, i)]);
                }
        for (int k = 0; k < P->nb; ++k)
            for (long i = 0; i < nc; ++i) {
                double S = 0.0;
                for (int d = 0; d < P->nd; ++d) S += P->w[d] * en[EIDX(P, k, d, i)];
                gtau[k] += mu[i] * (P->C[k] * TL[i] - S) / (P->tau[k] * D);
            }
        orc_adjoint_step(P, en, lam, lam2);
        memcpy(lam, lam2, sizeof(double) * total);
    }
    free(cps); free(traj); free(lam); free(lam2); free(TL); free(mu);
    return 0;
}
