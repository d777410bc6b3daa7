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
        return e[EIDX(P, k, d, cidx(P, cc))];
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
void orc_step(const orc_problem *P, const double *e_in, double *e_out, const float *Q, double amp) {
    const long nc = ncell_of(P);
    const double W = total_weight(P), SC = sum_C(P);
    double *TL = (double *)malloc(sizeof(double) * nc);
    double *ediff = (double *)calloc((size_t)6 * P->nb * nc, sizeof(double));
    orc_lattice_temperature(P, e_in, TL);
    diffuse_wall_values(P, e_in, ediff);
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
void orc_energy(const orc_problem *P, const double *e, double *E_total, double *wall_flux) {
    const long nc = ncell_of(P);
    const double V = cell_volume(P);
    double E = 0.0;
    for (int k = 0; k < P->nb; ++k)
        for (int d = 0; d < P->nd; ++d)
            for (long i = 0; i < nc; ++i) E += P->w[d] * e[EIDX(P, k, d, i)];
    *E_total = V * E;
    double *ediff = (double *)calloc((size_t)6 * P->nb * nc, sizeof(double));
    diffuse_wall_values(P, e, ediff);
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
    free(ediff);
}
