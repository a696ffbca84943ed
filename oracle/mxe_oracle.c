/*
 * mxe_oracle.c -- plain, slow, FP64 CPU oracle of the MXE hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark load this file's library.  It shares no
 * code, header, table or helper with the CUDA library; both sides only read
 * the same seeded input arrays.
 *
 * Every function follows the paper (Mendez & Ponga, "MXE: A package for
 * simulating long-term diffusive mass transport phenomena in nanoscale
 * systems") in its own order and notation; nothing is blocked, fused or
 * reordered beyond what the definition states.  Compiled with
 * -ffp-contract=off so that no multiply-add is contracted.
 *
 *   neighbour sets        Sec. 4 / Algorithm 1 (neighbour list step), brute force
 *   quadrature nodes      App. A (third-degree rule, M = 2 N_q nodes, r^2 = N_q/2)
 *   thermalized EAM       App. B.2 (Eqs. EAM_mxe, F_taylor_mxe, EAM-Substitutional-ave,
 *                         EAM-density-substitutional-ave); the exact embedding average
 *                         (App. A's rule over a site and its neighbours, before Eq. F_taylor)
 *   free energy           Sec. 2.1 (Eq. Grand-Canonical-Free-Energy) read per site as
 *                         <V_i> - 3 kB T_i ln sigma_i + kB T_i sum_k x ln x (vacancy included)
 *   gradients             derivatives of the above, written out term by term
 *   mass transport        Sec. 3.1 (Eqs. MassTransport, attempt_freq_mass), forward Euler (Sec. 4)
 *   relaxation            FIRE (Bitzek et al., PRL 97, 170201, 2006) on (q, sigma)
 *
 * Parity status: every function here is pinned by a CPU test (quadrature moments
 * and Gaussian limit, sigma -> 0 static EAM, central finite differences of F,
 * perfect-lattice symmetry, translation invariance, brute-force neighbours,
 * linear-Fick closed form, mass conservation, FIRE stationarity).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAXS 4
#define ORC_KB 8.617333262e-5   /* eV/K */
#define ORC_NODES 12            /* pair: N = 2 sites, N_q = 6, M = 2 N_q */
#define ORC_RMIN 0.5            /* smallest admissible node distance (A) */
#define ORC_RHO_MIN 1e-12       /* smallest admissible static density */
#define ORC_X_TOL 1e-12         /* admissible excursion of x outside [0, 1] */
#define ORC_SIGMA_MIN 1e-3      /* FIRE keeps sigma >= this (A) */
#define ORC_LOG_FLOOR 1e-300    /* argument floor of ln x in the full chemical potential */

enum { ORC_OK = 0, ORC_ERR_ARG = 1, ORC_ERR_BOX_TOO_SMALL = 4, ORC_ERR_NBR_OVERFLOW = 5,
       ORC_ERR_GEOMETRY = 6, ORC_ERR_NONFINITE = 7, ORC_ERR_X_RANGE = 8, ORC_ERR_NO_CONVERGE = 9 };

typedef struct {
    int32_t n_species;
    int32_t cross_geomean;
    double phi_A[ORC_MAXS][ORC_MAXS], phi_p[ORC_MAXS][ORC_MAXS], phi_r0[ORC_MAXS][ORC_MAXS];
    double f_xi[ORC_MAXS][ORC_MAXS], f_q[ORC_MAXS][ORC_MAXS], f_r0[ORC_MAXS][ORC_MAXS];
    double E[ORC_MAXS];
    double r_switch, r_cut;
    /* Thermalized Lennard-Jones pair terms (App. C.1) in place of phi when
       lj != 0: phi_kl = 4 eps_kl [(s_kl / r)^12 - (s_kl / r)^6] S(r).  An
       element with E_k = 0 has no embedding energy. */
    int32_t lj;
    int32_t pad;
    double lj_eps[ORC_MAXS][ORC_MAXS], lj_sigma[ORC_MAXS][ORC_MAXS];
} orc_potential;

typedef struct {
    int64_t n;
    int32_t S;
    int32_t pad;
    double L[3];
    const double *q;      /* [3][n] */
    const double *sigma;  /* [n] */
    const double *x;      /* [S][n] */
    const double *T;      /* [n] */
} orc_system;

typedef struct {
    double dt0, dt_max, f_inc, f_dec, alpha0, f_alpha;
    double sigma_max;   /* upper bound of sigma (A); <= 0 or inf: none */
    int32_t n_min;
    int32_t pad;
} orc_fire;

/* Force on sigma projected on the box [lo, hi]: zero where a bound blocks it. */
static double proj_fsig(double gs, double sigma, double lo, double hi)
{
    double f = -gs;
    if (sigma >= hi && f > 0.0) return 0.0;
    if (sigma <= lo && f < 0.0) return 0.0;
    return f;
}

/* ------------------------------------------------------------------ */
/* Pairwise summation (deterministic, accurate totals).                */
/* ------------------------------------------------------------------ */
static double pairwise_sum(const double *v, int64_t n)
{
    if (n <= 8) {
        double s = 0.0;
        for (int64_t i = 0; i < n; ++i) s += v[i];
        return s;
    }
    int64_t h = n / 2;
    return pairwise_sum(v, h) + pairwise_sum(v + h, n - h);
}

/* ------------------------------------------------------------------ */
/* Minimum image (periodic box, rounding half to even).                */
/* ------------------------------------------------------------------ */
static void min_image(const double L[3], const double qi[3], const double qj[3], double d[3])
{
    for (int a = 0; a < 3; ++a) {
        double invL = 1.0 / L[a];
        double da = qj[a] - qi[a];
        double k = nearbyint(da * invL);
        double shift = L[a] * k;
        d[a] = da - shift;
    }
}

static double dist2(const double d[3])
{
    double s = d[0] * d[0];
    s = s + d[1] * d[1];
    s = s + d[2] * d[2];
    return s;
}

static void load_q(const double *q, int64_t n, int64_t i, double out[3])
{
    out[0] = q[i];
    out[1] = q[n + i];
    out[2] = q[2 * n + i];
}

/* ------------------------------------------------------------------ */
/* Neighbour sets: every j != i with |minimum image of q_j - q_i| < r_list,
 * each row sorted by j.  Brute force over all pairs.  Requires L >= 2 r_list
 * on every axis so that at most one periodic image can be in range.        */
/* ------------------------------------------------------------------ */
int orc_neighbors(int64_t n, const double *q, const double L[3], double r_list,
                  int32_t *offsets, int32_t *idx, int64_t cap, int64_t *n_pairs)
{
    if (n < 0 || !(r_list > 0.0)) return ORC_ERR_ARG;
    for (int a = 0; a < 3; ++a)
        if (!(L[a] >= 2.0 * r_list)) return ORC_ERR_BOX_TOO_SMALL;
    double rl2 = r_list * r_list;
    int64_t count = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (offsets) offsets[i] = (int32_t)count;
        double qi[3];
        load_q(q, n, i, qi);
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double qj[3], d[3];
            load_q(q, n, j, qj);
            min_image(L, qi, qj, d);
            if (dist2(d) < rl2) {
                if (idx && count < cap) idx[count] = (int32_t)j;
                ++count;
            }
        }
    }
    if (offsets) offsets[n] = (int32_t)count;
    *n_pairs = count;
    return count > cap ? ORC_ERR_NBR_OVERFLOW : ORC_OK;
}

/* One row of the same set, for sampled checks on large systems. */
int orc_neighbor_row(int64_t n, const double *q, const double L[3], double r_list, int64_t i,
                     int32_t *row, int64_t cap, int64_t *count_out)
{
    double rl2 = r_list * r_list;
    double qi[3];
    load_q(q, n, i, qi);
    int64_t count = 0;
    for (int64_t j = 0; j < n; ++j) {
        if (j == i) continue;
        double qj[3], d[3];
        load_q(q, n, j, qj);
        min_image(L, qi, qj, d);
        if (dist2(d) < rl2) {
            if (count < cap) row[count] = (int32_t)j;
            ++count;
        }
    }
    *count_out = count;
    return count > cap ? ORC_ERR_NBR_OVERFLOW : ORC_OK;
}

/* The same set found through a cell grid (cells no smaller than r_list,
 * each distinct neighbouring cell visited once, rows sorted by j).  Used
 * where brute force is too slow; tested against orc_neighbors.            */
static int cmp_i32(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

int orc_neighbors_binned(int64_t n, const double *q, const double L[3], double r_list,
                         int32_t *offsets, int32_t *idx, int64_t cap, int64_t *n_pairs)
{
    if (n < 0 || !(r_list > 0.0)) return ORC_ERR_ARG;
    for (int a = 0; a < 3; ++a)
        if (!(L[a] >= 2.0 * r_list)) return ORC_ERR_BOX_TOO_SMALL;
    int nc[3];
    for (int a = 0; a < 3; ++a) {
        nc[a] = (int)floor(L[a] / (r_list * (1.0 + 1e-9)));
        if (nc[a] < 3) nc[a] = 1;
    }
    int64_t ncell = (int64_t)nc[0] * nc[1] * nc[2];
    int64_t *cell = (int64_t *)malloc(sizeof(int64_t) * (n + 1));
    int64_t *start = (int64_t *)calloc((size_t)(ncell + 1), sizeof(int64_t));
    int64_t *fill = (int64_t *)calloc((size_t)(ncell + 1), sizeof(int64_t));
    int32_t *sorted = (int32_t *)malloc(sizeof(int32_t) * (n + 1));
    for (int64_t i = 0; i < n; ++i) {
        int c3[3];
        for (int a = 0; a < 3; ++a) {
            double u = q[a * n + i] / L[a];
            u = u - floor(u);
            int c = (int)(u * nc[a]);
            if (c >= nc[a]) c = nc[a] - 1;
            if (c < 0) c = 0;
            c3[a] = c;
        }
        cell[i] = ((int64_t)c3[0] * nc[1] + c3[1]) * nc[2] + c3[2];
        start[cell[i] + 1] += 1;
    }
    for (int64_t c = 0; c < ncell; ++c) start[c + 1] += start[c];
    for (int64_t i = 0; i < n; ++i) sorted[start[cell[i]] + fill[cell[i]]++] = (int32_t)i;
    double rl2 = r_list * r_list;
    int64_t count = 0;
    int32_t *row = (int32_t *)malloc(sizeof(int32_t) * (n + 1));
    for (int64_t i = 0; i < n; ++i) {
        if (offsets) offsets[i] = (int32_t)count;
        int64_t ci = cell[i];
        int c3[3] = {(int)(ci / ((int64_t)nc[1] * nc[2])), (int)((ci / nc[2]) % nc[1]), (int)(ci % nc[2])};
        int offs[3][3], noff[3];
        for (int a = 0; a < 3; ++a) {
            noff[a] = 0;
            for (int o = -1; o <= 1; ++o) {
                int v = ((c3[a] + o) % nc[a] + nc[a]) % nc[a];
                int dup = 0;
                for (int t = 0; t < noff[a]; ++t) dup |= offs[a][t] == v;
                if (!dup) offs[a][noff[a]++] = v;
            }
        }
        double qi[3];
        load_q(q, n, i, qi);
        int64_t m = 0;
        for (int ax = 0; ax < noff[0]; ++ax)
            for (int ay = 0; ay < noff[1]; ++ay)
                for (int az = 0; az < noff[2]; ++az) {
                    int64_t c = ((int64_t)offs[0][ax] * nc[1] + offs[1][ay]) * nc[2] + offs[2][az];
                    for (int64_t t = start[c]; t < start[c + 1]; ++t) {
                        int64_t j = sorted[t];
                        if (j == i) continue;
                        double qj[3], d[3];
                        load_q(q, n, j, qj);
                        min_image(L, qi, qj, d);
                        if (dist2(d) < rl2) row[m++] = (int32_t)j;
                    }
                }
        qsort(row, (size_t)m, sizeof(int32_t), cmp_i32);
        for (int64_t t = 0; t < m; ++t) {
            if (idx && count < cap) idx[count] = row[t];
            ++count;
        }
    }
    if (offsets) offsets[n] = (int32_t)count;
    *n_pairs = count;
    free(cell); free(start); free(fill); free(sorted); free(row);
    return count > cap ? ORC_ERR_NBR_OVERFLOW : ORC_OK;
}

/* Bond set for the master equation (Sec. 3: the sum runs over nearest
 * neighbours): j in the neighbour row of i with r < r_bond, on the same
 * sublattice, that sublattice mobile.                                       */
int orc_bonds(int64_t n, const double *q, const double L[3], double r_bond,
              const uint8_t *sublattice, uint32_t mobile_mask,
              const int32_t *nb_off, const int32_t *nb_idx,
              int32_t *offsets, int32_t *idx, int64_t cap, int64_t *n_bonds)
{
    double rb2 = r_bond * r_bond;
    int64_t count = 0;
    for (int64_t i = 0; i < n; ++i) {
        offsets[i] = (int32_t)count;
        int si = sublattice ? sublattice[i] : 0;
        if (!((mobile_mask >> si) & 1u)) continue;
        double qi[3];
        load_q(q, n, i, qi);
        for (int32_t e = nb_off[i]; e < nb_off[i + 1]; ++e) {
            int64_t j = nb_idx[e];
            int sj = sublattice ? sublattice[j] : 0;
            if (sj != si) continue;
            double qj[3], d[3];
            load_q(q, n, j, qj);
            min_image(L, qi, qj, d);
            if (dist2(d) < rb2) {
                if (count < cap) idx[count] = (int32_t)j;
                ++count;
            }
        }
    }
    offsets[n] = (int32_t)count;
    *n_bonds = count;
    return count > cap ? ORC_ERR_NBR_OVERFLOW : ORC_OK;
}

/* ------------------------------------------------------------------ */
/* App. A quadrature for one pair (sites "first" and "second").
 * The pair has N = 2 sites, N_q = 3N = 6 coordinates, M = 2 N_q = 12 nodes at
 * chi = +-r e_m with r^2 = N_q / 2 = 3 and equal normalised weights 1/12.  In
 * physical units q - qbar = sqrt(2) sigma chi (chi = (q - qbar)/(sqrt(2) sigma),
 * sigma the per-component standard deviation), so each node moves one site
 * by +-sqrt(6) sigma along one axis.  With d = q_second - q_first the nodes
 * are d - (+-sqrt6 sigma_first) e_a (first site moved) and
 * d + (+-sqrt6 sigma_second) e_a (second site moved).
 * Node p: disp[p] = the relative displacement vector; which[p] = 0 if the
 * first site moved, 1 if the second; dsig[p] = d(disp[p][axis[p]])/d(sigma).   */
/* ------------------------------------------------------------------ */
void orc_quad_nodes(const double dbar[3], double sigma_first, double sigma_second,
                    double disp[ORC_NODES][3], int32_t which[ORC_NODES],
                    int32_t axis[ORC_NODES], double dsig[ORC_NODES])
{
    const double r = sqrt(3.0);            /* r^2 = N_q/2 = 3 */
    int p = 0;
    for (int site = 0; site < 2; ++site) {
        double sg = site == 0 ? sigma_first : sigma_second;
        /* moving the first site by +u changes d = q2 - q1 by -u */
        double sign_site = site == 0 ? -1.0 : 1.0;
        for (int a = 0; a < 3; ++a) {
            for (int s = 0; s < 2; ++s) {
                double chi = s == 0 ? r : -r;
                double u = sqrt(2.0) * sg * chi;           /* displacement of the site */
                for (int b = 0; b < 3; ++b) disp[p][b] = dbar[b];
                disp[p][a] = dbar[a] + sign_site * u;
                which[p] = site;
                axis[p] = a;
                dsig[p] = sign_site * sqrt(2.0) * chi;     /* d(disp_a)/d(sigma) */
                ++p;
            }
        }
    }
}

/* ------------------------------------------------------------------ */
/* Potential functions (App. B.2, analytic forms with a quintic switch).   */
/* ------------------------------------------------------------------ */
static void switch_fn(const orc_potential *P, double r, double *S, double *dS)
{
    if (r <= P->r_switch) { *S = 1.0; *dS = 0.0; return; }
    if (r >= P->r_cut) { *S = 0.0; *dS = 0.0; return; }
    double w = P->r_cut - P->r_switch;
    double t = (r - P->r_switch) / w;
    double t2 = t * t, t3 = t2 * t, t4 = t3 * t, t5 = t4 * t;
    *S = 1.0 - 10.0 * t3 + 15.0 * t4 - 6.0 * t5;
    *dS = (-30.0 * t2 + 60.0 * t3 - 30.0 * t4) / w;
}

static void expo_fn(double A, double p, double r0, double r, double *v, double *dv)
{
    if (A == 0.0) { *v = 0.0; *dv = 0.0; return; }
    double e = A * exp(-p * (r / r0 - 1.0));
    *v = e;
    *dv = -p / r0 * e;
}

/* phi_kl(r) and its derivative. */
static void phi_fn(const orc_potential *P, int k, int l, double r, double *v, double *dv)
{
    double S, dS;
    switch_fn(P, r, &S, &dS);
    if (P->lj) {
        const double eps = P->lj_eps[k][l], s = P->lj_sigma[k][l];
        const double x6 = pow(s / r, 6.0), x12 = x6 * x6;
        const double e = 4.0 * eps * (x12 - x6);
        const double de = 4.0 * eps * (-12.0 * x12 + 6.0 * x6) / r;
        *v = e * S;
        *dv = de * S + e * dS;
        return;
    }
    if (P->cross_geomean && k != l) {
        /* cross pair = pointwise geometric mean of the two pure pair terms */
        double eu, deu, ew, dew;
        expo_fn(P->phi_A[k][k], P->phi_p[k][k], P->phi_r0[k][k], r, &eu, &deu);
        expo_fn(P->phi_A[l][l], P->phi_p[l][l], P->phi_r0[l][l], r, &ew, &dew);
        double u = eu * S, du = deu * S + eu * dS;
        double w = ew * S, dw = dew * S + ew * dS;
        double g = sqrt(u * w);
        *v = g;
        *dv = g > 0.0 ? (du * w + u * dw) / (2.0 * g) : 0.0;
        return;
    }
    double e, de;
    expo_fn(P->phi_A[k][l], P->phi_p[k][l], P->phi_r0[k][l], r, &e, &de);
    *v = e * S;
    *dv = de * S + e * dS;
}

/* f_kl(r): density at a k-site from an l-neighbour, and its derivative. */
static void f_fn(const orc_potential *P, int k, int l, double r, double *v, double *dv)
{
    double S, dS, e, de;
    switch_fn(P, r, &S, &dS);
    expo_fn(P->f_xi[k][l], P->f_q[k][l], P->f_r0[k][l], r, &e, &de);
    *v = e * S;
    *dv = de * S + e * dS;
}

/* Embedding F_k(rho) = -E_k sqrt(rho) and its first two derivatives. */
static void embed_fn(const orc_potential *P, int k, double rho, double *F, double *dF, double *d2F)
{
    double s = sqrt(rho);
    *F = -P->E[k] * s;
    *dF = -P->E[k] / (2.0 * s);
    *d2F = P->E[k] / (4.0 * rho * s);
}

/* ------------------------------------------------------------------ */
/* Phase average of a function of the pair distance over the 12 nodes, with
 * its derivatives w.r.t. d = q_second - q_first and the two sigmas.
 * kind 0: phi_kl, kind 1: f_kl.                                            */
/* ------------------------------------------------------------------ */
typedef struct {
    double avg;          /* <g> */
    double d_dd[3];      /* d<g>/d(d) : d/dq_second = +, d/dq_first = - */
    double d_dsig[2];    /* d<g>/d(sigma_first), d<g>/d(sigma_second) */
    double stat;         /* g at the mean distance (static point) */
    double stat_dd[3];   /* dg(|d|)/d(d) at the static point */
    int bad;             /* a node closer than ORC_RMIN */
} orc_pair_avg;

static void pair_average(const orc_potential *P, int kind, int k, int l,
                         const double dbar[3], double s_first, double s_second,
                         orc_pair_avg *out)
{
    double disp[ORC_NODES][3], dsig[ORC_NODES];
    int32_t which[ORC_NODES], axis[ORC_NODES];
    orc_quad_nodes(dbar, s_first, s_second, disp, which, axis, dsig);
    memset(out, 0, sizeof(*out));
    const double w = 1.0 / (double)ORC_NODES;
    for (int p = 0; p < ORC_NODES; ++p) {
        double r = sqrt(dist2(disp[p]));
        if (r < ORC_RMIN) out->bad = 1;
        double g, dg;
        if (kind == 0) phi_fn(P, k, l, r, &g, &dg);
        else f_fn(P, k, l, r, &g, &dg);
        out->avg += w * g;
        for (int b = 0; b < 3; ++b) out->d_dd[b] += w * dg * disp[p][b] / r;
        out->d_dsig[which[p]] += w * dg * (disp[p][axis[p]] / r) * dsig[p];
    }
    double r = sqrt(dist2(dbar));
    if (r < ORC_RMIN) out->bad = 1;
    double g, dg;
    if (kind == 0) phi_fn(P, k, l, r, &g, &dg);
    else f_fn(P, k, l, r, &g, &dg);
    out->stat = g;
    for (int b = 0; b < 3; ++b) out->stat_dd[b] = dg * dbar[b] / r;
}

/* Exposed for the quadrature pins. */
double orc_pair_average_value(const orc_potential *P, int kind, int k, int l,
                              const double dbar[3], double s_first, double s_second)
{
    orc_pair_avg a;
    pair_average(P, kind, k, l, dbar, s_first, s_second, &a);
    return a.avg;
}

/* ------------------------------------------------------------------ */
/* Free energy and gradients.
 *
 *   rho_bar_i^k = sum_j sum_l x_jl f_kl(|dbar_ij|)            (static point)
 *   <rho_i^k>   = sum_j sum_l x_jl <f_kl>_ij                  (Eq. EAM-density-substitutional-ave)
 *   e_i^k       = F_k(rho_bar) + F_k'(rho_bar)(<rho> - rho_bar) (Eq. F_taylor_mxe)
 *   <V_i>       = 1/2 sum_j sum_kl x_ik x_jl <phi_kl>_ij + sum_k x_ik e_i^k
 *                                                              (Eq. EAM-Substitutional-ave)
 *   F           = sum_i [<V_i> - 3 kB T_i ln sigma_i + kB T_i (sum_k x_ik ln x_ik + x_iv ln x_iv)]
 *
 * a_i^k = x_ik F_k''(rho_bar)(<rho> - rho_bar) and b_i^k = x_ik F_k'(rho_bar) are
 * the derivatives of sum_k x_ik e_i^k w.r.t. rho_bar_i^k and <rho_i^k>.
 * Outputs: F4 = (E_V, F_vib, F_mix, F); gq [3][n] = dF/dq; gs [n] = dF/dsigma;
 * mu_ex [S][n] = dE_V/dx_ik (vacancy dependent); mu [S][n] = dF/dx_ik (optional);
 * site arrays rho_bar, rho_avg, a, b, e [S][n] (optional).
 * mode 0: everything; mode 1: energies only.                               */
/* ------------------------------------------------------------------ */
int orc_free_energy(const orc_system *sys, const orc_potential *P,
                    const int32_t *nb_off, const int32_t *nb_idx, int mode,
                    double *F4, double *gq, double *gs, double *mu_ex, double *mu,
                    double *rho_bar, double *rho_avg, double *a_out, double *b_out, double *e_out)
{
    const int64_t n = sys->n;
    const int S = sys->S;
    if (S < 1 || S > ORC_MAXS || S != P->n_species) return ORC_ERR_ARG;
    const double *q = sys->q, *sig = sys->sigma, *x = sys->x, *T = sys->T;

    double *rb = (double *)calloc((size_t)(S * n + 1), sizeof(double));
    double *ra = (double *)calloc((size_t)(S * n + 1), sizeof(double));
    double *A = (double *)calloc((size_t)(S * n + 1), sizeof(double));
    double *B = (double *)calloc((size_t)(S * n + 1), sizeof(double));
    double *e = (double *)calloc((size_t)(S * n + 1), sizeof(double));
    double *site_EV = (double *)calloc((size_t)(n + 1), sizeof(double));
    double *site_vib = (double *)calloc((size_t)(n + 1), sizeof(double));
    double *site_mix = (double *)calloc((size_t)(n + 1), sizeof(double));
    int geometry = 0;

    /* Pass 1: densities at every site, then the embedding terms. */
#pragma omp parallel for schedule(dynamic, 64) reduction(| : geometry)
    for (int64_t i = 0; i < n; ++i) {
        double qi[3];
        load_q(q, n, i, qi);
        for (int k = 0; k < S; ++k) {
            double sb = 0.0, sa = 0.0;
            for (int32_t t = nb_off[i]; t < nb_off[i + 1]; ++t) {
                int64_t j = nb_idx[t];
                double qj[3], d[3];
                load_q(q, n, j, qj);
                min_image(sys->L, qi, qj, d);
                for (int l = 0; l < S; ++l) {
                    orc_pair_avg pa;
                    pair_average(P, 1, k, l, d, sig[i], sig[j], &pa);
                    geometry |= pa.bad;
                    sb += x[l * n + j] * pa.stat;
                    sa += x[l * n + j] * pa.avg;
                }
            }
            rb[k * n + i] = sb;
            ra[k * n + i] = sa;
            if (P->E[k] == 0.0) {  /* no embedding energy for this element */
                e[k * n + i] = A[k * n + i] = B[k * n + i] = 0.0;
                continue;
            }
            if (!(sb > ORC_RHO_MIN)) { geometry = 1; continue; }
            double F, dF, d2F;
            embed_fn(P, k, sb, &F, &dF, &d2F);
            e[k * n + i] = F + dF * (sa - sb);
            A[k * n + i] = x[k * n + i] * d2F * (sa - sb);
            B[k * n + i] = x[k * n + i] * dF;
        }
    }
    int status = geometry ? ORC_ERR_GEOMETRY : ORC_OK;

    /* Pass 2: site energies and, in mode 0, the three gradients. */
    if (status == ORC_OK) {
#pragma omp parallel for schedule(dynamic, 64)
        for (int64_t i = 0; i < n; ++i) {
            double qi[3];
            load_q(q, n, i, qi);
            double Epair = 0.0, g[3] = {0.0, 0.0, 0.0}, gsig = 0.0;
            double mu_i[ORC_MAXS] = {0.0, 0.0, 0.0, 0.0};
            for (int32_t t = nb_off[i]; t < nb_off[i + 1]; ++t) {
                int64_t j = nb_idx[t];
                double qj[3], dij[3], dji[3];
                load_q(q, n, j, qj);
                min_image(sys->L, qi, qj, dij);   /* q_j - q_i */
                min_image(sys->L, qj, qi, dji);   /* q_i - q_j */
                for (int k = 0; k < S; ++k) {
                    for (int l = 0; l < S; ++l) {
                        /* pair (i, j): site i first */
                        orc_pair_avg phi_ij, f_ij;
                        pair_average(P, 0, k, l, dij, sig[i], sig[j], &phi_ij);
                        double wij = x[k * n + i] * x[l * n + j];
                        Epair += 0.5 * wij * phi_ij.avg;
                        if (mode == 1) continue;
                        pair_average(P, 1, k, l, dij, sig[i], sig[j], &f_ij);
                        /* pair (j, i): site j first, species k at j and l at i */
                        orc_pair_avg phi_ji, f_ji;
                        pair_average(P, 0, k, l, dji, sig[j], sig[i], &phi_ji);
                        pair_average(P, 1, k, l, dji, sig[j], sig[i], &f_ji);
                        double wji = x[k * n + j] * x[l * n + i];
                        double aik = A[k * n + i], bik = B[k * n + i];
                        double ajk = A[k * n + j], bjk = B[k * n + j];
                        double xjl = x[l * n + j], xil = x[l * n + i];
                        for (int c = 0; c < 3; ++c) {
                            /* q_i is the first site of (i,j): d/dq_i = -d/dd;
                               q_i is the second site of (j,i): d/dq_i = +d/dd */
                            g[c] += 0.5 * wij * (-phi_ij.d_dd[c]) + 0.5 * wji * phi_ji.d_dd[c];
                            g[c] += aik * xjl * (-f_ij.stat_dd[c]) + bik * xjl * (-f_ij.d_dd[c]);
                            g[c] += ajk * xil * f_ji.stat_dd[c] + bjk * xil * f_ji.d_dd[c];
                        }
                        gsig += 0.5 * wij * phi_ij.d_dsig[0] + 0.5 * wji * phi_ji.d_dsig[1];
                        gsig += bik * xjl * f_ij.d_dsig[0] + bjk * xil * f_ji.d_dsig[1];
                        /* d/dx_ik: pair term from (i,j) with k at i, and from (j,i) with
                           k at i in the second slot (species index l there). */
                        mu_i[k] += 0.5 * xjl * phi_ij.avg;
                        mu_i[l] += 0.5 * x[k * n + j] * phi_ji.avg;
                        /* d/dx_il through the densities at j: rho_j^k includes x_il f_kl(r_ji) */
                        mu_i[l] += ajk * f_ji.stat + bjk * f_ji.avg;
                    }
                }
            }
            double emb = 0.0;
            for (int k = 0; k < S; ++k) emb += x[k * n + i] * e[k * n + i];
            site_EV[i] = Epair + emb;
            double kT = ORC_KB * T[i];
            site_vib[i] = -3.0 * kT * log(sig[i]);
            double xv = 1.0, mix = 0.0;
            for (int k = 0; k < S; ++k) {
                double xk = x[k * n + i];
                xv -= xk;
                if (xk > 0.0) mix += xk * log(xk);
            }
            if (xv > 0.0) mix += xv * log(xv);
            site_mix[i] = kT * mix;
            if (mode == 1) continue;
            for (int c = 0; c < 3; ++c) gq[c * n + i] = g[c];
            gs[i] = gsig - 3.0 * kT / sig[i];
            for (int k = 0; k < S; ++k) {
                double m = mu_i[k] + e[k * n + i];
                mu_ex[k * n + i] = m;
                if (mu) {
                    double lx = log(fmax(x[k * n + i], ORC_LOG_FLOOR));
                    double lv = log(fmax(xv, ORC_LOG_FLOOR));
                    mu[k * n + i] = m + kT * (lx - lv);
                }
            }
        }
        double EV = pairwise_sum(site_EV, n);
        double Fv = pairwise_sum(site_vib, n);
        double Fm = pairwise_sum(site_mix, n);
        F4[0] = EV;
        F4[1] = Fv;
        F4[2] = Fm;
        F4[3] = EV + Fv + Fm;
        if (!isfinite(F4[3])) status = ORC_ERR_NONFINITE;
        if (mode == 0 && status == ORC_OK) {
            for (int64_t i = 0; i < 3 * n && status == ORC_OK; ++i)
                if (!isfinite(gq[i])) status = ORC_ERR_NONFINITE;
            for (int64_t i = 0; i < n && status == ORC_OK; ++i)
                if (!isfinite(gs[i])) status = ORC_ERR_NONFINITE;
            for (int64_t i = 0; i < S * n && status == ORC_OK; ++i)
                if (!isfinite(mu_ex[i])) status = ORC_ERR_NONFINITE;
        }
    }
    if (rho_bar) memcpy(rho_bar, rb, sizeof(double) * S * n);
    if (rho_avg) memcpy(rho_avg, ra, sizeof(double) * S * n);
    if (a_out) memcpy(a_out, A, sizeof(double) * S * n);
    if (b_out) memcpy(b_out, B, sizeof(double) * S * n);
    if (e_out) memcpy(e_out, e, sizeof(double) * S * n);
    free(rb); free(ra); free(A); free(B); free(e);
    free(site_EV); free(site_vib); free(site_mix);
    return status;
}

/* ------------------------------------------------------------------ */
/* Exact phase average of the embedding term (App. B.2: the third-degree rule
 * of App. A applied to the many-body function F_k(rho_i), which the paper then
 * replaces by its Taylor form, Eq. F_taylor_mxe).
 *
 * The rule of site i covers the N sites "inside the potential cut-off
 * radius": i itself and every neighbour j with |qbar_j - qbar_i| < r_cut
 * (the set J_i).  The many-body function is
 *     F_k(rho_i^k),  rho_i^k = sum_{j in J_i} sum_l x_jl f_kl(|q_j - q_i|),
 * a function of N_q = 3N coordinates.  The rule has M = 2 N_q nodes
 * chi = +-r e_m, r^2 = N_q / 2, each with normalised weight 1/M; in physical
 * units q - qbar = sqrt(2) sigma chi, so each node moves ONE site s of the
 * rule by +-sigma_s sqrt(N_q) along one axis and leaves the others at their
 * means:
 *     <F_k(rho_i^k)> = (1/M) sum_nodes F_k(rho_i^k(node)).
 * The free energy is that of orc_free_energy with every embedding term
 * e_i^k replaced by <F_k(rho_i^k)>:
 *     E_V = sum_i [1/2 sum_j sum_kl x_ik x_jl <phi_kl>_ij + sum_k x_ik <F_k(rho_i^k)>].
 * Gradients, written out from the node sum (the rule's membership and N are
 * held fixed: they change only where a mean distance crosses r_cut):
 *   d/dq_j of F_k(rho(node)) = F_k'(rho(node)) sum_l x_jl f_kl'(r_ij) u_ij  (j in J_i),
 *   and minus the sum of these for q_i (u_ij = (q_j - q_i)/r_ij at the node);
 *   d/dsigma_s: the moved coordinate of a node moving s is qbar_s +- sigma_s
 *   sqrt(N_q), so d/dsigma_s = +-sqrt(N_q) times the derivative along it;
 *   d/dx_jl = x_ik (1/M) sum_nodes F_k'(rho(node)) f_kl(r_ij(node)),
 *   d/dx_ik = <F_k(rho_i^k)>.
 * GEOMETRY if a node distance is below ORC_RMIN or rho(node) <= ORC_RHO_MIN for
 * an occupied element with an embedding energy.  Each thread accumulates the
 * contributions of its sites in its own buffer; the buffers are added in
 * thread order.  Outputs as orc_free_energy; emb_out [S][n] (optional)
 * receives <F_k(rho_i^k)>.
 */
/* ------------------------------------------------------------------ */
int orc_free_energy_exact(const orc_system *sys, const orc_potential *P,
                          const int32_t *nb_off, const int32_t *nb_idx,
                          double *F4, double *gq, double *gs, double *mu_ex, double *mu, double *emb_out)
{
    const int64_t n = sys->n;
    const int S = sys->S;
    if (S < 1 || S > ORC_MAXS || S != P->n_species) return ORC_ERR_ARG;
    const double *q = sys->q, *sig = sys->sigma, *x = sys->x, *T = sys->T;

    /* the pair terms, F_vib and F_mix: the same free energy with no embedding */
    orc_potential P0 = *P;
    for (int k = 0; k < ORC_MAXS; ++k) P0.E[k] = 0.0;
    int status = orc_free_energy(sys, &P0, nb_off, nb_idx, 0, F4, gq, gs, mu_ex, NULL,
                                 NULL, NULL, NULL, NULL, NULL);
    if (status != ORC_OK && status != ORC_ERR_NONFINITE) return status;

    int nthr = 1;
#ifdef _OPENMP
    nthr = omp_get_max_threads();
#endif
    const int64_t width = 4 + S;  /* per site: dF/dq (3), dF/dsigma, dE_V/dx (S) */
    double *acc = (double *)calloc((size_t)(nthr * n * width + 1), sizeof(double));
    double *emb = (double *)calloc((size_t)(S * n + 1), sizeof(double));
    double *site_emb = (double *)calloc((size_t)(n + 1), sizeof(double));
    int geometry = 0;
#pragma omp parallel reduction(| : geometry)
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double *my = acc + (int64_t)tid * n * width;
        int cap = 256;
        int64_t *J = (int64_t *)malloc(sizeof(int64_t) * cap);
        double *dbar = (double *)malloc(sizeof(double) * 3 * cap);
#pragma omp for schedule(static)
        for (int64_t i = 0; i < n; ++i) {
            double qi[3];
            load_q(q, n, i, qi);
            /* the rule's sites: i and its neighbours inside r_cut */
            int m = 0;
            for (int32_t t = nb_off[i]; t < nb_off[i + 1]; ++t) {
                int64_t j = nb_idx[t];
                double qj[3], d[3];
                load_q(q, n, j, qj);
                min_image(sys->L, qi, qj, d);
                if (!(sqrt(dist2(d)) < P->r_cut)) continue;
                if (m == cap) {
                    cap *= 2;
                    J = (int64_t *)realloc(J, sizeof(int64_t) * cap);
                    dbar = (double *)realloc(dbar, sizeof(double) * 3 * cap);
                }
                J[m] = j;
                for (int c = 0; c < 3; ++c) dbar[3 * m + c] = d[c];
                ++m;
            }
            const int N = m + 1;
            const double Nq = 3.0 * N;
            const int M = 2 * 3 * N;
            const double w = 1.0 / (double)M;
            const double hs = sqrt(Nq);   /* displacement / sigma of a node */
            double e_site = 0.0;
            for (int k = 0; k < S; ++k) {
                double xik = x[k * n + i];
                if (P->E[k] == 0.0) { emb[k * n + i] = 0.0; continue; }
                double Fsum = 0.0;
                /* node (s, a, pm): site s of the rule (0 = i, 1..m = J[s-1]) moved by
                   pm sigma_s sqrt(N_q) along axis a */
                for (int s_ = 0; s_ <= m; ++s_) {
                    for (int a = 0; a < 3; ++a) {
                        for (int pm = -1; pm <= 1; pm += 2) {
                            double shift_i[3] = {0.0, 0.0, 0.0}, shift_s[3] = {0.0, 0.0, 0.0};
                            int64_t site_s = (s_ == 0) ? i : J[s_ - 1];
                            double h = pm * sig[site_s] * hs;
                            if (s_ == 0) shift_i[a] = h;
                            else shift_s[a] = h;
                            /* density at the node */
                            double rho = 0.0;
                            for (int jj = 0; jj < m; ++jj) {
                                int64_t j = J[jj];
                                double v[3];
                                for (int c = 0; c < 3; ++c)
                                    v[c] = dbar[3 * jj + c] + (s_ == jj + 1 ? shift_s[c] : 0.0) - shift_i[c];
                                double r = sqrt(dist2(v));
                                if (r < ORC_RMIN) geometry = 1;
                                for (int l = 0; l < S; ++l) {
                                    double f, df;
                                    f_fn(P, k, l, r, &f, &df);
                                    rho += x[l * n + j] * f;
                                }
                            }
                            if (!(rho > ORC_RHO_MIN)) {
                                if (xik > 0.0) geometry = 1;
                                continue;
                            }
                            double F, dF, d2F;
                            embed_fn(P, k, rho, &F, &dF, &d2F);
                            Fsum += F;
                            /* derivatives of x_ik F_k(rho(node)) / M */
                            double c0 = xik * dF * w;
                            for (int jj = 0; jj < m; ++jj) {
                                int64_t j = J[jj];
                                double v[3];
                                for (int c = 0; c < 3; ++c)
                                    v[c] = dbar[3 * jj + c] + (s_ == jj + 1 ? shift_s[c] : 0.0) - shift_i[c];
                                double r = sqrt(dist2(v));
                                double gj = 0.0;
                                for (int l = 0; l < S; ++l) {
                                    double f, df;
                                    f_fn(P, k, l, r, &f, &df);
                                    gj += x[l * n + j] * df;
                                    /* dE_V/dx_jl through rho_i^k */
                                    my[j * width + 4 + l] += c0 * f;
                                }
                                for (int c = 0; c < 3; ++c) {
                                    double gc = c0 * gj * v[c] / r;
                                    my[j * width + c] += gc;   /* d/dq_j */
                                    my[i * width + c] -= gc;   /* d/dq_i */
                                }
                                /* d/dsigma of the moved site: along axis a, +-sqrt(N_q) */
                                double ga = c0 * gj * v[a] / r;
                                if (s_ == 0) my[i * width + 3] -= ga * pm * hs;
                                else if (s_ == jj + 1) my[j * width + 3] += ga * pm * hs;
                            }
                        }
                    }
                }
                emb[k * n + i] = Fsum * w;
                e_site += xik * emb[k * n + i];
                /* dE_V/dx_ik through the factor x_ik */
                my[i * width + 4 + k] += emb[k * n + i];
            }
            site_emb[i] = e_site;
        }
        free(J);
        free(dbar);
    }
    if (geometry) {
        free(acc); free(emb); free(site_emb);
        return ORC_ERR_GEOMETRY;
    }
    for (int t = 1; t < nthr; ++t)
        for (int64_t v = 0; v < n * width; ++v) acc[v] += acc[(int64_t)t * n * width + v];
    double Eemb = pairwise_sum(site_emb, n);
    F4[0] += Eemb;
    F4[3] = F4[0] + F4[1] + F4[2];
    status = isfinite(F4[3]) ? ORC_OK : ORC_ERR_NONFINITE;
    for (int64_t i = 0; i < n; ++i) {
        for (int c = 0; c < 3; ++c) gq[c * n + i] += acc[i * width + c];
        gs[i] += acc[i * width + 3];
        double xv = 1.0;
        for (int k = 0; k < S; ++k) xv -= x[k * n + i];
        for (int k = 0; k < S; ++k) {
            mu_ex[k * n + i] += acc[i * width + 4 + k];
            if (mu) {
                double kT = ORC_KB * T[i];
                double lx = log(fmax(x[k * n + i], ORC_LOG_FLOOR));
                double lv = log(fmax(xv, ORC_LOG_FLOOR));
                mu[k * n + i] = mu_ex[k * n + i] + kT * (lx - lv);
            }
        }
    }
    for (int64_t v = 0; v < 3 * n && status == ORC_OK; ++v)
        if (!isfinite(gq[v])) status = ORC_ERR_NONFINITE;
    for (int64_t v = 0; v < n && status == ORC_OK; ++v)
        if (!isfinite(gs[v])) status = ORC_ERR_NONFINITE;
    if (emb_out) memcpy(emb_out, emb, sizeof(double) * S * n);
    free(acc); free(emb); free(site_emb);
    return status;
}

/* ------------------------------------------------------------------ */
/* One forward-Euler step of the master equation (Eq. MassTransport,
 * tau_r = 0), in the reading used throughout this project:
 *   rate of the hop i -> j for species k:
 *     J_{i->j} = nu0 exp(-beta_i Qm) x_ik x_jv exp(beta_i (mu_ik - mu_jk))
 *   (origin-site beta as in the exponents of Eq. MassTransport, the sign that
 *   sends mass down the chemical-potential difference, mu = the excess
 *   chemical potential dE_V/dx, and (1 - x_j) read as the vacancy fraction).
 *   dx_ik/dt = sum_{j in bonds(i)} (J_{j->i} - J_{i->j});  x' = x + dt dx/dt.
 * x is updated in place only if every x'_ik >= -tol and sum_k x'_ik <= 1 + tol.
 */
/* ------------------------------------------------------------------ */
int orc_diffuse_step_res(int64_t n, int S, double *x, const double *T, const double *mu_ex,
                         const int32_t *b_off, const int32_t *b_idx, double dt, double nu0, double Qm,
                         const uint8_t *fix_x_mask, const double *fix_x_value,
                         const uint8_t *fix_mu_mask, const double *fix_mu_value)
{
    /* Reservoirs (Sec. 4: fix setchemicalpotential, fix setatomicfraction):
       a site in the chemical-potential group enters every rate with the held
       value in place of its computed mu; a site in the molar-fraction group
       has its x set to the held value after the Euler step. */
    double *mu = (double *)malloc(sizeof(double) * (size_t)(S * n + 1));
    for (int k = 0; k < S; ++k)
        for (int64_t i = 0; i < n; ++i)
            mu[k * n + i] = (fix_mu_mask && fix_mu_mask[i]) ? fix_mu_value[k * n + i] : mu_ex[k * n + i];
    double *xn = (double *)malloc(sizeof(double) * (size_t)(S * n + 1));
    int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad)
    for (int64_t i = 0; i < n; ++i) {
        double beta_i = 1.0 / (ORC_KB * T[i]);
        double xiv = 1.0;
        for (int k = 0; k < S; ++k) xiv -= x[k * n + i];
        double tot = 0.0;
        for (int k = 0; k < S; ++k) {
            double rate = 0.0;
            for (int32_t t = b_off[i]; t < b_off[i + 1]; ++t) {
                int64_t j = b_idx[t];
                double beta_j = 1.0 / (ORC_KB * T[j]);
                double xjv = 1.0;
                for (int kk = 0; kk < S; ++kk) xjv -= x[kk * n + j];
                double Dij = nu0 * exp(-beta_i * Qm);
                double Dji = nu0 * exp(-beta_j * Qm);
                double out_ij = Dij * x[k * n + i] * xjv * exp(beta_i * (mu[k * n + i] - mu[k * n + j]));
                double in_ji = Dji * x[k * n + j] * xiv * exp(beta_j * (mu[k * n + j] - mu[k * n + i]));
                rate += in_ji - out_ij;
            }
            double v = x[k * n + i] + dt * rate;
            if (fix_x_mask && fix_x_mask[i]) v = fix_x_value[k * n + i];
            xn[k * n + i] = v;
            tot += v;
            if (!(v >= -ORC_X_TOL)) bad = 1;
        }
        if (!(tot <= 1.0 + ORC_X_TOL)) bad = 1;
    }
    if (!bad) memcpy(x, xn, sizeof(double) * (size_t)(S * n));
    free(xn);
    free(mu);
    return bad ? ORC_ERR_X_RANGE : ORC_OK;
}

int orc_diffuse_step(int64_t n, int S, double *x, const double *T, const double *mu_ex,
                     const int32_t *b_off, const int32_t *b_idx,
                     double dt, double nu0, double Qm)
{
    return orc_diffuse_step_res(n, S, x, T, mu_ex, b_off, b_idx, dt, nu0, Qm, NULL, NULL, NULL, NULL);
}

/* ------------------------------------------------------------------ */
/* Variants of the transport step (Sec. 3, Eq. Transport and Eq. MassTransport).
 *
 * Host exchange (host >= 0): the exchange partner of every species k != host
 * is the host species instead of the vacancy, as in a binary alloy without
 * vacancies where x and 1 - x are the two species of Eq. MassTransport:
 *   J^k_{i->j} = D_i x_ik x_j,host exp(beta_i (m_ik - m_jk)),
 *   m_k = mu_k - mu_host (the chemical potential of exchanging a host atom
 *   for a k atom), and every k atom leaving i is replaced by a host atom:
 *   R_ik = sum_j (J^k_{j->i} - J^k_{i->j}),  R_i,host = -sum_{k != host} R_ik.
 * host < 0 is the vacancy-mediated law of orc_diffuse_step.
 *
 * Ballistic term (tau > 0): tau d2x/dt2 + dx/dt = R.  Written as dx/dt = v,
 * tau dv/dt = R - v, and integrated over one step with R held at its value
 * at the start of the step (the analogue of the explicit Euler step):
 *   v' = R + (v - R) e,    x' = x + dt R + tau (v - R)(1 - e),  e = exp(-dt/tau).
 * tau = 0 is the Euler step x' = x + dt R (v, if given, becomes R).
 * The range rule of orc_diffuse_step applies to x'; on failure x and v are
 * unchanged.                                                              */
/* ------------------------------------------------------------------ */
int orc_transport_step(int64_t n, int S, double *x, const double *T, const double *mu_ex,
                       const int32_t *b_off, const int32_t *b_idx, double dt, double nu0, double Qm,
                       int host, double tau, double *v)
{
    if (host >= S) return ORC_ERR_ARG;
    if (tau > 0.0 && !v) return ORC_ERR_ARG;
    double *R = (double *)calloc((size_t)(S * n + 1), sizeof(double));
    double *xn = (double *)malloc(sizeof(double) * (size_t)(S * n + 1));
    double *vn = (double *)malloc(sizeof(double) * (size_t)(S * n + 1));
    int bad = 0;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        const double beta_i = 1.0 / (ORC_KB * T[i]);
        const double Di = nu0 * exp(-beta_i * Qm);
        double part_i = 1.0;                      /* vacancy fraction, or the host's */
        if (host < 0) {
            for (int k = 0; k < S; ++k) part_i -= x[k * n + i];
        } else {
            part_i = x[host * n + i];
        }
        for (int k = 0; k < S; ++k) {
            if (k == host) continue;
            double rate = 0.0;
            for (int32_t t = b_off[i]; t < b_off[i + 1]; ++t) {
                const int64_t j = b_idx[t];
                const double beta_j = 1.0 / (ORC_KB * T[j]);
                const double Dj = nu0 * exp(-beta_j * Qm);
                double part_j = 1.0;
                if (host < 0) {
                    for (int kk = 0; kk < S; ++kk) part_j -= x[kk * n + j];
                } else {
                    part_j = x[host * n + j];
                }
                double mi = mu_ex[k * n + i], mj = mu_ex[k * n + j];
                if (host >= 0) {
                    mi -= mu_ex[host * n + i];
                    mj -= mu_ex[host * n + j];
                }
                const double out_ij = Di * x[k * n + i] * part_j * exp(beta_i * (mi - mj));
                const double in_ji = Dj * x[k * n + j] * part_i * exp(beta_j * (mj - mi));
                rate += in_ji - out_ij;
            }
            R[k * n + i] = rate;
        }
        if (host >= 0) {
            double r = 0.0;
            for (int k = 0; k < S; ++k)
                if (k != host) r -= R[k * n + i];
            R[host * n + i] = r;
        }
    }
#pragma omp parallel for schedule(static) reduction(| : bad)
    for (int64_t i = 0; i < n; ++i) {
        double tot = 0.0;
        for (int k = 0; k < S; ++k) {
            const int64_t a = k * n + i;
            double xv, vv;
            if (tau > 0.0) {
                const double e = exp(-dt / tau);
                xv = x[a] + dt * R[a] + tau * (v[a] - R[a]) * (1.0 - e);
                vv = R[a] + (v[a] - R[a]) * e;
            } else {
                xv = x[a] + dt * R[a];
                vv = R[a];
            }
            xn[a] = xv;
            vn[a] = vv;
            tot += xv;
            if (!(xv >= -ORC_X_TOL)) bad = 1;
        }
        if (!(tot <= 1.0 + ORC_X_TOL)) bad = 1;
    }
    if (!bad) {
        memcpy(x, xn, sizeof(double) * (size_t)(S * n));
        if (v) memcpy(v, vn, sizeof(double) * (size_t)(S * n));
    }
    free(R);
    free(xn);
    free(vn);
    return bad ? ORC_ERR_X_RANGE : ORC_OK;
}

/* ------------------------------------------------------------------ */
/* FIRE relaxation of (q, sigma) at fixed x (Bitzek et al. 2006), in the one
 * variant this project fixes for both implementations:
 *   y = (q, sigma), force f = -(dF/dq, dF/dsigma), unit masses, v = 0, dt = dt0,
 *   alpha = alpha0, n_pos = 0.  Iteration it = 0, 1, ...:
 *     1. evaluate f(y) (neighbour sets rebuilt from scratch every iteration);
 *        fmax = max_i max(|dF/dq_i|_2, |dF/dsigma_i|); stop if fmax <= ftol
 *     2. stop with NO_CONVERGE if it == max_iter
 *     3. if it > 0: P = f.v; P > 0: n_pos += 1, and if n_pos > n_min
 *        dt = min(f_inc dt, dt_max), alpha = f_alpha alpha;
 *        P <= 0: n_pos = 0, dt = f_dec dt, alpha = alpha0, v = 0
 *     4. v = v + dt f;  v = (1 - alpha) v + alpha |v| f / |f|  (global norms)
 *     5. y = y + dt v;  sigma is kept in [sigma_min, sigma_max]: a sigma that
 *        leaves the box is set to the bound and its velocity to zero
 *   The sigma force is projected on the box (zero where a bound blocks it)
 *   in fmax, P, |f| and the update.  sigma_max (default: none) bounds the
 *   width of a site whose occupied fraction is zero: the literal free energy
 *   gives such a site -3 kB T ln sigma and nothing else, so its width would
 *   grow without bound.  Global dot products and norms are pairwise sums.
 * On GEOMETRY / NONFINITE the input state is restored.                   */
/* ------------------------------------------------------------------ */
/* One FIRE update (Bitzek et al. 2006) of y = (q, sigma) from the forces
 * f = (-gq, fs) (fs: the sigma force projected on [s_lo, s_hi]) at iteration
 * `it`, in this order: power check P = f.v (it > 0): P > 0 counts a good step
 * and, after n_min of them, raises dt (to dt_max at most) and lowers alpha;
 * P <= 0 halves dt, resets alpha and zeroes v.  Then the semi-implicit Euler
 * kick v += dt f, the mixing v = (1 - alpha) v + alpha |v| f / |f| (global
 * norms), and the drift y += dt v; a sigma leaving the box is set to the
 * bound with its velocity zeroed.  tmp: n doubles of scratch.              */
typedef struct {
    double dt, alpha;
    int n_pos;
} orc_fire_state;

static void fire_update(int64_t n, double *q, double *sigma, double *vq, double *vs, const double *gq,
                        const double *fs, double *tmp, int it, orc_fire_state *st, const orc_fire *fp,
                        double s_lo, double s_hi)
{
    if (it > 0) {
        for (int64_t i = 0; i < n; ++i)
            tmp[i] = -(gq[i] * vq[i] + gq[n + i] * vq[n + i] + gq[2 * n + i] * vq[2 * n + i]) + fs[i] * vs[i];
        double Pw = pairwise_sum(tmp, n);
        if (Pw > 0.0) {
            st->n_pos += 1;
            if (st->n_pos > fp->n_min) {
                st->dt = fmin(st->dt * fp->f_inc, fp->dt_max);
                st->alpha = st->alpha * fp->f_alpha;
            }
        } else {
            st->n_pos = 0;
            st->dt = st->dt * fp->f_dec;
            st->alpha = fp->alpha0;
            memset(vq, 0, sizeof(double) * 3 * n);
            memset(vs, 0, sizeof(double) * n);
        }
    }
    for (int64_t i = 0; i < n; ++i) {
        for (int c = 0; c < 3; ++c) vq[c * n + i] += st->dt * (-gq[c * n + i]);
        vs[i] += st->dt * fs[i];
    }
    for (int64_t i = 0; i < n; ++i)
        tmp[i] = vq[i] * vq[i] + vq[n + i] * vq[n + i] + vq[2 * n + i] * vq[2 * n + i] + vs[i] * vs[i];
    double vnorm = sqrt(pairwise_sum(tmp, n));
    for (int64_t i = 0; i < n; ++i)
        tmp[i] = gq[i] * gq[i] + gq[n + i] * gq[n + i] + gq[2 * n + i] * gq[2 * n + i] + fs[i] * fs[i];
    double fnorm = sqrt(pairwise_sum(tmp, n));
    double mix = fnorm > 0.0 ? st->alpha * vnorm / fnorm : 0.0;
    for (int64_t i = 0; i < n; ++i) {
        for (int c = 0; c < 3; ++c)
            vq[c * n + i] = (1.0 - st->alpha) * vq[c * n + i] + mix * (-gq[c * n + i]);
        vs[i] = (1.0 - st->alpha) * vs[i] + mix * fs[i];
    }
    for (int64_t i = 0; i < n; ++i) {
        for (int c = 0; c < 3; ++c) q[c * n + i] += st->dt * vq[c * n + i];
        double sn = sigma[i] + st->dt * vs[i];
        if (sn < s_lo || sn > s_hi) {
            sn = sn < s_lo ? s_lo : s_hi;
            vs[i] = 0.0;
        }
        sigma[i] = sn;
    }
}

/* FIRE on the separable quadratic F = 1/2 sum_c kq_c q_c^2 over the 3n
 * coordinates q (sigma fixed at 1 with no force), with the update above:
 * the trajectory (iters + 1 rows of 3n positions, the start first) pins the
 * step order of the relaxation on a case worked out by hand.               */
void orc_fire_quadratic(int64_t n, const double *kq, double *q, int iters, const orc_fire *fp, double *traj)
{
    double *sigma = (double *)malloc(sizeof(double) * n);
    double *vq = (double *)calloc(3 * n, sizeof(double));
    double *vs = (double *)calloc(n, sizeof(double));
    double *gq = (double *)malloc(sizeof(double) * 3 * n);
    double *fs = (double *)calloc(n, sizeof(double));
    double *tmp = (double *)malloc(sizeof(double) * n);
    for (int64_t i = 0; i < n; ++i) sigma[i] = 1.0;
    orc_fire_state st = {fp->dt0, fp->alpha0, 0};
    memcpy(traj, q, sizeof(double) * 3 * n);
    for (int it = 0; it < iters; ++it) {
        for (int64_t c = 0; c < 3 * n; ++c) gq[c] = kq[c] * q[c];
        fire_update(n, q, sigma, vq, vs, gq, fs, tmp, it, &st, fp, ORC_SIGMA_MIN, INFINITY);
        memcpy(traj + (int64_t)(it + 1) * 3 * n, q, sizeof(double) * 3 * n);
    }
    free(sigma); free(vq); free(vs); free(gq); free(fs); free(tmp);
}

int orc_relax(orc_system *sys_in, double *q, double *sigma, const orc_potential *P,
              double r_list, double ftol, int max_iter, const orc_fire *fp,
              int *iters_out, double *fmax_out, int exact_embedding)
{
    const int64_t n = sys_in->n;
    const int S = sys_in->S;
    orc_system sys = *sys_in;
    sys.q = q;
    sys.sigma = sigma;
    double *q0 = (double *)malloc(sizeof(double) * 3 * n);
    double *s0 = (double *)malloc(sizeof(double) * n);
    memcpy(q0, q, sizeof(double) * 3 * n);
    memcpy(s0, sigma, sizeof(double) * n);
    double *vq = (double *)calloc(3 * n, sizeof(double));
    double *vs = (double *)calloc(n, sizeof(double));
    double *gq = (double *)malloc(sizeof(double) * 3 * n);
    double *gs = (double *)malloc(sizeof(double) * n);
    double *mu_ex = (double *)malloc(sizeof(double) * S * n);
    double *tmp = (double *)malloc(sizeof(double) * n);
    int32_t *off = (int32_t *)malloc(sizeof(int32_t) * (n + 1));
    int64_t cap = 64 * n + 64, npairs = 0;
    int32_t *idx = (int32_t *)malloc(sizeof(int32_t) * cap);
    orc_fire_state fst = {fp->dt0, fp->alpha0, 0};
    double F4[4];
    const double s_lo = ORC_SIGMA_MIN;
    const double s_hi = (fp->sigma_max > 0.0) ? fp->sigma_max : INFINITY;
    double *fs = (double *)malloc(sizeof(double) * n);
    int status = ORC_OK, it = 0;
    double fmx = 0.0;
    for (it = 0;; ++it) {
        /* neighbour sets for the current widths: r_list covers r_cut + sqrt6 max sigma */
        double smax = 0.0;
        for (int64_t i = 0; i < n; ++i) smax = fmax(smax, sigma[i]);
        double rl = fmax(r_list, P->r_cut + sqrt(6.0) * smax + 1e-9);
        for (;;) {
            status = orc_neighbors_binned(n, q, sys.L, rl, off, idx, cap, &npairs);
            if (status != ORC_ERR_NBR_OVERFLOW) break;
            cap = npairs + 64;
            idx = (int32_t *)realloc(idx, sizeof(int32_t) * cap);
        }
        if (status != ORC_OK) break;
        /* the Taylor form of the embedding average, or the exact rule */
        if (exact_embedding)
            status = orc_free_energy_exact(&sys, P, off, idx, F4, gq, gs, mu_ex, NULL, NULL);
        else
            status = orc_free_energy(&sys, P, off, idx, 0, F4, gq, gs, mu_ex, NULL,
                                     NULL, NULL, NULL, NULL, NULL);
        if (status != ORC_OK) break;
        fmx = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            fs[i] = proj_fsig(gs[i], sigma[i], s_lo, s_hi);
            double gqi = sqrt(gq[i] * gq[i] + gq[n + i] * gq[n + i] + gq[2 * n + i] * gq[2 * n + i]);
            fmx = fmax(fmx, fmax(gqi, fabs(fs[i])));
        }
        if (fmx <= ftol) break;
        if (it == max_iter) { status = ORC_ERR_NO_CONVERGE; break; }
        fire_update(n, q, sigma, vq, vs, gq, fs, tmp, it, &fst, fp, s_lo, s_hi);
    }
    if (status != ORC_OK && status != ORC_ERR_NO_CONVERGE) {
        memcpy(q, q0, sizeof(double) * 3 * n);
        memcpy(sigma, s0, sizeof(double) * n);
    }
    *iters_out = it;
    *fmax_out = fmx;
    free(q0); free(s0); free(vq); free(vs); free(gq); free(gs); free(mu_ex); free(tmp); free(fs);
    free(off); free(idx);
    return status;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
