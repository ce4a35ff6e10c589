/*
 * chfpe_oracle.c -- plain FP64 CPU restatement of the multimode classical hierarchical
 * Fokker-Planck equations (CHFPE) on a uniform (q,p) grid.
 *
 * TEST INFRASTRUCTURE.  This file is the oracle that the CUDA path is checked against.  It is
 * loaded only by the tests, by the smoke check and by the benchmark's CPU-baseline / reference
 * leg.  It shares no code, header, table or helper with the CUDA library; it is written from
 * the paper's equations alone, in the order the paper states them, with plain nested loops.
 *
 * What it computes (arXiv 2509.25840):
 *   potential      U(q)   Eq. "sec: Potenentials" + Eq. "sec: Potential ss'" (+ a quartic term
 *                         g4 q^4/4! in the same Taylor convention)
 *   bath coupling  V_s(q) = V_LL q + V_SL q^2/2                     (Sec. II A, after Eq. h_int)
 *   hierarchy      dW^(n)/dt = (L - sum_s n_s gamma_s) W^(n) + sum_s Phi_s W^(n+e_s)
 *                              + sum_s n_s Theta_s W^(n-e_s)      (Eq. HEOM, Drude, one index
 *                              per mode; the n_s factor on Theta as in Appendix A)
 *   Liouvillian    L W = sum_s [ dU/dq_s dW/dp_s - (p_s/m_s) dW/dq_s ]      (Eq. CL_liouville)
 *   Phi_s   = V_s'(q_s) d/dp_s                                               (Eq. Phi)
 *   Theta_s = m_s zeta_s gamma_s kT V_s'(q_s) d/dp_s + zeta_s gamma_s p_s V_s'(q_s)  (Eq. Theta)
 *   insertion      X^x W = sum_s dX/dq_s dW/dp_s, applied to every member   (Eq. Opticalexc)
 *   observable     R = integral C(q) W^(0) dq dp                  (Eqs. 1Dresponse, 2Dresponse)
 *   optical poly   X(q) = sum_s X_s q_s + 1/2 sum_{s,s'} X_ss' q_s q_s'      (Eqs. NLdip, NLpol)
 *
 * Representation.  As in Appendix A, which factors psi_0(p) exp(-U/2kT) (= exp(-H/2kT) up to a
 * constant) out of every member, the unknowns are the symmetrised members
 *   g^(n) = W^(n) exp(+H_sys/2kT) / lambda_n,   lambda_n = prod_s sqrt(n_s! c_s^n_s),
 *   c_s = zeta_s gamma_s m_s kT.
 * Substituting into Eq. HEOM (using mkT d/dp + p = mkT e^{-p^2/2mkT} d/dp e^{+p^2/2mkT} and
 * L exp(-H/2kT) = 0) gives
 *   dg^(n)/dt = L g^(n) - sum_s n_s gamma_s g^(n)
 *             + sum_s sqrt((n_s+1) c_s) V_s' (d/dp_s - p_s/(2 m_s kT)) g^(n+e_s)
 *             + sum_s sqrt(n_s c_s)     V_s' (d/dp_s + p_s/(2 m_s kT)) g^(n-e_s),
 * the insertion becomes X^x -> sum_s dX/dq_s (d/dp_s - p_s/(2 m_s kT)) on every member, and the
 * observable integral C(q) W^(0) becomes integral C(q) exp(-H/2kT) g^(0).  On the grid the two
 * coupling operators are exact negative transposes of each other and L is antisymmetric, so the
 * discrete generator is antisymmetric minus a non-negative diagonal: no growing modes.  (The
 * same central differences applied to W^(n) itself give growing modes.)
 *
 * Discretisation (on the p-grid representation the paper's compact scheme is replaced by an
 * explicit one; the Hermite representation below offers both): every axis is a uniform grid
 * with both end points, derivatives are the 6th-order central difference
 *   (D f)_i = [45 (f_{i+1}-f_{i-1}) - 9 (f_{i+2}-f_{i-2}) + (f_{i+3}-f_{i-3})] / (60 h)
 * with zero values outside the grid, the hierarchy is truncated at n_1+...+n_d <= depth, and
 * time stepping is the textbook classical Runge-Kutta method (k1..k4).
 *
 * Layout of a state: [member][q_1]..[q_d][p_1]..[p_d], p_d fastest; members ordered by tier
 * |n| and, inside a tier, lexicographically ascending in (n_1, ..., n_d).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAXD 3
#define ORC_MAXM 512

typedef struct {
    int d;
    int depth;
    double kT;
    double m[3], omega[3], g3[3], g4[3];
    double g2[3][3], g_s2s[3][3], g_ss2[3][3];
    double zeta[3], gamma[3], V_LL[3], V_SL[3];
    int nq[3], np[3];
    double qmin[3], qmax[3], pmin[3], pmax[3];
    int qscheme;         /* q-derivatives of the Hermite representation: 0 = the explicit
                            6th-order central difference, 1 = the compact scheme of Sec. III B,
                            2 = its skew-symmetric part (orc_compact_skew_deriv1d) */
} orc_problem;

typedef struct {
    double lin[3];
    double quad[3][3];
} orc_optical;

/* ------------------------------------------------------------------------------------------ */
/* geometry                                                                                   */
/* ------------------------------------------------------------------------------------------ */

typedef struct {
    int d, naxes;
    long n[2 * ORC_MAXD];
    long stride[2 * ORC_MAXD];
    double lo[2 * ORC_MAXD];
    double h[2 * ORC_MAXD];
    long P;              /* points per member */
    int M;               /* members */
    int mem[ORC_MAXM][ORC_MAXD];
} orc_geom;

int orc_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* All n in N^d with n_1+..+n_d <= depth, by tier, then lexicographically ascending. */
int orc_members(int d, int depth, int *out /* [M][3] */)
{
    int count = 0;
    for (int t = 0; t <= depth; ++t) {
        if (d == 1) {
            out[3 * count + 0] = t; out[3 * count + 1] = 0; out[3 * count + 2] = 0; ++count;
        } else if (d == 2) {
            for (int a = 0; a <= t; ++a) {
                out[3 * count + 0] = a; out[3 * count + 1] = t - a; out[3 * count + 2] = 0; ++count;
            }
        } else {
            for (int a = 0; a <= t; ++a)
                for (int b = 0; b <= t - a; ++b) {
                    out[3 * count + 0] = a; out[3 * count + 1] = b; out[3 * count + 2] = t - a - b;
                    ++count;
                }
        }
    }
    return count;
}

static int count_members(int d, int depth)
{
    int M = 0;
    for (int t = 0; t <= depth; ++t) {
        long c = 1;   /* C(t+d-1, d-1) members in tier t */
        for (int k = 1; k < d; ++k) c = c * (t + k) / k;
        M += (int)c;
    }
    return M;
}

static int geom_init(const orc_problem *pr, orc_geom *g)
{
    int d = pr->d;
    if (d < 1 || d > ORC_MAXD || pr->depth < 0) return -1;
    g->d = d;
    g->naxes = 2 * d;
    for (int s = 0; s < d; ++s) {
        g->n[s] = pr->nq[s];
        g->lo[s] = pr->qmin[s];
        g->h[s] = (pr->qmax[s] - pr->qmin[s]) / (double)(pr->nq[s] - 1);
        g->n[d + s] = pr->np[s];
        g->lo[d + s] = pr->pmin[s];
        g->h[d + s] = (pr->pmax[s] - pr->pmin[s]) / (double)(pr->np[s] - 1);
    }
    g->stride[2 * d - 1] = 1;
    for (int a = 2 * d - 2; a >= 0; --a) g->stride[a] = g->stride[a + 1] * g->n[a + 1];
    g->P = g->stride[0] * g->n[0];
    int M = count_members(d, pr->depth);
    if (M > ORC_MAXM) return -2;
    int tmp[ORC_MAXM * 3];
    orc_members(d, pr->depth, tmp);
    g->M = M;
    for (int i = 0; i < M; ++i)
        for (int s = 0; s < ORC_MAXD; ++s) g->mem[i][s] = (s < d) ? tmp[3 * i + s] : 0;
    return 0;
}

int orc_member_count(int d, int depth)
{
    int M = count_members(d, depth);
    return (M > ORC_MAXM) ? -1 : M;
}

long orc_points(const orc_problem *pr)
{
    orc_geom g;
    if (geom_init(pr, &g)) return -1;
    return g.P;
}

/* index of member n (or -1 when n lies outside the truncated hierarchy) */
static int member_index(const orc_geom *g, const int *n)
{
    for (int i = 0; i < g->M; ++i) {
        int same = 1;
        for (int s = 0; s < g->d; ++s)
            if (g->mem[i][s] != n[s]) same = 0;
        if (same) return i;
    }
    return -1;
}

static void decode(const orc_geom *g, long x, long *idx)
{
    for (int a = 0; a < g->naxes; ++a) idx[a] = (x / g->stride[a]) % g->n[a];
}

/* ------------------------------------------------------------------------------------------ */
/* model functions                                                                            */
/* ------------------------------------------------------------------------------------------ */

/* U(q): Eq. "sec: Potenentials" (+ quartic) summed over modes, + Eq. "sec: Potential ss'" */
double orc_potential(const orc_problem *pr, const double *q)
{
    double U = 0.0;
    for (int s = 0; s < pr->d; ++s) {
        double x = q[s];
        U += 0.5 * pr->m[s] * pr->omega[s] * pr->omega[s] * x * x
           + pr->g3[s] * x * x * x / 6.0
           + pr->g4[s] * x * x * x * x / 24.0;
    }
    for (int a = 0; a < pr->d; ++a)
        for (int b = a + 1; b < pr->d; ++b) {
            U += pr->g2[a][b] * q[a] * q[b]
               + (pr->g_s2s[a][b] * q[a] * q[a] * q[b] + pr->g_ss2[a][b] * q[a] * q[b] * q[b]) / 6.0;
        }
    return U;
}

/* dU/dq_s, by differentiating the polynomial above term by term */
double orc_dUdq(const orc_problem *pr, const double *q, int s)
{
    double x = q[s];
    double F = pr->m[s] * pr->omega[s] * pr->omega[s] * x
             + pr->g3[s] * x * x / 2.0
             + pr->g4[s] * x * x * x / 6.0;
    for (int b = s + 1; b < pr->d; ++b)          /* pairs (s, b), s < b */
        F += pr->g2[s][b] * q[b]
           + (2.0 * pr->g_s2s[s][b] * x * q[b] + pr->g_ss2[s][b] * q[b] * q[b]) / 6.0;
    for (int a = 0; a < s; ++a)                  /* pairs (a, s), a < s */
        F += pr->g2[a][s] * q[a]
           + (pr->g_s2s[a][s] * q[a] * q[a] + 2.0 * pr->g_ss2[a][s] * q[a] * x) / 6.0;
    return F;
}

/* V_s'(q_s) for V_s(q) = V_LL q + V_SL q^2 / 2 */
static double dVdq(const orc_problem *pr, int s, double qs)
{
    return pr->V_LL[s] + pr->V_SL[s] * qs;
}

/* X(q) = sum_s X_s q_s + 1/2 sum_{s,s'} X_ss' q_s q_s'   (Eqs. NLdip / NLpol) */
double orc_optical_value(const orc_optical *X, int d, const double *q)
{
    double v = 0.0;
    for (int s = 0; s < d; ++s) v += X->lin[s] * q[s];
    for (int a = 0; a < d; ++a)
        for (int b = 0; b < d; ++b) v += 0.5 * X->quad[a][b] * q[a] * q[b];
    return v;
}

/* dX/dq_s of the polynomial above */
double orc_optical_grad(const orc_optical *X, int d, const double *q, int s)
{
    double v = X->lin[s];
    for (int b = 0; b < d; ++b) v += 0.5 * (X->quad[s][b] + X->quad[b][s]) * q[b];
    return v;
}

/* ------------------------------------------------------------------------------------------ */
/* finite differences                                                                         */
/* ------------------------------------------------------------------------------------------ */

/* 6th-order central first derivative of a 1-D array with zero values outside [0, n). */
void orc_deriv1d(long n, double h, const double *f, double *out)
{
    const double c[4] = {0.0, 45.0, -9.0, 1.0};
    for (long i = 0; i < n; ++i) {
        double acc = 0.0;
        for (int k = 1; k <= 3; ++k) {
            double fp = (i + k < n) ? f[i + k] : 0.0;
            double fm = (i - k >= 0) ? f[i - k] : 0.0;
            acc += c[k] * (fp - fm);
        }
        out[i] = acc / (60.0 * h);
    }
}

/* Compact (Pade) first derivative of Sec. III B on a 1-D array: solve A f' = B f / h with
 *   A = tridiag(alpha, 1, alpha)                 (first row 1, alpha; last row alpha, 1)
 *   (B f)_i = a (f_{i+1} - f_{i-1}) + b (f_{i+2} - f_{i-2}),  zero values outside [0, n)
 * alpha = 1/3, a = 7/9, b = 1/36: the sixth-order tridiagonal scheme of Lele (J. Comput. Phys.
 * 103, 16 (1992)), whose interior consistency on f = x needs 2a + 4b = 1 + 2 alpha; the paper
 * prints a = beta/2 = 7/18, which fails that condition, and the reading taken is a = 7/9 (the
 * paper's beta = 14/9 halved).  The tridiagonal system is solved by forward elimination and
 * back substitution (Thomas algorithm). */
void orc_compact_deriv1d(long n, double h, const double *f, double *out)
{
    const double alpha = 1.0 / 3.0, a = 7.0 / 9.0, b = 1.0 / 36.0;
    double *cp = malloc(sizeof(double) * (n > 0 ? n : 1));
    for (long i = 0; i < n; ++i) {
        double f1p = (i + 1 < n) ? f[i + 1] : 0.0, f1m = (i >= 1) ? f[i - 1] : 0.0;
        double f2p = (i + 2 < n) ? f[i + 2] : 0.0, f2m = (i >= 2) ? f[i - 2] : 0.0;
        out[i] = (a * (f1p - f1m) + b * (f2p - f2m)) / h;
    }
    /* forward elimination: row i becomes x_i + cp_i x_{i+1} = out_i */
    for (long i = 0; i < n; ++i) {
        double sub = (i >= 1) ? alpha : 0.0;
        double sup = (i + 1 < n) ? alpha : 0.0;
        double piv = 1.0 - ((i >= 1) ? sub * cp[i - 1] : 0.0);
        cp[i] = sup / piv;
        out[i] = (out[i] - ((i >= 1) ? sub * out[i - 1] : 0.0)) / piv;
    }
    for (long i = n - 2; i >= 0; --i) out[i] -= cp[i] * out[i + 1];
    free(cp);
}

/* The skew-symmetric part of the compact derivative: (A^{-1} B + B A^{-1}) f / (2 h).  With the
 * truncated end rows of Sec. III B, A^{-1} B is not antisymmetric (A and B do not commute near the
 * ends), and in the hierarchy's generator that non-antisymmetric part gives growing modes; this
 * operator is antisymmetric (B^T = -B, A^T = A) and equals the compact derivative wherever the end
 * effects have decayed (they fall off by 0.38 per point).  Two tridiagonal solves (Thomas). */
void orc_compact_skew_deriv1d(long n, double h, const double *f, double *out)
{
    const double alpha = 1.0 / 3.0, a = 7.0 / 9.0, b = 1.0 / 36.0;
    double *x1 = malloc(sizeof(double) * (n > 0 ? n : 1));
    double *y = malloc(sizeof(double) * (n > 0 ? n : 1));
    double *cp = malloc(sizeof(double) * (n > 0 ? n : 1));
    orc_compact_deriv1d(n, h, f, x1);                 /* A^{-1} B f / h */
    for (long i = 0; i < n; ++i) y[i] = f[i];         /* A^{-1} f */
    for (long i = 0; i < n; ++i) {
        double sub = (i >= 1) ? alpha : 0.0;
        double sup = (i + 1 < n) ? alpha : 0.0;
        double piv = 1.0 - ((i >= 1) ? sub * cp[i - 1] : 0.0);
        cp[i] = sup / piv;
        y[i] = (y[i] - ((i >= 1) ? sub * y[i - 1] : 0.0)) / piv;
    }
    for (long i = n - 2; i >= 0; --i) y[i] -= cp[i] * y[i + 1];
    for (long i = 0; i < n; ++i) {                    /* B A^{-1} f / h, then the mean */
        double y1p = (i + 1 < n) ? y[i + 1] : 0.0, y1m = (i >= 1) ? y[i - 1] : 0.0;
        double y2p = (i + 2 < n) ? y[i + 2] : 0.0, y2m = (i >= 2) ? y[i - 2] : 0.0;
        out[i] = 0.5 * (x1[i] + (a * (y1p - y1m) + b * (y2p - y2m)) / h);
    }
    free(x1); free(y); free(cp);
}

/* the same derivative along axis a of one member's field, at point x */
static double deriv_axis(const orc_geom *g, const double *f, long x, const long *idx, int a)
{
    const double c[4] = {0.0, 45.0, -9.0, 1.0};
    double acc = 0.0;
    for (int k = 1; k <= 3; ++k) {
        double fp = (idx[a] + k < g->n[a]) ? f[x + k * g->stride[a]] : 0.0;
        double fm = (idx[a] - k >= 0) ? f[x - k * g->stride[a]] : 0.0;
        acc += c[k] * (fp - fm);
    }
    return acc / (60.0 * g->h[a]);
}

/* ------------------------------------------------------------------------------------------ */
/* right-hand side of the symmetrised hierarchy (Eq. HEOM with Eqs. CL_liouville, Phi, Theta) */
/* ------------------------------------------------------------------------------------------ */

int orc_rhs(const orc_problem *pr, const double *W, double *K)
{
    orc_geom g;
    if (geom_init(pr, &g)) return -1;
    const int d = g.d;
    const long P = g.P;
    const double kT = pr->kT;

    int up[ORC_MAXM][ORC_MAXD], dn[ORC_MAXM][ORC_MAXD];
    for (int i = 0; i < g.M; ++i)
        for (int s = 0; s < d; ++s) {
            int n[ORC_MAXD] = {0, 0, 0};
            for (int r = 0; r < d; ++r) n[r] = g.mem[i][r];
            n[s] += 1;
            up[i][s] = member_index(&g, n);
            n[s] -= 2;
            dn[i][s] = (n[s] >= 0) ? member_index(&g, n) : -1;
        }

#pragma omp parallel for collapse(2) schedule(static)
    for (int i = 0; i < g.M; ++i) {
        for (long x = 0; x < P; ++x) {
            long idx[2 * ORC_MAXD];
            double q[ORC_MAXD], p[ORC_MAXD];
            decode(&g, x, idx);
            for (int s = 0; s < d; ++s) {
                q[s] = g.lo[s] + idx[s] * g.h[s];
                p[s] = g.lo[d + s] + idx[d + s] * g.h[d + s];
            }
            const double *Wi = W + (long)i * P;
            double val = 0.0;
            /* classical Liouvillian: {H_sys, W}_PB */
            for (int s = 0; s < d; ++s) {
                val += orc_dUdq(pr, q, s) * deriv_axis(&g, Wi, x, idx, d + s)
                     - (p[s] / pr->m[s]) * deriv_axis(&g, Wi, x, idx, s);
            }
            /* damping -sum_s n_s gamma_s */
            double damp = 0.0;
            for (int s = 0; s < d; ++s) damp += g.mem[i][s] * pr->gamma[s];
            val -= damp * Wi[x];
            /* Phi_s W^(n+e_s) and n_s Theta_s W^(n-e_s), symmetrised */
            for (int s = 0; s < d; ++s) {
                double Vp = dVdq(pr, s, q[s]);
                double c = pr->zeta[s] * pr->gamma[s] * pr->m[s] * kT;
                double a = p[s] / (2.0 * pr->m[s] * kT);
                if (up[i][s] >= 0) {
                    const double *Wu = W + (long)up[i][s] * P;
                    double coef = sqrt((g.mem[i][s] + 1) * c) * Vp;
                    val += coef * (deriv_axis(&g, Wu, x, idx, d + s) - a * Wu[x]);
                }
                if (dn[i][s] >= 0) {
                    const double *Wd = W + (long)dn[i][s] * P;
                    double coef = sqrt(g.mem[i][s] * c) * Vp;
                    val += coef * (deriv_axis(&g, Wd, x, idx, d + s) + a * Wd[x]);
                }
            }
            K[(long)i * P + x] = val;
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* classical fourth-order Runge-Kutta, textbook form                                          */
/* ------------------------------------------------------------------------------------------ */

int orc_rk4(const orc_problem *pr, double *y, double dt, long nsteps)
{
    orc_geom g;
    if (geom_init(pr, &g)) return -1;
    const long N = (long)g.M * g.P;
    double *k1 = malloc(sizeof(double) * N), *k2 = malloc(sizeof(double) * N);
    double *k3 = malloc(sizeof(double) * N), *k4 = malloc(sizeof(double) * N);
    double *tmp = malloc(sizeof(double) * N);
    if (!k1 || !k2 || !k3 || !k4 || !tmp) {
        free(k1); free(k2); free(k3); free(k4); free(tmp);
        return -3;
    }
    for (long step = 0; step < nsteps; ++step) {
        orc_rhs(pr, y, k1);
#pragma omp parallel for schedule(static)
        for (long j = 0; j < N; ++j) tmp[j] = y[j] + 0.5 * dt * k1[j];
        orc_rhs(pr, tmp, k2);
#pragma omp parallel for schedule(static)
        for (long j = 0; j < N; ++j) tmp[j] = y[j] + 0.5 * dt * k2[j];
        orc_rhs(pr, tmp, k3);
#pragma omp parallel for schedule(static)
        for (long j = 0; j < N; ++j) tmp[j] = y[j] + dt * k3[j];
        orc_rhs(pr, tmp, k4);
#pragma omp parallel for schedule(static)
        for (long j = 0; j < N; ++j) y[j] += dt / 6.0 * (k1[j] + 2.0 * k2[j] + 2.0 * k3[j] + k4[j]);
    }
    free(k1); free(k2); free(k3); free(k4); free(tmp);
    return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* optical insertion and observable                                                           */
/* ------------------------------------------------------------------------------------------ */

/* out^(n) = X^x applied to member n (Eq. Opticalexc), in the symmetrised representation:
 *   sum_s dX/dq_s (d/dp_s - p_s / (2 m_s kT)) g^(n) */
int orc_insert(const orc_problem *pr, const orc_optical *X, const double *W, double *out)
{
    orc_geom g;
    if (geom_init(pr, &g)) return -1;
    const int d = g.d;
#pragma omp parallel for collapse(2) schedule(static)
    for (int i = 0; i < g.M; ++i) {
        for (long x = 0; x < g.P; ++x) {
            long idx[2 * ORC_MAXD];
            double q[ORC_MAXD];
            decode(&g, x, idx);
            for (int s = 0; s < d; ++s) q[s] = g.lo[s] + idx[s] * g.h[s];
            const double *Wi = W + (long)i * g.P;
            double v = 0.0;
            for (int s = 0; s < d; ++s) {
                double p = g.lo[d + s] + idx[d + s] * g.h[d + s];
                v += orc_optical_grad(X, d, q, s)
                   * (deriv_axis(&g, Wi, x, idx, d + s) - p / (2.0 * pr->m[s] * pr->kT) * Wi[x]);
            }
            out[(long)i * g.P + x] = v;
        }
    }
    return 0;
}

/* integral of C(q) W^(0)(q,p) = C(q) exp(-H/2kT) g^(0) over phase space, rectangle rule on the
 * grid nodes */
double orc_observe(const orc_problem *pr, const orc_optical *C, const double *W)
{
    orc_geom g;
    if (geom_init(pr, &g)) return NAN;
    const int d = g.d;
    double vol = 1.0;
    for (int a = 0; a < g.naxes; ++a) vol *= g.h[a];
    double sum = 0.0;
#pragma omp parallel for reduction(+ : sum) schedule(static)
    for (long x = 0; x < g.P; ++x) {
        long idx[2 * ORC_MAXD];
        double q[ORC_MAXD];
        decode(&g, x, idx);
        double H = 0.0;
        for (int s = 0; s < d; ++s) {
            q[s] = g.lo[s] + idx[s] * g.h[s];
            double p = g.lo[d + s] + idx[d + s] * g.h[d + s];
            H += p * p / (2.0 * pr->m[s]);
        }
        H += orc_potential(pr, q);
        sum += orc_optical_value(C, d, q) * exp(-H / (2.0 * pr->kT)) * W[x];
    }
    return vol * sum;
}

/* ------------------------------------------------------------------------------------------ */
/* equilibrium                                                                                */
/* ------------------------------------------------------------------------------------------ */

/* W^(0) = exp(-H_sys / kT) / Z with unit integral on the grid, W^(n != 0) = 0; stored
 * symmetrised: g^(0) = exp(-H_sys / 2kT) / Z */
int orc_boltzmann(const orc_problem *pr, double *W)
{
    orc_geom g;
    if (geom_init(pr, &g)) return -1;
    const int d = g.d;
    double vol = 1.0;
    for (int a = 0; a < g.naxes; ++a) vol *= g.h[a];
    double Z = 0.0;
    for (long x = 0; x < g.P; ++x) {
        long idx[2 * ORC_MAXD];
        double q[ORC_MAXD], E = 0.0;
        decode(&g, x, idx);
        for (int s = 0; s < d; ++s) {
            q[s] = g.lo[s] + idx[s] * g.h[s];
            double p = g.lo[d + s] + idx[d + s] * g.h[d + s];
            E += p * p / (2.0 * pr->m[s]);
        }
        E += orc_potential(pr, q);
        W[x] = exp(-E / (2.0 * pr->kT));
        Z += W[x] * W[x];
    }
    Z *= vol;
    for (long x = 0; x < g.P; ++x) W[x] /= Z;
    for (long j = g.P; j < (long)g.M * g.P; ++j) W[j] = 0.0;
    return 0;
}

/* W^(n) = lambda_n exp(-H/2kT) g^(n): back to the distributions of Eq. HEOM */
int orc_to_density(const orc_problem *pr, const double *G, double *W)
{
    orc_geom g;
    if (geom_init(pr, &g)) return -1;
    const int d = g.d;
    for (int i = 0; i < g.M; ++i) {
        double lam = 1.0;
        for (int s = 0; s < d; ++s) {
            double c = pr->zeta[s] * pr->gamma[s] * pr->m[s] * pr->kT;
            for (int k = 1; k <= g.mem[i][s]; ++k) lam *= sqrt(k * c);
        }
        for (long x = 0; x < g.P; ++x) {
            long idx[2 * ORC_MAXD];
            double q[ORC_MAXD], E = 0.0;
            decode(&g, x, idx);
            for (int s = 0; s < d; ++s) {
                q[s] = g.lo[s] + idx[s] * g.h[s];
                double p = g.lo[d + s] + idx[d + s] * g.h[d + s];
                E += p * p / (2.0 * pr->m[s]);
            }
            E += orc_potential(pr, q);
            W[(long)i * g.P + x] = lam * exp(-E / (2.0 * pr->kT)) * G[(long)i * g.P + x];
        }
    }
    return 0;
}

/* max|M W| / max|W| over the whole hierarchy */
double orc_residual(const orc_problem *pr, const double *W)
{
    orc_geom g;
    if (geom_init(pr, &g)) return NAN;
    const long N = (long)g.M * g.P;
    double *K = malloc(sizeof(double) * N);
    if (!K) return NAN;
    orc_rhs(pr, W, K);
    double kmax = 0.0, wmax = 0.0;
    for (long j = 0; j < N; ++j) {
        if (fabs(K[j]) > kmax) kmax = fabs(K[j]);
        if (fabs(W[j]) > wmax) wmax = fabs(W[j]);
    }
    free(K);
    return kmax / wmax;
}

/* Propagate W in blocks of check_every RK4 steps until the residual drops below tol or
 * max_steps steps have been taken.  Returns the steps taken; *residual gets the last value. */
long orc_equilibrate(const orc_problem *pr, double *W, double dt, long max_steps, double tol,
                     long check_every, double *residual)
{
    long steps = 0;
    double r = orc_residual(pr, W);
    while (steps < max_steps && r >= tol) {
        long n = check_every;
        if (n > max_steps - steps) n = max_steps - steps;
        if (orc_rk4(pr, W, dt, n)) return -1;
        steps += n;
        r = orc_residual(pr, W);
    }
    if (residual) *residual = r;
    return steps;
}

/* ------------------------------------------------------------------------------------------ */
/* response functions                                                                         */
/* ------------------------------------------------------------------------------------------ */

/* R1(k dt stride) = integral C G(t) A^x W_eq  (Eq. 1Dresponse with the observed operator C;
 * the paper uses C = A), k = 0..nt-1. */
int orc_response1(const orc_problem *pr, const orc_optical *A, const orc_optical *C,
                  const double *Weq, double dt, int nt, long stride, double *R)
{
    orc_geom g;
    if (geom_init(pr, &g)) return -1;
    const long N = (long)g.M * g.P;
    double *W = malloc(sizeof(double) * N);
    if (!W) return -3;
    orc_insert(pr, A, Weq, W);
    for (int k = 0; k < nt; ++k) {
        R[k] = orc_observe(pr, C, W);
        if (k + 1 < nt) orc_rk4(pr, W, dt, stride);
    }
    free(W);
    return 0;
}

/* R2[i][j] = integral C G(t2) B^x G(t1) A^x W_eq  (Eq. 2Dresponse) with t1 = i dt stride,
 * t2 = j dt stride; every t1 branch is propagated on its own, one after the other. */
int orc_response2(const orc_problem *pr, const orc_optical *A, const orc_optical *B,
                  const orc_optical *C, const double *Weq, double dt, int nt1, int nt2,
                  long stride, double *R)
{
    orc_geom g;
    if (geom_init(pr, &g)) return -1;
    const long N = (long)g.M * g.P;
    double *Wc = malloc(sizeof(double) * N), *Wb = malloc(sizeof(double) * N);
    if (!Wc || !Wb) { free(Wc); free(Wb); return -3; }
    orc_insert(pr, A, Weq, Wc);
    for (int i = 0; i < nt1; ++i) {
        orc_insert(pr, B, Wc, Wb);
        for (int j = 0; j < nt2; ++j) {
            R[(long)i * nt2 + j] = orc_observe(pr, C, Wb);
            if (j + 1 < nt2) orc_rk4(pr, Wb, dt, stride);
        }
        if (i + 1 < nt1) orc_rk4(pr, Wc, dt, stride);
    }
    free(Wc); free(Wb);
    return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* Hermite-function representation of the momenta (Sec. III A, Appendix A, Eq. HEOM2FP-H)    */
/* ------------------------------------------------------------------------------------------ */
/*
 * The paper expands every member as W^(n) = psi_0(p) exp(-U/2kT) sum_k c^(n)_k(q) psi_k(p) with
 * the Hermite functions psi_j(p) = H_j(p/a) exp(-p^2/2a^2) / sqrt(2^j j! a sqrt(pi)),
 * a = sqrt(2 m kT) (one index k_s per mode).  psi_0(p) exp(-U/2kT) is exp(-H/2kT) up to a
 * constant, so the coefficients are those of the symmetrised member g^(n) in the orthonormal
 * functions psi_k:  g^(n)(q,p) = sum_k c^(n)_k(q) prod_s psi_{k_s}(p_s)  (with the member scale
 * lambda_n of the grid representation).  The ladder identities
 *     p psi_k   = sqrt(m kT) [sqrt(k) psi_{k-1} + sqrt(k+1) psi_{k+1}]
 *     d/dp psi_k = [sqrt(k) psi_{k-1} - sqrt(k+1) psi_{k+1}] / (2 sqrt(m kT))
 * turn the symmetrised hierarchy into (coefficient of psi_k, member n, mode s terms summed)
 *     dc^(n)_k/dt = sum_s [ sqrt(k_s+1) D+_s c^(n)_{k+e_s} - sqrt(k_s) D-_s c^(n)_{k-e_s} ]
 *                 - sum_s n_s gamma_s c^(n)_k
 *                 - sum_s sqrt((n_s+1) c_s) V_s' sqrt(k_s) / sqrt(m_s kT) c^(n+e_s)_{k-e_s}
 *                 + sum_s sqrt(n_s c_s) V_s' sqrt(k_s+1) / sqrt(m_s kT) c^(n-e_s)_{k+e_s}
 *     D+-_s = dU/dq_s / (2 sqrt(m_s kT)) -+ (sqrt(m_s kT) / m_s) d/dq_s,
 * which is Eq. HEOM2FP-H (its Theta^(s)_j and Phi^(s)_j with the member scale lambda_n divided
 * out); (d/dp - p/2mkT) psi_k = -sqrt(k+1) psi_{k+1} / sqrt(mkT) is the raising operator the
 * Phi link and the insertion use, (d/dp + p/2mkT) the matching lowering operator.  Coefficients
 * with k_s outside [0, K_s) are zero (truncation).  d/dq_s is the same 6th-order central
 * difference with zero values outside the q-grid (qscheme 0), or the compact scheme of
 * Sec. III B, orc_compact_deriv1d (qscheme 1), or its skew-symmetric part (qscheme 2).
 *
 * Layout: [member][q_1]..[q_d][k_1]..[k_d], k_d fastest; the orc_problem's np[s] holds K_s
 * (pmin/pmax are not used).
 */

#define ORC_PI 3.14159265358979323846

static int hgeom_init(const orc_problem *pr, orc_geom *g)
{
    int r = geom_init(pr, g);
    if (r) return r;
    for (int s = 0; s < g->d; ++s) {   /* the k axes are indices, not coordinates */
        g->lo[g->d + s] = 0.0;
        g->h[g->d + s] = 1.0;
    }
    return 0;
}

/* coefficient c^(member)_k at the point x shifted by `dk` along k_s; 0 outside [0, K_s) */
static double hcoef(const orc_geom *g, const double *C, int member, long x, const long *idx, int s,
                    int dk)
{
    if (member < 0) return 0.0;
    long k = idx[g->d + s] + dk;
    if (k < 0 || k >= g->n[g->d + s]) return 0.0;
    return C[(long)member * g->P + x + dk * g->stride[g->d + s]];
}

/* d/dq_s of c^(i)_{k + dk e_s} at the point x (zero outside the q-grid and outside [0, K_s));
 * Dpre == NULL: the explicit central difference; else Dpre[(s M + i) P + x] holds the compact
 * derivatives (h_compact_derivs) */
static double hderiv_q(const orc_geom *g, const double *C, int i, long x, const long *idx, int s,
                       int dk, const double *Dpre)
{
    long k = idx[g->d + s] + dk;
    if (k < 0 || k >= g->n[g->d + s]) return 0.0;
    if (Dpre) return Dpre[((long)s * g->M + i) * g->P + x + dk * g->stride[g->d + s]];
    return deriv_axis(g, C + (long)i * g->P, x + dk * g->stride[g->d + s], idx, s);
}

/* the compact derivative (Sec. III B) of every member's coefficients along every q axis, line by
 * line: D[(s M + i) P + x] = d/dq_s c^(i) at x.  NULL when out of memory. */
static double *h_compact_derivs(const orc_geom *g, const double *C, int skew)
{
    const int d = g->d;
    const long P = g->P;
    double *D = malloc(sizeof(double) * d * g->M * P);
    if (!D) return NULL;
    int bad = 0;
    for (int s = 0; s < d; ++s) {
        const long n = g->n[s], st = g->stride[s];
#pragma omp parallel for collapse(2) schedule(static)
        for (int i = 0; i < g->M; ++i) {
            for (long x0 = 0; x0 < P; ++x0) {
                if ((x0 / st) % n != 0) continue;      /* one line per start point q_s = q_min */
                double *f = malloc(sizeof(double) * n), *df = malloc(sizeof(double) * n);
                if (!f || !df) {
                    free(f); free(df);
#pragma omp atomic write
                    bad = 1;
                    continue;
                }
                for (long j = 0; j < n; ++j) f[j] = C[(long)i * P + x0 + j * st];
                if (skew)
                    orc_compact_skew_deriv1d(n, g->h[s], f, df);
                else
                    orc_compact_deriv1d(n, g->h[s], f, df);
                for (long j = 0; j < n; ++j) D[((long)s * g->M + i) * P + x0 + j * st] = df[j];
                free(f); free(df);
            }
        }
    }
    if (bad) { free(D); return NULL; }
    return D;
}

int orc_h_rhs(const orc_problem *pr, const double *Cin, double *K)
{
    orc_geom g;
    if (hgeom_init(pr, &g)) return -1;
    const int d = g.d;
    const long P = g.P;
    const double kT = pr->kT;
    double *Dpre = NULL;
    if (pr->qscheme == 1 || pr->qscheme == 2) {
        Dpre = h_compact_derivs(&g, Cin, pr->qscheme == 2);
        if (!Dpre) return -3;
    } else if (pr->qscheme != 0) {
        return -1;
    }
    int up[ORC_MAXM][ORC_MAXD], dn[ORC_MAXM][ORC_MAXD];
    for (int i = 0; i < g.M; ++i)
        for (int s = 0; s < d; ++s) {
            int n[ORC_MAXD] = {0, 0, 0};
            for (int r = 0; r < d; ++r) n[r] = g.mem[i][r];
            n[s] += 1;
            up[i][s] = member_index(&g, n);
            n[s] -= 2;
            dn[i][s] = (n[s] >= 0) ? member_index(&g, n) : -1;
        }
#pragma omp parallel for collapse(2) schedule(static)
    for (int i = 0; i < g.M; ++i) {
        for (long x = 0; x < P; ++x) {
            long idx[2 * ORC_MAXD];
            double q[ORC_MAXD];
            decode(&g, x, idx);
            for (int s = 0; s < d; ++s) q[s] = g.lo[s] + idx[s] * g.h[s];
            double val = 0.0;
            for (int s = 0; s < d; ++s) {
                const double smkT = sqrt(pr->m[s] * kT);
                const double F = orc_dUdq(pr, q, s);
                const double ks = (double)idx[d + s];
                /* sqrt(k+1) D+ c_{k+e_s} - sqrt(k) D- c_{k-e_s} */
                const double cp = hcoef(&g, Cin, i, x, idx, s, +1);
                const double cm = hcoef(&g, Cin, i, x, idx, s, -1);
                const double dcp = hderiv_q(&g, Cin, i, x, idx, s, +1, Dpre);
                const double dcm = hderiv_q(&g, Cin, i, x, idx, s, -1, Dpre);
                val += sqrt(ks + 1.0) * (F / (2.0 * smkT) * cp - smkT / pr->m[s] * dcp);
                val -= sqrt(ks) * (F / (2.0 * smkT) * cm + smkT / pr->m[s] * dcm);
                /* hierarchy links */
                const double c = pr->zeta[s] * pr->gamma[s] * pr->m[s] * kT;
                const double Vp = dVdq(pr, s, q[s]);
                const double ni = (double)g.mem[i][s];
                val -= sqrt((ni + 1.0) * c) * Vp * sqrt(ks) / smkT *
                       hcoef(&g, Cin, up[i][s], x, idx, s, -1);
                val += sqrt(ni * c) * Vp * sqrt(ks + 1.0) / smkT *
                       hcoef(&g, Cin, dn[i][s], x, idx, s, +1);
            }
            double damp = 0.0;
            for (int s = 0; s < d; ++s) damp += g.mem[i][s] * pr->gamma[s];
            val -= damp * Cin[(long)i * P + x];
            K[(long)i * P + x] = val;
        }
    }
    free(Dpre);
    return 0;
}

int orc_h_rk4(const orc_problem *pr, double *y, double dt, long nsteps)
{
    orc_geom g;
    if (hgeom_init(pr, &g)) return -1;
    const long N = (long)g.M * g.P;
    double *k1 = malloc(sizeof(double) * N), *k2 = malloc(sizeof(double) * N);
    double *k3 = malloc(sizeof(double) * N), *k4 = malloc(sizeof(double) * N);
    double *tmp = malloc(sizeof(double) * N);
    if (!k1 || !k2 || !k3 || !k4 || !tmp) {
        free(k1); free(k2); free(k3); free(k4); free(tmp);
        return -3;
    }
    for (long step = 0; step < nsteps; ++step) {
        orc_h_rhs(pr, y, k1);
#pragma omp parallel for schedule(static)
        for (long j = 0; j < N; ++j) tmp[j] = y[j] + 0.5 * dt * k1[j];
        orc_h_rhs(pr, tmp, k2);
#pragma omp parallel for schedule(static)
        for (long j = 0; j < N; ++j) tmp[j] = y[j] + 0.5 * dt * k2[j];
        orc_h_rhs(pr, tmp, k3);
#pragma omp parallel for schedule(static)
        for (long j = 0; j < N; ++j) tmp[j] = y[j] + dt * k3[j];
        orc_h_rhs(pr, tmp, k4);
#pragma omp parallel for schedule(static)
        for (long j = 0; j < N; ++j) y[j] += dt / 6.0 * (k1[j] + 2.0 * k2[j] + 2.0 * k3[j] + k4[j]);
    }
    free(k1); free(k2); free(k3); free(k4); free(tmp);
    return 0;
}

/* X^x on every member (Eq. Opticalexc): sum_s dX/dq_s (d/dp_s - p_s/2m_skT) acts on psi_k as
 * -sqrt(k_s+1)/sqrt(m_s kT) psi_{k+e_s}:  out_k = -sum_s dX/dq_s sqrt(k_s)/sqrt(m_s kT) c_{k-e_s} */
int orc_h_insert(const orc_problem *pr, const orc_optical *X, const double *Cin, double *out)
{
    orc_geom g;
    if (hgeom_init(pr, &g)) return -1;
    const int d = g.d;
#pragma omp parallel for collapse(2) schedule(static)
    for (int i = 0; i < g.M; ++i) {
        for (long x = 0; x < g.P; ++x) {
            long idx[2 * ORC_MAXD];
            double q[ORC_MAXD];
            decode(&g, x, idx);
            for (int s = 0; s < d; ++s) q[s] = g.lo[s] + idx[s] * g.h[s];
            double v = 0.0;
            for (int s = 0; s < d; ++s)
                v -= orc_optical_grad(X, d, q, s) * sqrt((double)idx[d + s]) /
                     sqrt(pr->m[s] * pr->kT) * hcoef(&g, Cin, i, x, idx, s, -1);
            out[(long)i * g.P + x] = v;
        }
    }
    return 0;
}

/* integral C(q) exp(-H/2kT) g^(0) dq dp: the p-integral of exp(-p^2/4mkT) psi_k is
 * sqrt(a sqrt(pi)) for k = 0 and 0 otherwise, so only c^(0)_0 contributes; rectangle rule on
 * the q nodes */
double orc_h_observe(const orc_problem *pr, const orc_optical *C, const double *Cin)
{
    orc_geom g;
    if (hgeom_init(pr, &g)) return NAN;
    const int d = g.d;
    double pre = 1.0;
    for (int s = 0; s < d; ++s) pre *= g.h[s] * sqrt(sqrt(2.0 * pr->m[s] * pr->kT) * sqrt(ORC_PI));
    const long Pq = g.P / g.stride[d - 1];   /* q points: P = Pq * prod K_s */
    double sum = 0.0;
    for (long x = 0; x < g.P; x += g.stride[d - 1]) {
        long idx[2 * ORC_MAXD];
        double q[ORC_MAXD];
        decode(&g, x, idx);
        for (int s = 0; s < d; ++s) q[s] = g.lo[s] + idx[s] * g.h[s];
        sum += orc_optical_value(C, d, q) * exp(-orc_potential(pr, q) / (2.0 * pr->kT)) * Cin[x];
    }
    (void)Pq;
    return pre * sum;
}

/* equilibrium sample: c^(0)_0(q) = exp(-U/2kT) prod_s sqrt(a_s sqrt(pi)) / Z with
 * Z = (h^d sum_q exp(-U/kT)) prod_s sqrt(2 pi m_s kT) (the p-integral taken exactly), so that
 * the density integrates to 1; every other coefficient and member is 0 */
int orc_h_boltzmann(const orc_problem *pr, double *Cout)
{
    orc_geom g;
    if (hgeom_init(pr, &g)) return -1;
    const int d = g.d;
    memset(Cout, 0, sizeof(double) * (long)g.M * g.P);
    double Zq = 0.0, norm = 1.0, vol = 1.0;
    for (int s = 0; s < d; ++s) {
        vol *= g.h[s];
        norm *= sqrt(sqrt(2.0 * pr->m[s] * pr->kT) * sqrt(ORC_PI)) / sqrt(2.0 * ORC_PI * pr->m[s] * pr->kT);
    }
    for (long x = 0; x < g.P; x += g.stride[d - 1]) {
        long idx[2 * ORC_MAXD];
        double q[ORC_MAXD];
        decode(&g, x, idx);
        for (int s = 0; s < d; ++s) q[s] = g.lo[s] + idx[s] * g.h[s];
        Zq += exp(-orc_potential(pr, q) / pr->kT);
    }
    Zq *= vol;
    for (long x = 0; x < g.P; x += g.stride[d - 1]) {
        long idx[2 * ORC_MAXD];
        double q[ORC_MAXD];
        decode(&g, x, idx);
        for (int s = 0; s < d; ++s) q[s] = g.lo[s] + idx[s] * g.h[s];
        Cout[x] = exp(-orc_potential(pr, q) / (2.0 * pr->kT)) * norm / Zq;
    }
    return 0;
}
