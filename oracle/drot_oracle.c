/*
 * FP64 CPU oracle for DROT (Douglas-Rachford splitting for optimal transport).
 *
 * TEST INFRASTRUCTURE.  This file is the slow, plain reference that the CUDA
 * path is compared against.  Only the test suite, the package smoke check and
 * the CPU-baseline leg of the benchmark load it; the solver library never
 * does, and the two share no code.
 *
 * Problem (Sec. 1, eq. ot:dist):  minimise <C, X> over X >= 0 with
 * X e = p and X^T f = q, where e = 1_n, f = 1_m (Sec. 2, "Notation").
 *
 * The iteration is Algorithm 1 (Sec. 3.1) taken step by step, in double
 * precision, with plain loops and no blocking or fusion beyond what the
 * algorithm states:
 *   step 4   X_{k+1} = [X_k + phi_k e^T + f psi_k^T - rho C]_+
 *   step 5   r = X_{k+1} e - p,  s = X_{k+1}^T f - q,  beta = f^T r / (m+n)
 *   step 6   phi_{k+1} = (a_k - 2 r + (2 beta - alpha_k) f) / n
 *   step 7   psi_{k+1} = (b_k - 2 s + (2 beta - alpha_k) e) / m
 *   step 8   a -= r,  b -= s,  alpha -= beta
 * (the paper writes the column-side vector as \varphi; here it is psi).
 *
 * Stopping quantities (Sec. 3.1, "Stopping criteria"), with mu = phi / rho
 * and nu = psi / rho (Appendix A.2, eq. dual:var):
 *   primal   <C, X_k>
 *   dual     (p^T phi_k + q^T psi_k) / rho
 *   gap      |primal - dual|
 *   r_primal ||r||, reported both as l1 (||r||_1 + ||s||_1) and l2
 *   r_dual   ||[(phi_k/rho) e^T + f (psi_k/rho)^T - C]_+||_F
 * r_dual for (phi_k, psi_k) needs one pass over C with those vectors; the
 * pass that produces X_{k+1} is that pass, so each iteration reports r_dual of
 * the vectors it started from ("lagged").  The stop rule is: gap <= tol and
 * l1 residual <= tol (optionally, by a bitmask: 1 gap, 2 l1 residual, 4 lagged r_dual).
 *
 * Initial state (Algorithm 1, lines before the loop, generalised to a warm
 * start): Y_0 = X_0 + phi_0 e^T + f psi_0^T, a_0 = Y_0 e - p,
 * b_0 = Y_0^T f - q, alpha_0 = f^T a_0 / (m+n).  With phi_0 = psi_0 = 0 this is
 * the paper's a_0 = X_0 e - p, b_0 = X_0^T f - q.  The cold start is
 * X_0 = p q^T (Sec. 4).
 *
 * Mutations: oracle_set_mutation(k) plants one deliberate mistake (k > 0) so
 * the tests can show that their pins catch it.  k = 0 is the oracle proper.
 *
 * Threads: the same source is built twice.  Without OpenMP (the parity
 * reference) the pragmas below are ignored and every loop runs in the order
 * written.  With -fopenmp (used only to time the oracle on all host cores)
 * the loops over rows, and the column-sum loop over columns, are split across
 * threads; each r_i, s_j and X_ij is still formed by one thread in the order
 * written, and only the three scalar totals (sum r, <C,X>, r_dual^2) are
 * combined in an unspecified order.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* layout of the stats array filled by oracle_iterate / oracle_solve */
enum {
    ORC_PRIMAL = 0,
    ORC_DUAL = 1,
    ORC_GAP = 2,
    ORC_RES_L1 = 3,
    ORC_RES_L2 = 4,
    ORC_DUAL_RES_PREV = 5, /* r_dual of the vectors the iteration started from */
    ORC_BETA = 6,
    ORC_NSTATS = 7
};

static int g_mutation = 0;

void oracle_set_mutation(int k) { g_mutation = k; }
int oracle_nstats(void) { return ORC_NSTATS; }

/* Threads the iteration uses (1 unless built with OpenMP). */
int oracle_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* a_0, b_0, alpha_0 of Algorithm 1 for a start (X0, phi0, psi0). */
void oracle_init(int64_t m, int64_t n, const double *p, const double *q,
                 const double *X, const double *phi, const double *psi,
                 double *a, double *b, double *alpha)
{
    double sum_phi = 0.0, sum_psi = 0.0;
    for (int64_t i = 0; i < m; ++i) sum_phi += phi[i];
    for (int64_t j = 0; j < n; ++j) sum_psi += psi[j];
    /* a = Y0 e - p = X0 e - p + n phi0 + (e^T psi0) f */
    for (int64_t i = 0; i < m; ++i) {
        double row = 0.0;
        for (int64_t j = 0; j < n; ++j) row += X[i * n + j];
        a[i] = row - p[i] + (double)n * phi[i] + sum_psi;
    }
    /* b = Y0^T f - q = X0^T f - q + m psi0 + (f^T phi0) e */
    for (int64_t j = 0; j < n; ++j) {
        double col = 0.0;
        for (int64_t i = 0; i < m; ++i) col += X[i * n + j];
        b[j] = col - q[j] + (double)m * psi[j] + sum_phi;
    }
    double sa = 0.0;
    for (int64_t i = 0; i < m; ++i) sa += a[i];
    *alpha = sa / (double)(m + n);
}

/* One pass of Algorithm 1 (steps 4-8) in place, plus the stopping quantities
 * of the new iterate (and r_dual of the vectors the pass started from). */
void oracle_iterate(int64_t m, int64_t n, const double *C, const double *p, const double *q,
                    double rho, double *X, double *phi, double *psi, double *a, double *b,
                    double *alpha, double *stats, double *work /* m + n doubles */)
{
    double *r = work;      /* m */
    double *s = work + m;  /* n */

    /* step 4, and ||[phi_k + psi_k - rho C]_+||_F^2 along the way */
    double dual_sq = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : dual_sq)
    for (int64_t i = 0; i < m; ++i) {
        for (int64_t j = 0; j < n; ++j) {
            double c = C[i * n + j];
            double shift = phi[i] + psi[j] - rho * c;
            if (g_mutation == 7) shift = phi[i] + psi[j];          /* drop -rho C */
            double x = X[i * n + j] + shift;
            X[i * n + j] = x > 0.0 ? x : 0.0;
            if (shift > 0.0) dual_sq += shift * shift;
        }
    }

    /* step 5: residuals of the new iterate and beta */
    double sum_r = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : sum_r)
    for (int64_t i = 0; i < m; ++i) {
        double row = 0.0;
        for (int64_t j = 0; j < n; ++j) row += X[i * n + j];
        r[i] = row - p[i];
        sum_r += r[i];
    }
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n; ++j) {
        double col = 0.0;
        for (int64_t i = 0; i < m; ++i) col += X[i * n + j];
        s[j] = col - q[j];
    }
    double beta = sum_r / (double)(m + n);

    /* steps 6-7 */
    double shift_term = 2.0 * beta - *alpha;
    if (g_mutation == 2) shift_term = -2.0 * beta - *alpha;       /* wrong sign on beta */
    for (int64_t i = 0; i < m; ++i) {
        double two_r = 2.0 * r[i];
        if (g_mutation == 1) two_r = r[i];                          /* dropped factor 2 */
        double div = (g_mutation == 3) ? (double)m : (double)n;     /* swapped divisor */
        phi[i] = (a[i] - two_r + shift_term) / div;
    }
    for (int64_t j = 0; j < n; ++j) {
        double bj = (g_mutation == 6) ? a[j % m] : b[j];            /* wrong state vector */
        psi[j] = (bj - 2.0 * s[j] + shift_term) / (double)m;
    }

    /* step 8 */
    for (int64_t i = 0; i < m; ++i) a[i] -= r[i];
    for (int64_t j = 0; j < n; ++j) b[j] -= s[j];
    if (g_mutation != 4) *alpha -= beta;                            /* 4: alpha frozen */

    /* stopping quantities at the new iterate */
    double primal = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : primal)
    for (int64_t i = 0; i < m; ++i)
        for (int64_t j = 0; j < n; ++j) primal += C[i * n + j] * X[i * n + j];
    double pphi = 0.0, qpsi = 0.0, l1 = 0.0, l2 = 0.0;
    for (int64_t i = 0; i < m; ++i) {
        pphi += p[i] * phi[i];
        l1 += fabs(r[i]);
        l2 += r[i] * r[i];
    }
    for (int64_t j = 0; j < n; ++j) {
        qpsi += q[j] * psi[j];
        l1 += fabs(s[j]);
        l2 += s[j] * s[j];
    }
    double dual = (pphi + qpsi) / rho;
    if (g_mutation == 5) dual = (pphi - qpsi) / rho;                /* sign slip in q^T nu */
    stats[ORC_PRIMAL] = primal;
    stats[ORC_DUAL] = dual;
    stats[ORC_GAP] = fabs(primal - dual);
    stats[ORC_RES_L1] = l1;
    stats[ORC_RES_L2] = sqrt(l2);
    stats[ORC_DUAL_RES_PREV] = sqrt(dual_sq) / rho;
    stats[ORC_BETA] = beta;
}

/* Full solve.  X (m*n, row-major) holds X0 on entry when warm != 0 and the
 * final iterate on exit; mu, nu hold the warm duals on entry (warm != 0) and
 * phi/rho, psi/rho on exit.  history (optional) receives ORC_NSTATS doubles per
 * iteration.  Returns 0 when the stop rule fired, 1 when max_iter ran out,
 * 2 on a non-finite value, -1 on bad arguments or allocation failure. */
int oracle_solve(int64_t m, int64_t n, const double *C, const double *p, const double *q,
                 double rho, double tol, int64_t max_iter, int stop_rule, int warm,
                 double *X, double *mu, double *nu, double *stats, int64_t *iters, double *history)
{
    if (m <= 0 || n <= 0 || !(rho > 0.0) || max_iter < 0) return -1;
    double *phi = (double *)malloc(sizeof(double) * (size_t)m);
    double *psi = (double *)malloc(sizeof(double) * (size_t)n);
    double *a = (double *)malloc(sizeof(double) * (size_t)m);
    double *b = (double *)malloc(sizeof(double) * (size_t)n);
    double *work = (double *)malloc(sizeof(double) * (size_t)(m + n));
    if (!phi || !psi || !a || !b || !work) {
        free(phi); free(psi); free(a); free(b); free(work);
        return -1;
    }
    if (warm) {
        for (int64_t i = 0; i < m; ++i) phi[i] = rho * mu[i];
        for (int64_t j = 0; j < n; ++j) psi[j] = rho * nu[j];
    } else {
        for (int64_t i = 0; i < m; ++i)
            for (int64_t j = 0; j < n; ++j) X[i * n + j] = p[i] * q[j];
        memset(phi, 0, sizeof(double) * (size_t)m);
        memset(psi, 0, sizeof(double) * (size_t)n);
    }
    double alpha = 0.0;
    oracle_init(m, n, p, q, X, phi, psi, a, b, &alpha);

    int rc = 1;
    int64_t k = 0;
    for (int i = 0; i < ORC_NSTATS; ++i) stats[i] = NAN;
    while (k < max_iter) {
        oracle_iterate(m, n, C, p, q, rho, X, phi, psi, a, b, &alpha, stats, work);
        if (history) memcpy(history + k * ORC_NSTATS, stats, sizeof(double) * ORC_NSTATS);
        ++k;
        int finite = 1;
        for (int i = 0; i < ORC_NSTATS; ++i) finite &= isfinite(stats[i]) ? 1 : 0;
        if (!finite) { rc = 2; break; }
        int rule = (stop_rule & 7) ? (stop_rule & 7) : 3;
        int done = (!(rule & 1) || stats[ORC_GAP] <= tol) && (!(rule & 2) || stats[ORC_RES_L1] <= tol) &&
                   (!(rule & 4) || stats[ORC_DUAL_RES_PREV] <= tol);
        if (done) { rc = 0; break; }
    }
    for (int64_t i = 0; i < m; ++i) mu[i] = phi[i] / rho;
    for (int64_t j = 0; j < n; ++j) nu[j] = psi[j] / rho;
    *iters = k;
    free(phi); free(psi); free(a); free(b); free(work);
    return rc;
}
