/*
 * FP64 CPU oracle for the direct Debye summation of Berlin, Gumerov,
 * Duraiswami and Fushman, "Performance of a GPU-based Direct Summation
 * Algorithm for Computation of Small Angle Scattering Profile".
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the CUDA library links, includes or
 * calls this file; only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg load it.  It shares no code, header, table or constant
 * with the GPU path.
 *
 * Everything here is the plain definition, written out with no blocking,
 * type factoring, recurrence or reordering beyond what the definition needs:
 *
 *   f_j(q)  = sum_{k=1..4} a_k exp(-b_k (q/4pi)^2) + c         (per atom, from its type;
 *             or given per atom and q directly, oracle_profile_atomic)
 *   I(q)    = sum_k sum_j f_k(q) f_j(q) sin(q r_jk)/(q r_jk)   (Section I-A, Eq. 2)
 *           = sum_i f_i^2 + 2 sum_{i<j} f_i f_j sinc(q r_ij)   (only j <= k, Section II)
 *
 * and its derivative with respect to the positions (vector-Jacobian products, with typed or
 * per-atom form factors), the chi^2 of a profile against a target, and pair-distance counts.
 *
 * with sinc(0) = 1 (the diagonal, and coincident atoms), r_ij in double,
 * libm sin/cos/exp/sqrt, and Neumaier-compensated sums.  Per-row partial
 * sums are stored and merged in row order, so results do not depend on the
 * number of OpenMP threads.
 *
 * Build with -ffp-contract=off so that no multiply-add is fused behind the
 * source's back (x86 and aarch64 then round identically).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_PI 3.14159265358979323846264338327950288

/* ---------------------------------------------------------------------- */
/* Neumaier compensated summation                                          */
/* ---------------------------------------------------------------------- */
typedef struct {
    double s, c;
} nsum_t;

static inline void nadd(nsum_t *a, double x)
{
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x))
        a->c += (a->s - t) + x;
    else
        a->c += (x - t) + a->s;
    a->s = t;
}

static inline double nval(const nsum_t *a) { return a->s + a->c; }

static void set_threads(int n_threads)
{
#ifdef _OPENMP
    if (n_threads > 0)
        omp_set_num_threads(n_threads);
#else
    (void)n_threads;
#endif
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---------------------------------------------------------------------- */
/* form factors (per atom; no table by type)                               */
/* ---------------------------------------------------------------------- */

/* f(q) = sum_{k<4} a_k exp(-b_k (q/4pi)^2) + c, coefficients (a1..a4, b1..b4, c). */
static double form_factor(const double *cf, double q)
{
    double s = q / (4.0 * ORACLE_PI);
    double f = cf[8];
    for (int k = 0; k < 4; ++k)
        f += cf[k] * exp(-cf[4 + k] * s * s);
    return f;
}

static int check_types(int64_t n, const int32_t *types, int n_types)
{
    for (int64_t i = 0; i < n; ++i)
        if (types[i] < 0 || types[i] >= n_types)
            return -1;
    return 0;
}

/* f_out[i*n_q + k] = f_{type(i)}(q_k) */
int oracle_form_factors(int64_t n, const int32_t *types, int n_types, const double *coef,
                        int n_q, const double *q, double *f_out)
{
    if (check_types(n, types, n_types))
        return -1;
    for (int64_t i = 0; i < n; ++i)
        for (int k = 0; k < n_q; ++k)
            f_out[i * n_q + k] = form_factor(coef + 9 * types[i], q[k]);
    return 0;
}

static double *atom_form_factors(int64_t n, const int32_t *types, const double *coef, int n_q,
                                 const double *q)
{
    double *f = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1) * (size_t)n_q);
    if (!f)
        return NULL;
    for (int64_t i = 0; i < n; ++i)
        for (int k = 0; k < n_q; ++k)
            f[i * n_q + k] = form_factor(coef + 9 * types[i], q[k]);
    return f;
}

static inline double sinc(double x) { return x == 0.0 ? 1.0 : sin(x) / x; }

static inline double dist(const double *a, const double *b)
{
    double dx = a[0] - b[0], dy = a[1] - b[1], dz = a[2] - b[2];
    return sqrt(dx * dx + dy * dy + dz * dz);
}

/* ---------------------------------------------------------------------- */
/* Eq. 2 over i<j (the paper's j <= k form), compensated                   */
/* ---------------------------------------------------------------------- */

/*
 * I_out[k]     = I(q_k)
 * kappa_out[k] = (sum_i f_i^2 + 2 sum_{i<j} |f_i f_j sinc|) / |I(q_k)|  (conditioning; may be NULL)
 * Returns 0, -1 on a type out of range, -2 on allocation failure.
 */
static int profile_core(int64_t n, const double *xyz, const double *f, int n_q, const double *q,
                        int n_threads, double *I_out, double *kappa_out);

int oracle_profile(int64_t n, const double *xyz, const int32_t *types, int n_types,
                   const double *coef, int n_q, const double *q, int n_threads,
                   double *I_out, double *kappa_out)
{
    if (check_types(n, types, n_types))
        return -1;
    double *f = atom_form_factors(n, types, coef, n_q, q);
    if (!f)
        return -2;
    int rc = profile_core(n, xyz, f, n_q, q, n_threads, I_out, kappa_out);
    free(f);
    return rc;
}

/*
 * The same sum with every atom's form factor given directly, with no types: ff[k * n + i] =
 * f_i(q_k), one row of N values per q (Section II keeps, for each q value, one form factor per
 * atom; Section I-A: with a hydration layer the products f_k f_j do not reduce to a few types).
 * Returns 0 or -2 on allocation failure.
 */
int oracle_profile_atomic(int64_t n, const double *xyz, const double *ff, int n_q, const double *q,
                          int n_threads, double *I_out, double *kappa_out)
{
    double *f = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1) * (size_t)n_q);
    if (!f)
        return -2;
    for (int64_t i = 0; i < n; ++i)
        for (int k = 0; k < n_q; ++k)
            f[i * n_q + k] = ff[(int64_t)k * n + i];
    int rc = profile_core(n, xyz, f, n_q, q, n_threads, I_out, kappa_out);
    free(f);
    return rc;
}

/* f[i * n_q + k] = f_i(q_k), atom-major. */
static int profile_core(int64_t n, const double *xyz, const double *f, int n_q, const double *q,
                        int n_threads, double *I_out, double *kappa_out)
{
    if (n == 0) {
        for (int k = 0; k < n_q; ++k) {
            I_out[k] = 0.0;
            if (kappa_out)
                kappa_out[k] = 0.0;
        }
        return 0;
    }
    double *row = (double *)malloc(sizeof(double) * (size_t)n * (size_t)n_q);
    double *rowabs = (double *)malloc(sizeof(double) * (size_t)n * (size_t)n_q);
    if (!row || !rowabs) {
        free(row);
        free(rowabs);
        return -2;
    }
    set_threads(n_threads);
    int fail = 0;
#pragma omp parallel
    {
        nsum_t *acc = (nsum_t *)malloc(sizeof(nsum_t) * (size_t)n_q);
        double *aab = (double *)malloc(sizeof(double) * (size_t)n_q);
        if (!acc || !aab) {
#pragma omp atomic write
            fail = 1;
        }
#pragma omp for schedule(dynamic, 8)
        for (int64_t i = 0; i < n; ++i) {
            if (!acc || !aab)
                continue;
            memset(acc, 0, sizeof(nsum_t) * (size_t)n_q);
            memset(aab, 0, sizeof(double) * (size_t)n_q);
            const double *fi = f + i * n_q;
            for (int64_t j = i + 1; j < n; ++j) {
                const double *fj = f + j * n_q;
                double r = dist(xyz + 3 * i, xyz + 3 * j);
                for (int k = 0; k < n_q; ++k) {
                    double term = fi[k] * fj[k] * sinc(q[k] * r);
                    nadd(&acc[k], term);
                    aab[k] += fabs(term);
                }
            }
            for (int k = 0; k < n_q; ++k) {
                row[i * n_q + k] = nval(&acc[k]);
                rowabs[i * n_q + k] = aab[k];
            }
        }
        free(acc);
        free(aab);
    }
    if (!fail) {
        for (int k = 0; k < n_q; ++k) {
            nsum_t tot = {0.0, 0.0};
            double mag = 0.0;
            for (int64_t i = 0; i < n; ++i) {
                double d = f[i * n_q + k] * f[i * n_q + k];
                nadd(&tot, d);
                mag += d;
            }
            for (int64_t i = 0; i < n; ++i) {
                nadd(&tot, 2.0 * row[i * n_q + k]);
                mag += 2.0 * rowabs[i * n_q + k];
            }
            I_out[k] = nval(&tot);
            if (kappa_out)
                kappa_out[k] = I_out[k] != 0.0 ? mag / fabs(I_out[k]) : INFINITY;
        }
    }
    free(row);
    free(rowabs);
    return fail ? -2 : 0;
}

/* ---------------------------------------------------------------------- */
/* Eq. 2 literally: both sums over all N atoms, diagonal included          */
/* ---------------------------------------------------------------------- */

/* Single-threaded; meant for small N (brute force).  Returns 0 / -1 / -2. */
int oracle_profile_full(int64_t n, const double *xyz, const int32_t *types, int n_types,
                        const double *coef, int n_q, const double *q, double *I_out)
{
    if (check_types(n, types, n_types))
        return -1;
    double *f = atom_form_factors(n, types, coef, n_q, q);
    if (!f)
        return -2;
    for (int k = 0; k < n_q; ++k) {
        nsum_t tot = {0.0, 0.0};
        for (int64_t a = 0; a < n; ++a)
            for (int64_t b = 0; b < n; ++b) {
                double r = dist(xyz + 3 * a, xyz + 3 * b);
                nadd(&tot, f[a * n_q + k] * f[b * n_q + k] * sinc(q[k] * r));
            }
        I_out[k] = nval(&tot);
    }
    free(f);
    return 0;
}

/* ---------------------------------------------------------------------- */
/* per-type-pair sinc sums                                                 */
/* ---------------------------------------------------------------------- */

/* Index of the unordered type pair {a, b}, a <= b, row-major over the upper triangle. */
static int pair_index(int a, int b, int T)
{
    if (a > b) {
        int t = a;
        a = b;
        b = t;
    }
    return a * T - a * (a - 1) / 2 + (b - a);
}

/*
 * S_out[p*n_q + k] = sum over unordered pairs i<j whose types are {a,b} of sinc(q_k r_ij),
 * p = index of {a,b}.  Single-threaded per pair row; the row order is fixed.
 */
int oracle_pair_sums(int64_t n, const double *xyz, const int32_t *types, int n_types, int n_q,
                     const double *q, int n_threads, double *S_out)
{
    if (check_types(n, types, n_types))
        return -1;
    int P = n_types * (n_types + 1) / 2;
    double *row = (double *)calloc((size_t)(n > 0 ? n : 1) * (size_t)P * (size_t)n_q, sizeof(double));
    if (!row)
        return -2;
    set_threads(n_threads);
    int fail = 0;
#pragma omp parallel
    {
        nsum_t *acc = (nsum_t *)malloc(sizeof(nsum_t) * (size_t)P * (size_t)n_q);
        if (!acc) {
#pragma omp atomic write
            fail = 1;
        }
#pragma omp for schedule(dynamic, 8)
        for (int64_t i = 0; i < n; ++i) {
            if (!acc)
                continue;
            memset(acc, 0, sizeof(nsum_t) * (size_t)P * (size_t)n_q);
            for (int64_t j = i + 1; j < n; ++j) {
                int p = pair_index(types[i], types[j], n_types);
                double r = dist(xyz + 3 * i, xyz + 3 * j);
                for (int k = 0; k < n_q; ++k)
                    nadd(&acc[p * n_q + k], sinc(q[k] * r));
            }
            for (int p = 0; p < P * n_q; ++p)
                row[(size_t)i * P * n_q + p] = nval(&acc[p]);
        }
        free(acc);
    }
    if (!fail)
        for (int p = 0; p < P * n_q; ++p) {
            nsum_t tot = {0.0, 0.0};
            for (int64_t i = 0; i < n; ++i)
                nadd(&tot, row[(size_t)i * P * n_q + p]);
            S_out[p] = nval(&tot);
        }
    free(row);
    return fail ? -2 : 0;
}

/* ---------------------------------------------------------------------- */
/* gradient: the derivative of Eq. 2 with respect to the positions         */
/* ---------------------------------------------------------------------- */

/*
 * Vector-Jacobian product of Eq. 2:
 *   grad_out[i] = sum_q gI_q dI(q)/dx_i
 *               = sum_{j != i} [ sum_q gI_q 2 f_i f_j (cos(q r) - sinc(q r)) / r^2 ] (x_i - x_j)
 * because d sinc(q r)/dr = (cos(q r) - sinc(q r)) / r.  Terms with q = 0 or r = 0 are
 * zero (the bracket vanishes, or x_i - x_j does).  Each row i sums over all j != i, so
 * the result needs no scatter.  Returns 0 / -1 / -2.
 */
/* f[i * n_q + k] = f_i(q_k), atom-major. */
static void vjp_core(int64_t n, const double *xyz, const double *f, int n_q, const double *q,
                     const double *gI, int n_threads, double *grad_out)
{
    set_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 8)
    for (int64_t i = 0; i < n; ++i) {
        nsum_t g[3] = {{0, 0}, {0, 0}, {0, 0}};
        for (int64_t j = 0; j < n; ++j) {
            if (j == i)
                continue;
            double r = dist(xyz + 3 * i, xyz + 3 * j);
            if (r == 0.0)
                continue;
            nsum_t w = {0.0, 0.0};
            for (int k = 0; k < n_q; ++k) {
                if (q[k] == 0.0)
                    continue;
                double x = q[k] * r;
                double br = (cos(x) - sin(x) / x) / (r * r);
                nadd(&w, gI[k] * 2.0 * f[i * n_q + k] * f[j * n_q + k] * br);
            }
            double wij = nval(&w);
            for (int c = 0; c < 3; ++c)
                nadd(&g[c], wij * (xyz[3 * i + c] - xyz[3 * j + c]));
        }
        for (int c = 0; c < 3; ++c)
            grad_out[3 * i + c] = nval(&g[c]);
    }
}

int oracle_vjp(int64_t n, const double *xyz, const int32_t *types, int n_types, const double *coef,
               int n_q, const double *q, const double *gI, int n_threads, double *grad_out)
{
    if (check_types(n, types, n_types))
        return -1;
    double *f = atom_form_factors(n, types, coef, n_q, q);
    if (!f)
        return -2;
    vjp_core(n, xyz, f, n_q, q, gI, n_threads, grad_out);
    free(f);
    return 0;
}

/*
 * The same product with per-atom form factors ff[k * n + i] = f_i(q_k) (no types): the form
 * factors do not depend on the positions, so the bracket above holds with f_i(q), f_j(q) per atom.
 */
int oracle_vjp_atomic(int64_t n, const double *xyz, const double *ff, int n_q, const double *q,
                      const double *gI, int n_threads, double *grad_out)
{
    double *f = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1) * (size_t)n_q);
    if (!f)
        return -2;
    for (int k = 0; k < n_q; ++k)
        for (int64_t i = 0; i < n; ++i)
            f[i * n_q + k] = ff[i + (int64_t)k * n];
    vjp_core(n, xyz, f, n_q, q, gI, n_threads, grad_out);
    free(f);
    return 0;
}

/*
 * chi^2 = sum_q w_q (I(q) - T(q))^2 and its gradient d chi^2 / d x (= the VJP with
 * gI_q = 2 w_q (I(q) - T(q))).  I_out (may be NULL) receives I(q).
 */
int oracle_chi2_grad(int64_t n, const double *xyz, const int32_t *types, int n_types,
                     const double *coef, int n_q, const double *q, const double *target,
                     const double *weights, int n_threads, double *chi2_out, double *grad_out,
                     double *I_out)
{
    double *I = (double *)malloc(sizeof(double) * (size_t)n_q);
    double *gI = (double *)malloc(sizeof(double) * (size_t)n_q);
    if (!I || !gI) {
        free(I);
        free(gI);
        return -2;
    }
    int rc = oracle_profile(n, xyz, types, n_types, coef, n_q, q, n_threads, I, NULL);
    if (rc == 0) {
        nsum_t c2 = {0.0, 0.0};
        for (int k = 0; k < n_q; ++k) {
            double d = I[k] - target[k];
            nadd(&c2, weights[k] * d * d);
            gI[k] = 2.0 * weights[k] * d;
        }
        *chi2_out = nval(&c2);
        if (I_out)
            memcpy(I_out, I, sizeof(double) * (size_t)n_q);
        if (grad_out)
            rc = oracle_vjp(n, xyz, types, n_types, coef, n_q, q, gI, n_threads, grad_out);
    }
    free(I);
    free(gI);
    return rc;
}

/* ---------------------------------------------------------------------- */
/* pair-distance histogram                                                 */
/* ---------------------------------------------------------------------- */

/*
 * Exact integer counts of unordered pairs i<j by type pair and distance bin.
 * Distances are squared in float32 with a fixed sequence of roundings,
 *   dx = x_i - x_j (and dy, dz);  r2 = fmaf(dz, dz, fmaf(dy, dy, dx*dx)),
 * and bin k holds the pairs with e_k^2 <= r2 < e_{k+1}^2, where
 *   w = r_max / n_bins,  e_k = (float)k * w,  e_k^2 = e_k * e_k   (all float32).
 * Pairs with r2 >= e_{n_bins}^2 are not binned; they are counted in *dropped.
 * hist_out[p*n_bins + k] (p = type-pair index) is overwritten.
 */
int oracle_pair_histogram(int64_t n, const float *xyz, const int32_t *types, int n_types,
                          int n_bins, float r_max, int32_t *hist_out, int64_t *dropped)
{
    if (check_types(n, types, n_types) || n_bins <= 0)
        return -1;
    int P = n_types * (n_types + 1) / 2;
    float w = r_max / (float)n_bins;
    float *e2 = (float *)malloc(sizeof(float) * (size_t)(n_bins + 1));
    if (!e2)
        return -2;
    for (int k = 0; k <= n_bins; ++k) {
        float ek = (float)k * w;
        e2[k] = ek * ek;
    }
    memset(hist_out, 0, sizeof(int32_t) * (size_t)P * (size_t)n_bins);
    int64_t drop = 0;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = i + 1; j < n; ++j) {
            float dx = xyz[3 * i] - xyz[3 * j];
            float dy = xyz[3 * i + 1] - xyz[3 * j + 1];
            float dz = xyz[3 * i + 2] - xyz[3 * j + 2];
            float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
            /* k = max{k in [0, n_bins] : e2[k] <= r2} by bisection (e2 is increasing) */
            int lo = 0, hi = n_bins;
            while (lo < hi) {
                int mid = (lo + hi + 1) / 2;
                if (e2[mid] <= r2)
                    lo = mid;
                else
                    hi = mid - 1;
            }
            if (lo >= n_bins)
                ++drop;
            else
                hist_out[pair_index(types[i], types[j], n_types) * n_bins + lo] += 1;
        }
    if (dropped)
        *dropped = drop;
    free(e2);
    return 0;
}
