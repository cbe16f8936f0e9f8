/*
 * edm_oracle.c -- plain, slow, FP64 CPU reference of the all-pairs CCM path.
 *
 * TEST INFRASTRUCTURE.  Only the tests, the smoke check and the CPU-baseline
 * leg of the benchmark may load this library.  The product path (the CUDA
 * library and its Python binding) never calls it, and the two share no code:
 * no headers, no helpers, no tables.
 *
 * Everything is computed in IEEE double precision from the caller's values,
 * with no blocking, fusion or reordering beyond what the paper's algorithms
 * state.  Build with -ffp-contract=off so every product is rounded before it
 * is added (the operation order below is the definition of the reference).
 *
 * What each routine follows (arXiv 2011.11082, "mpEDM"):
 *   - time-delay embedding v(t) = (x(t), x(t-tau), ..., x(t-(E-1)tau)),
 *     Sec. II-B; lags run backwards from the newest coordinate;
 *   - kNN: all-to-all squared Euclidean distances over the E lags computed
 *     on the fly, then a partial sort keeping the E+1 nearest, Algorithm 3
 *     and the text of Sec. III-B (nearest = ascending distance; ties go to
 *     the smaller candidate index);
 *   - normalize: distances to exponential scale, each row normalised,
 *     the normalisation step of Algorithm 1; weights u_n = exp(-d_n / d_1), w = u/sum(u)
 *     with d_1 the nearest distance; when d_1 = 0 only exact duplicates
 *     (d_n = 0) carry weight;
 *   - lookup: prediction(t) = sum_n w[t,n] * y(s_n + Tp), Algorithm 5, one
 *     step ahead (Tp = 1) as in Sec. II-B;
 *   - corrcoef: Pearson correlation, two-pass (means first), NaN when either
 *     side has zero variance;
 *   - simplex projection (phase 1, Algorithm 1): library = first floor(T/2)
 *     samples, target = the rest, each half embedded within itself; optimal
 *     E = argmax over E of rho_E (NaN counts as -inf, ties -> smallest E);
 *   - CCM (phase 2, Algorithm 2): per library series i and embedding
 *     dimension E one kNN table over the library's own embedded points
 *     (queries = candidates = t in [(E-1)tau, T-1-Tp], a query never matches
 *     candidates within the exclusion radius of itself, radius 0 = itself
 *     only, radius -1 = no exclusion), reused for every target j with
 *     optE[j] = E; rho[i][j] = corrcoef(observed y_j(t+Tp), prediction).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_ERR_INVALID 1
#define ORC_ERR_NOMEM 2

/* ----------------------------------------------------------------------- */
/* Distance between embedded points a(ta) and b(tb): sum over the E lags.   */
/* ----------------------------------------------------------------------- */
static double embed_dist2(const double *xa, int64_t ta, const double *xb, int64_t tb, int E, int tau)
{
    double d = 0.0;
    for (int m = 0; m < E; ++m) {
        double diff = xa[ta - (int64_t)m * tau] - xb[tb - (int64_t)m * tau];
        double sq = diff * diff;
        d = d + sq;
    }
    return d;
}

static int pair_before(double da, int64_t ia, double db, int64_t ib)
{
    return (da < db) || (da == db && ia < ib);
}

/*
 * The k nearest candidates of query point t (series xq) among candidate
 * points s in [s_lo, s_hi] of series xc.  When `same` is set the two series
 * are the same and candidates with |s - t| <= excl are skipped (excl < 0:
 * none skipped).  Partial sort by insertion into a sorted list of length k.
 * Returns the number of neighbours found (k unless too few candidates).
 */
static int knn_query(const double *xq, int64_t t, const double *xc, int64_t s_lo, int64_t s_hi,
                     int E, int tau, int same, int excl, int k, int64_t *idx, double *d2)
{
    int n = 0;
    for (int64_t s = s_lo; s <= s_hi; ++s) {
        if (same && excl >= 0 && llabs(s - t) <= excl)
            continue;
        double d = embed_dist2(xq, t, xc, s, E, tau);
        int pos;
        if (n < k) {
            pos = n++;
        } else if (pair_before(d, s, d2[k - 1], idx[k - 1])) {
            pos = k - 1;
        } else {
            continue;
        }
        while (pos > 0 && pair_before(d, s, d2[pos - 1], idx[pos - 1])) {
            d2[pos] = d2[pos - 1];
            idx[pos] = idx[pos - 1];
            --pos;
        }
        d2[pos] = d;
        idx[pos] = s;
    }
    return n;
}

/* knn_query restricted to the candidates whose bit is set in `mask`
 * (bit s of word s / 32): a library subset for the convergence test. */
static int knn_query_masked(const double *x, int64_t t, int64_t s_lo, int64_t s_hi, const uint32_t *mask, int E,
                            int tau, int excl, int k, int64_t *idx, double *d2)
{
    int n = 0;
    for (int64_t s = s_lo; s <= s_hi; ++s) {
        if (!((mask[s / 32] >> (s % 32)) & 1u))
            continue;
        if (excl >= 0 && llabs(s - t) <= excl)
            continue;
        double d = embed_dist2(x, t, x, s, E, tau);
        int pos;
        if (n < k) {
            pos = n++;
        } else if (pair_before(d, s, d2[k - 1], idx[k - 1])) {
            pos = k - 1;
        } else {
            continue;
        }
        while (pos > 0 && pair_before(d, s, d2[pos - 1], idx[pos - 1])) {
            d2[pos] = d2[pos - 1];
            idx[pos] = idx[pos - 1];
            --pos;
        }
        d2[pos] = d;
        idx[pos] = s;
    }
    return n;
}

/* Distances (squared) of one kNN row -> normalised exponential weights. */
static void simplex_weights(const double *d2, int k, double *w)
{
    double d1 = sqrt(d2[0]);
    double sum = 0.0;
    for (int n = 0; n < k; ++n) {
        double dn = sqrt(d2[n]);
        double u;
        if (d1 > 0.0)
            u = exp(-dn / d1);
        else
            u = (dn == 0.0) ? 1.0 : 0.0;
        w[n] = u;
        sum = sum + u;
    }
    for (int n = 0; n < k; ++n)
        w[n] = w[n] / sum;
}

static double pearson(const double *a, const double *b, int64_t n)
{
    if (n < 2)
        return NAN;
    double ma = 0.0, mb = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        ma = ma + a[i];
        mb = mb + b[i];
    }
    ma = ma / (double)n;
    mb = mb / (double)n;
    double sab = 0.0, saa = 0.0, sbb = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double da = a[i] - ma, db = b[i] - mb;
        sab = sab + da * db;
        saa = saa + da * da;
        sbb = sbb + db * db;
    }
    if (!(saa > 0.0) || !(sbb > 0.0))
        return NAN;
    return sab / sqrt(saa * sbb);
}

/* ----------------------------------------------------------------------- */
/* Exported pieces                                                           */
/* ----------------------------------------------------------------------- */

/* Number of query rows of a CCM table (queries t in [(E-1)tau, T-1-Tp]). */
int64_t orc_ccm_rows(int64_t T, int E, int tau, int Tp)
{
    int64_t n = T - Tp - (int64_t)(E - 1) * tau;
    return n > 0 ? n : 0;
}

/*
 * Generic kNN over two series (used by the brute-force checks and by the
 * tables below).  Rows are queries t = t_lo..t_hi in order; each row holds k
 * candidate indices s (not shifted by Tp) and squared distances, ascending.
 */
int orc_knn(const double *xq, int64_t t_lo, int64_t t_hi, const double *xc, int64_t s_lo, int64_t s_hi,
            int E, int tau, int same, int excl, int k, int64_t *idx, double *d2)
{
    if (E < 1 || tau < 1 || k < 1 || t_hi < t_lo || s_hi < s_lo)
        return ORC_ERR_INVALID;
    if (t_lo < (int64_t)(E - 1) * tau || s_lo < (int64_t)(E - 1) * tau)
        return ORC_ERR_INVALID;
    for (int64_t t = t_lo; t <= t_hi; ++t) {
        int64_t r = t - t_lo;
        int got = knn_query(xq, t, xc, s_lo, s_hi, E, tau, same, excl, k, idx + r * k, d2 + r * k);
        if (got < k)
            return ORC_ERR_INVALID;
    }
    return ORC_OK;
}

void orc_weights(const double *d2, int k, double *w) { simplex_weights(d2, k, w); }

double orc_pearson(const double *a, const double *b, int64_t n) { return pearson(a, b, n); }

/*
 * Phase 1 for one series and one E (Algorithm 1, simplex projection):
 * returns rho_E, or NaN when it is undefined.
 */
double orc_simplex_rho(const double *x, int64_t T, int E, int tau, int Tp)
{
    int64_t h = T / 2;
    const double *lib = x;
    const double *tgt = x + h;
    int64_t Tl = h, Tt = T - h;
    int64_t L = (int64_t)(E - 1) * tau;
    int64_t t_lo = L, t_hi = Tt - 1 - Tp;
    int64_t s_lo = L, s_hi = Tl - 1 - Tp;
    int k = E + 1;
    if (t_hi < t_lo || s_hi - s_lo + 1 < k)
        return NAN;
    int64_t nq = t_hi - t_lo + 1;
    int64_t *idx = (int64_t *)malloc(sizeof(int64_t) * (size_t)k);
    double *d2 = (double *)malloc(sizeof(double) * (size_t)k);
    double *w = (double *)malloc(sizeof(double) * (size_t)k);
    double *pred = (double *)malloc(sizeof(double) * (size_t)nq);
    double *obs = (double *)malloc(sizeof(double) * (size_t)nq);
    double rho = NAN;
    if (idx && d2 && w && pred && obs) {
        for (int64_t t = t_lo; t <= t_hi; ++t) {
            knn_query(tgt, t, lib, s_lo, s_hi, E, tau, 0, -1, k, idx, d2);
            simplex_weights(d2, k, w);
            double p = 0.0;
            for (int n = 0; n < k; ++n)
                p = p + w[n] * lib[idx[n] + Tp];
            pred[t - t_lo] = p;
            obs[t - t_lo] = tgt[t + Tp];
        }
        rho = pearson(obs, pred, nq);
    }
    free(idx);
    free(d2);
    free(w);
    free(pred);
    free(obs);
    return rho;
}

/* argmax over E of rho_E; NaN never wins; ties go to the smaller E. */
static int32_t argmax_E(const double *rho, int E_max)
{
    int32_t best = 1;
    double bv = -INFINITY;
    int any = 0;
    for (int E = 1; E <= E_max; ++E) {
        double v = rho[E - 1];
        if (isnan(v))
            continue;
        if (!any || v > bv) {
            bv = v;
            best = E;
            any = 1;
        }
    }
    return best;
}

int orc_optimal_E(const double *Y, int64_t N, int64_t T, int64_t ldY, int E_max, int tau, int Tp,
                  int32_t *optE, double *rho_by_E, int nthreads)
{
    if (N < 1 || T < 2 || ldY < T || E_max < 1 || tau < 1 || Tp < 0)
        return ORC_ERR_INVALID;
#ifdef _OPENMP
    if (nthreads < 1)
        nthreads = 1;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
#endif
    for (int64_t i = 0; i < N; ++i) {
        double rho_local[64];
        double *rho = rho_by_E ? rho_by_E + i * E_max : rho_local;
        for (int E = 1; E <= E_max; ++E)
            rho[E - 1] = orc_simplex_rho(Y + i * ldY, T, E, tau, Tp);
        optE[i] = argmax_E(rho, E_max);
    }
    (void)nthreads;
    return ORC_OK;
}

/*
 * Phase 2 table for one library series and one E: rows t = (E-1)tau ..
 * T-1-Tp, k = E+1 columns of candidate indices s (not shifted) and weights.
 */
int orc_ccm_table(const double *x, int64_t T, int E, int tau, int Tp, int excl, int64_t *idx, double *w)
{
    int64_t L = (int64_t)(E - 1) * tau;
    int64_t t_lo = L, t_hi = T - 1 - Tp;
    int k = E + 1;
    if (t_hi < t_lo)
        return ORC_ERR_INVALID;
    double *d2 = (double *)malloc(sizeof(double) * (size_t)k);
    if (!d2)
        return ORC_ERR_NOMEM;
    int rc = ORC_OK;
    for (int64_t t = t_lo; t <= t_hi; ++t) {
        int64_t r = t - t_lo;
        int got = knn_query(x, t, x, t_lo, t_hi, E, tau, 1, excl, k, idx + r * k, d2);
        if (got < k) {
            rc = ORC_ERR_INVALID;
            break;
        }
        simplex_weights(d2, k, w + r * k);
    }
    free(d2);
    return rc;
}

/* Squared distances of a table row recomputed at frozen indices. */
int orc_ccm_table_d2(const double *x, int64_t T, int E, int tau, int Tp, const int64_t *idx, double *d2)
{
    int64_t L = (int64_t)(E - 1) * tau;
    int64_t nq = orc_ccm_rows(T, E, tau, Tp);
    int k = E + 1;
    for (int64_t r = 0; r < nq; ++r)
        for (int n = 0; n < k; ++n)
            d2[r * k + n] = embed_dist2(x, L + r, x, idx[r * k + n], E, tau);
    return ORC_OK;
}

/* Lookup + corrcoef for one target series with a given table (Alg. 5 + Alg. 1). */
double orc_lookup_rho(const double *y, int64_t T, int E, int tau, int Tp, const int64_t *idx, const double *w)
{
    int64_t L = (int64_t)(E - 1) * tau;
    int64_t nq = orc_ccm_rows(T, E, tau, Tp);
    int k = E + 1;
    double *pred = (double *)malloc(sizeof(double) * (size_t)(nq > 0 ? nq : 1));
    double *obs = (double *)malloc(sizeof(double) * (size_t)(nq > 0 ? nq : 1));
    double rho = NAN;
    if (pred && obs) {
        for (int64_t r = 0; r < nq; ++r) {
            double p = 0.0;
            for (int n = 0; n < k; ++n)
                p = p + w[r * k + n] * y[idx[r * k + n] + Tp];
            pred[r] = p;
            obs[r] = y[L + r + Tp];
        }
        rho = pearson(obs, pred, nq);
    }
    free(pred);
    free(obs);
    return rho;
}

/*
 * rho for a frozen table: distances recomputed from the (possibly perturbed)
 * library at the given indices, then weights, lookup and corrcoef.  Used by
 * the finite-difference checks of the adjoint (indices held fixed).
 */
double orc_rho_frozen(const double *x, const double *y, int64_t T, int E, int tau, int Tp, const int64_t *idx)
{
    int64_t nq = orc_ccm_rows(T, E, tau, Tp);
    int k = E + 1;
    double *d2 = (double *)malloc(sizeof(double) * (size_t)(nq * k));
    double *w = (double *)malloc(sizeof(double) * (size_t)(nq * k));
    double rho = NAN;
    if (d2 && w) {
        orc_ccm_table_d2(x, T, E, tau, Tp, idx, d2);
        for (int64_t r = 0; r < nq; ++r)
            simplex_weights(d2 + r * k, k, w + r * k);
        rho = orc_lookup_rho(y, T, E, tau, Tp, idx, w);
    }
    free(d2);
    free(w);
    return rho;
}

/*
 * Phase 2 over selected library rows and target columns (Algorithm 2):
 * for each library row, one table per distinct E among the selected targets,
 * reused for every target with that E.  rho is [n_rows][n_cols].
 * cols == NULL selects all N targets in order.
 */
int orc_ccm_rho_rows(const double *Y, int64_t N, int64_t T, int64_t ldY, const int32_t *optE,
                     const int64_t *rows, int64_t n_rows, const int64_t *cols, int64_t n_cols,
                     int tau, int Tp, int excl, double *rho, int nthreads)
{
    if (N < 1 || T < 2 || ldY < T || tau < 1 || Tp < 0 || n_rows < 0)
        return ORC_ERR_INVALID;
    if (!cols)
        n_cols = N;
    int E_top = 0;
    for (int64_t c = 0; c < n_cols; ++c) {
        int64_t j = cols ? cols[c] : c;
        if (j < 0 || j >= N || optE[j] < 1)
            return ORC_ERR_INVALID;
        if (optE[j] > E_top)
            E_top = optE[j];
    }
    int rc_all = ORC_OK;
#ifdef _OPENMP
    if (nthreads < 1)
        nthreads = 1;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
#endif
    for (int64_t r = 0; r < n_rows; ++r) {
        int64_t i = rows[r];
        const double *x = Y + i * ldY;
        for (int E = 1; E <= E_top; ++E) {
            int used = 0;
            for (int64_t c = 0; c < n_cols && !used; ++c)
                used = optE[cols ? cols[c] : c] == E;
            if (!used)
                continue;
            int64_t nq = orc_ccm_rows(T, E, tau, Tp);
            int k = E + 1;
            int64_t *idx = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nq * k));
            double *w = (double *)malloc(sizeof(double) * (size_t)(nq * k));
            int rc = (idx && w) ? orc_ccm_table(x, T, E, tau, Tp, excl, idx, w) : ORC_ERR_NOMEM;
            if (rc != ORC_OK) {
#ifdef _OPENMP
#pragma omp atomic write
#endif
                rc_all = rc;
            } else {
                for (int64_t c = 0; c < n_cols; ++c) {
                    int64_t j = cols ? cols[c] : c;
                    if (optE[j] != E)
                        continue;
                    rho[r * n_cols + c] = orc_lookup_rho(Y + j * ldY, T, E, tau, Tp, idx, w);
                }
            }
            free(idx);
            free(w);
        }
    }
    (void)nthreads;
    return rc_all;
}

/*
 * Time-delay cross mapping (the lagged cross-map skill the paper cites for
 * its adjacency maps, Sec. II-A; not defined there -- reading): for lags
 * lag_min..lag_max, one kNN table per library and E over the points whose
 * every lag stays inside the series -- queries = candidates = t in
 * [max((E-1)tau, -lag_min), T-1-max(lag_max, 0)] -- and for each lag l
 * prediction(t) = sum_n w[t,n] * y(s_n + l), observed y(t + l),
 * rho_l = corrcoef.  With lag_min = lag_max = Tp >= 0 this is exactly the
 * CCM above.  rho is [n_lags][n_rows][N] (library rows x all targets).
 */
int orc_ccm_rho_lags(const double *Y, int64_t N, int64_t T, int64_t ldY, const int32_t *optE,
                     const int64_t *rows, int64_t n_rows, int tau, int lag_min, int lag_max, int excl,
                     double *rho, int nthreads)
{
    if (N < 1 || T < 2 || ldY < T || tau < 1 || lag_max < lag_min || n_rows < 0)
        return ORC_ERR_INVALID;
    const int n_lags = lag_max - lag_min + 1;
    int E_top = 0;
    for (int64_t j = 0; j < N; ++j) {
        if (optE[j] < 1)
            return ORC_ERR_INVALID;
        if (optE[j] > E_top)
            E_top = optE[j];
    }
    int rc_all = ORC_OK;
#ifdef _OPENMP
    if (nthreads < 1)
        nthreads = 1;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
#endif
    for (int64_t r = 0; r < n_rows; ++r) {
        const double *x = Y + rows[r] * ldY;
        for (int E = 1; E <= E_top; ++E) {
            int used = 0;
            for (int64_t j = 0; j < N && !used; ++j)
                used = optE[j] == E;
            if (!used)
                continue;
            int64_t L = (int64_t)(E - 1) * tau;
            int64_t A = L > -(int64_t)lag_min ? L : -(int64_t)lag_min;
            int64_t B = T - 1 - (lag_max > 0 ? lag_max : 0);
            int k = E + 1;
            int64_t nq = B - A + 1;
            int rc = nq > k ? ORC_OK : ORC_ERR_INVALID;
            int64_t *idx = NULL;
            double *w = NULL, *d2 = NULL, *pred = NULL, *obs = NULL;
            if (rc == ORC_OK) {
                idx = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nq * k));
                w = (double *)malloc(sizeof(double) * (size_t)(nq * k));
                d2 = (double *)malloc(sizeof(double) * (size_t)k);
                pred = (double *)malloc(sizeof(double) * (size_t)nq);
                obs = (double *)malloc(sizeof(double) * (size_t)nq);
                if (!idx || !w || !d2 || !pred || !obs)
                    rc = ORC_ERR_NOMEM;
            }
            for (int64_t t = A; rc == ORC_OK && t <= B; ++t) {
                int64_t q = t - A;
                if (knn_query(x, t, x, A, B, E, tau, 1, excl, k, idx + q * k, d2) < k)
                    rc = ORC_ERR_INVALID;
                else
                    simplex_weights(d2, k, w + q * k);
            }
            if (rc == ORC_OK) {
                for (int64_t j = 0; j < N; ++j) {
                    if (optE[j] != E)
                        continue;
                    const double *y = Y + j * ldY;
                    for (int l = lag_min; l <= lag_max; ++l) {
                        for (int64_t q = 0; q < nq; ++q) {
                            double p = 0.0;
                            for (int n = 0; n < k; ++n)
                                p = p + w[q * k + n] * y[idx[q * k + n] + l];
                            pred[q] = p;
                            obs[q] = y[A + q + l];
                        }
                        rho[((int64_t)(l - lag_min) * n_rows + r) * N + j] = pearson(obs, pred, nq);
                    }
                }
            } else {
#ifdef _OPENMP
#pragma omp atomic write
#endif
                rc_all = rc;
            }
            free(idx);
            free(w);
            free(d2);
            free(pred);
            free(obs);
        }
    }
    (void)nthreads;
    (void)n_lags;
    return rc_all;
}

/*
 * CCM convergence (the library-size test of the original CCM that the paper
 * leaves out, Sec. III-A): the cross map of every library row with its
 * candidate points restricted to a subset -- bit s of mask[u * words + s/32]
 * set -- for each of n_sub subsets; queries are all points
 * t in [(E-1)tau, T-1-Tp] as in the plain cross map.  With every bit set it
 * is exactly that cross map.  rho is [n_sub][n_rows][N].
 */
int orc_ccm_rho_subsets(const double *Y, int64_t N, int64_t T, int64_t ldY, const int32_t *optE,
                        const int64_t *rows, int64_t n_rows, const uint32_t *masks, int64_t n_sub, int64_t words,
                        int tau, int Tp, int excl, double *rho, int nthreads)
{
    if (N < 1 || T < 2 || ldY < T || tau < 1 || Tp < 0 || n_rows < 0 || n_sub < 1 || words * 32 < T)
        return ORC_ERR_INVALID;
    int E_top = 0;
    for (int64_t j = 0; j < N; ++j) {
        if (optE[j] < 1)
            return ORC_ERR_INVALID;
        if (optE[j] > E_top)
            E_top = optE[j];
    }
    int rc_all = ORC_OK;
#ifdef _OPENMP
    if (nthreads < 1)
        nthreads = 1;
#pragma omp parallel for collapse(2) schedule(dynamic, 1) num_threads(nthreads)
#endif
    for (int64_t u = 0; u < n_sub; ++u)
        for (int64_t r = 0; r < n_rows; ++r) {
            const double *x = Y + rows[r] * ldY;
            const uint32_t *mask = masks + u * words;
            for (int E = 1; E <= E_top; ++E) {
                int used = 0;
                for (int64_t j = 0; j < N && !used; ++j)
                    used = optE[j] == E;
                if (!used)
                    continue;
                int64_t L = (int64_t)(E - 1) * tau;
                int64_t nq = orc_ccm_rows(T, E, tau, Tp);
                int k = E + 1;
                int64_t *idx = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nq * k));
                double *w = (double *)malloc(sizeof(double) * (size_t)(nq * k));
                double *d2 = (double *)malloc(sizeof(double) * (size_t)k);
                int rc = (idx && w && d2 && nq > 0) ? ORC_OK : ORC_ERR_NOMEM;
                for (int64_t q = 0; rc == ORC_OK && q < nq; ++q) {
                    if (knn_query_masked(x, L + q, L, T - 1 - Tp, mask, E, tau, excl, k, idx + q * k, d2) < k)
                        rc = ORC_ERR_INVALID;
                    else
                        simplex_weights(d2, k, w + q * k);
                }
                if (rc == ORC_OK) {
                    for (int64_t j = 0; j < N; ++j)
                        if (optE[j] == E)
                            rho[(u * n_rows + r) * N + j] = orc_lookup_rho(Y + j * ldY, T, E, tau, Tp, idx, w);
                } else {
#ifdef _OPENMP
#pragma omp atomic write
#endif
                    rc_all = rc;
                }
                free(idx);
                free(w);
                free(d2);
            }
        }
    (void)nthreads;
    return rc_all;
}

/* rho for a list of (library, target) pairs; each pair builds its own table. */
int orc_ccm_rho_pairs(const double *Y, int64_t N, int64_t T, int64_t ldY, const int32_t *optE,
                      const int64_t *li, const int64_t *lj, int64_t n_pairs, int tau, int Tp, int excl,
                      double *rho, int nthreads)
{
    if (N < 1 || T < 2 || ldY < T || tau < 1 || Tp < 0)
        return ORC_ERR_INVALID;
    int rc_all = ORC_OK;
#ifdef _OPENMP
    if (nthreads < 1)
        nthreads = 1;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
#endif
    for (int64_t p = 0; p < n_pairs; ++p) {
        int64_t i = li[p], j = lj[p];
        int E = optE[j];
        int64_t nq = orc_ccm_rows(T, E, tau, Tp);
        int k = E + 1;
        int64_t *idx = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nq * k));
        double *w = (double *)malloc(sizeof(double) * (size_t)(nq * k));
        int rc = (idx && w) ? orc_ccm_table(Y + i * ldY, T, E, tau, Tp, excl, idx, w) : ORC_ERR_NOMEM;
        if (rc != ORC_OK) {
#ifdef _OPENMP
#pragma omp atomic write
#endif
            rc_all = rc;
            rho[p] = NAN;
        } else {
            rho[p] = orc_lookup_rho(Y + j * ldY, T, E, tau, Tp, idx, w);
        }
        free(idx);
        free(w);
    }
    (void)nthreads;
    return rc_all;
}

/*
 * Phase-2 tables (as orc_ccm_table) of library rows rows[0..n_rows) of Y at
 * one E, one library per thread: idx[r][nq][E+1] and, if w is not NULL,
 * w[r][nq][E+1] (nq = orc_ccm_rows).  A convenience for checks that need
 * many libraries' frozen neighbour indices; the per-library arithmetic is
 * orc_ccm_table's.
 */
int orc_ccm_tables(const double *Y, int64_t ldY, int64_t T, const int64_t *rows, int64_t n_rows, int E, int tau,
                   int Tp, int excl, int64_t *idx, double *w, int nthreads)
{
    const int64_t nq = orc_ccm_rows(T, E, tau, Tp);
    const int k = E + 1;
    if (nq < 1)
        return ORC_ERR_INVALID;
    int rc_all = ORC_OK;
#ifdef _OPENMP
    if (nthreads < 1)
        nthreads = 1;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
#endif
    for (int64_t r = 0; r < n_rows; ++r) {
        double *wr = w ? w + r * nq * k : (double *)malloc(sizeof(double) * (size_t)(nq * k));
        int rc = wr ? orc_ccm_table(Y + rows[r] * ldY, T, E, tau, Tp, excl, idx + r * nq * k, wr) : ORC_ERR_NOMEM;
        if (!w)
            free(wr);
        if (rc != ORC_OK) {
#ifdef _OPENMP
#pragma omp atomic write
#endif
            rc_all = rc;
        }
    }
    (void)nthreads;
    return rc_all;
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
