/*
 * FP64 CPU oracle for atlas-based fiber bundle segmentation (arXiv:1912.11494).
 *
 * TEST INFRASTRUCTURE ONLY. Tests, the package smoke check and the benchmark's CPU-baseline leg
 * may call it; the product path never does. It shares no code with the CUDA path: every input
 * is a plain array promoted from float32 to double, and every result is computed here in double.
 *
 * What it computes (paper Section 2.3):
 *   Eq. 1   d_E(a_i, b_i) = || a_i - b_i ||_2
 *   Eq. 2   d_ME(a, b) = min( max_i d_E(a_i, b_i), max_i d_E(a_i, b_rev(i)) )
 *           with rev(i) = 20 - i for 0-based 21-point fibers (the reversal reading of the
 *           garbled flip index; test1 of Section 2.3 uses the centre point alone for both
 *           orientations, which only works if the centre maps to itself).
 *   Labelling (Algorithm 1, closest-bundle classification of Section 2.4): a centroid c passes
 *           when d_ME(f, c) <= theta of its bundle; the fiber takes the bundle of the passing
 *           centroid with the smallest d_ME, visiting bundles in increasing index and the
 *           centroids of a bundle in their given order, and replacing the best only on a strict
 *           decrease; no passing centroid gives label -1 and distance +inf.
 *   The length term TN (Eq. 3) is not part of this path: labels use the raw d_ME.
 *
 * Two labelling modes give identical results by construction:
 *   brute   - all 42 point distances of every pair, then the rule above (the plain definition);
 *   cascade - the paper's progressive discarding of fibers (Section 2.3 and Algorithm 1): test1 centre point, test2 end points, test3 four intermediate
 *             points, test4 all points, each orientation stopping at its first point distance
 *             above the threshold (Section 2.4, early evaluation of the discarding criterion).
 *
 * The gradient mode (not in the paper) differentiates C = sum over labelled fibers of
 * d_ME(T f, c_sigma(f)) with T y = M x + t, through the argmax point: with r = T(a_i*) - c_pi(i*)
 * and u = r / ||r||, dC/dM_rc += u_r a_i*,c, dC/dt += u, dC/dc_sigma,pi(i*) -= u. Conventions:
 * argmax = lowest index attaining the max; orientation ties go to the direct orientation;
 * ||r|| = 0 contributes a zero subgradient; unlabelled fibers contribute nothing.
 *
 * A fiber with a non-finite coordinate gets label -1 and distance NaN.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define NPTS 21
#define NC (NPTS * 3)
#define CENTRE 10

/* test3 point set: four intermediate points (the paper does not say which; any set is exact). */
static const int TEST3[4] = {5, 15, 3, 17};

static void set_threads(int nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

int oracle_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Eq. 1 in double. */
static double d_E(const double *p, const double *q) {
    double dx = p[0] - q[0], dy = p[1] - q[1], dz = p[2] - q[2];
    return sqrt(dx * dx + dy * dy + dz * dz);
}

static int rev(int i) { return NPTS - 1 - i; }

static void promote(const float *src, double *dst, int64_t count) {
    for (int64_t k = 0; k < count; ++k) dst[k] = (double)src[k];
}

static int all_finite(const double *a) {
    for (int k = 0; k < NC; ++k)
        if (!isfinite(a[k])) return 0;
    return 1;
}

/* Both orientation maxima of Eq. 2: dd = max_i d_E(a_i,b_i), dr = max_i d_E(a_i,b_{20-i}). */
static void dme_both(const double *a, const double *b, double *dd, double *dr) {
    double md = 0.0, mr = 0.0;
    for (int i = 0; i < NPTS; ++i) {
        double e = d_E(a + 3 * i, b + 3 * i);
        double f = d_E(a + 3 * i, b + 3 * rev(i));
        if (e > md) md = e;
        if (f > mr) mr = f;
    }
    *dd = md;
    *dr = mr;
}

/* Lowest point index attaining the max of d_E in orientation o (0 direct, 1 reversed). */
static int argmax_point(const double *a, const double *b, int o) {
    int best = 0;
    double m = -1.0;
    for (int i = 0; i < NPTS; ++i) {
        double e = d_E(a + 3 * i, b + 3 * (o ? rev(i) : i));
        if (e > m) {
            m = e;
            best = i;
        }
    }
    return best;
}

/* Second largest point distance in orientation o, for structure margins. */
static double second_max(const double *a, const double *b, int o, int imax) {
    double m = 0.0;
    for (int i = 0; i < NPTS; ++i) {
        if (i == imax) continue;
        double e = d_E(a + 3 * i, b + 3 * (o ? rev(i) : i));
        if (e > m) m = e;
    }
    return m;
}

/* Visiting order of Algorithm 1: bundles in increasing index, centroids of a bundle in their
 * given order. Returns a malloc'd array of M centroid indices, or NULL on a bad bundle id. */
static int64_t *bundle_order(const int32_t *bundle_of, int64_t M, int32_t B) {
    int64_t *cnt = calloc((size_t)B + 1, sizeof(int64_t));
    int64_t *ord = malloc((size_t)(M > 0 ? M : 1) * sizeof(int64_t));
    if (!cnt || !ord) {
        free(cnt);
        free(ord);
        return NULL;
    }
    for (int64_t c = 0; c < M; ++c) {
        if (bundle_of[c] < 0 || bundle_of[c] >= B) {
            free(cnt);
            free(ord);
            return NULL;
        }
        cnt[bundle_of[c] + 1]++;
    }
    for (int32_t j = 0; j < B; ++j) cnt[j + 1] += cnt[j];
    for (int64_t c = 0; c < M; ++c) ord[cnt[bundle_of[c]]++] = c;
    free(cnt);
    return ord;
}

/* d_ME and both orientation maxima for every (fiber, centroid) pair: out arrays [n][M]. */
int oracle_dme_matrix(const float *fib, int64_t n, const float *cen, int64_t M, double *dme,
                      double *dd, double *dr, int nthreads) {
    double *C = malloc((size_t)(M > 0 ? M : 1) * NC * sizeof(double));
    if (!C) return 1;
    promote(cen, C, M * NC);
    set_threads(nthreads);
#pragma omp parallel for schedule(static)
    for (int64_t f = 0; f < n; ++f) {
        double a[NC];
        promote(fib + f * NC, a, NC);
        for (int64_t c = 0; c < M; ++c) {
            double x, y;
            dme_both(a, C + c * NC, &x, &y);
            if (dd) dd[f * M + c] = x;
            if (dr) dr[f * M + c] = y;
            if (dme) dme[f * M + c] = x < y ? x : y;
        }
    }
    free(C);
    return 0;
}

typedef struct {
    int32_t label;
    int64_t cidx;
    int orient;
    double dist;
} result_t;

static void result_none(result_t *r) {
    r->label = -1;
    r->cidx = -1;
    r->orient = 0;
    r->dist = INFINITY;
}

/* Plain definition: all point distances of every pair, then the closest passing centroid. */
static void label_brute_one(const double *a, const double *C, const int32_t *bundle_of,
                            const double *thr, const int64_t *ord, int64_t M, result_t *r) {
    result_none(r);
    for (int64_t k = 0; k < M; ++k) {
        int64_t c = ord[k];
        double dd, dr;
        dme_both(a, C + c * NC, &dd, &dr);
        double d = dd <= dr ? dd : dr;
        if (d <= thr[bundle_of[c]] && d < r->dist) {
            r->dist = d;
            r->label = bundle_of[c];
            r->cidx = c;
            r->orient = dd <= dr ? 0 : 1;
        }
    }
}

/* Progressive discarding of Section 2.3 (test1..test4) with per-point early exit (Section
 * 2.4). cnt[s] counts point distances evaluated in test s+1, cnt[4+s] the pairs reaching it. */
static void label_cascade_one(const double *a, const double *C, const int32_t *bundle_of,
                              const double *thr, const int64_t *ord, int64_t M, result_t *r,
                              int64_t *cnt) {
    result_none(r);
    for (int64_t k = 0; k < M; ++k) {
        int64_t c = ord[k];
        const double *b = C + c * NC;
        double th = thr[bundle_of[c]];
        /* test1: the centre point serves both orientations */
        cnt[4]++;
        cnt[0]++;
        double e = d_E(a + 3 * CENTRE, b + 3 * CENTRE);
        if (e > th) continue;
        double md = e, mr = e;
        int alive_d = 1, alive_r = 1;
        /* test2: end points, each orientation on its own */
        cnt[5]++;
        const int ends[2] = {0, NPTS - 1};
        for (int q = 0; q < 2 && alive_d; ++q) {
            cnt[1]++;
            double x = d_E(a + 3 * ends[q], b + 3 * ends[q]);
            if (x > md) md = x;
            if (x > th) alive_d = 0;
        }
        for (int q = 0; q < 2 && alive_r; ++q) {
            cnt[1]++;
            double x = d_E(a + 3 * ends[q], b + 3 * rev(ends[q]));
            if (x > mr) mr = x;
            if (x > th) alive_r = 0;
        }
        if (!alive_d && !alive_r) continue;
        /* test3: four intermediate points */
        cnt[6]++;
        for (int q = 0; q < 4 && alive_d; ++q) {
            cnt[2]++;
            double x = d_E(a + 3 * TEST3[q], b + 3 * TEST3[q]);
            if (x > md) md = x;
            if (x > th) alive_d = 0;
        }
        for (int q = 0; q < 4 && alive_r; ++q) {
            cnt[2]++;
            double x = d_E(a + 3 * TEST3[q], b + 3 * rev(TEST3[q]));
            if (x > mr) mr = x;
            if (x > th) alive_r = 0;
        }
        if (!alive_d && !alive_r) continue;
        /* test4: every remaining point */
        cnt[7]++;
        for (int i = 0; i < NPTS && alive_d; ++i) {
            if (i == CENTRE || i == 0 || i == NPTS - 1 || i == 5 || i == 15 || i == 3 || i == 17)
                continue;
            cnt[3]++;
            double x = d_E(a + 3 * i, b + 3 * i);
            if (x > md) md = x;
            if (x > th) alive_d = 0;
        }
        for (int i = 0; i < NPTS && alive_r; ++i) {
            if (i == CENTRE || i == 0 || i == NPTS - 1 || i == 5 || i == 15 || i == 3 || i == 17)
                continue;
            cnt[3]++;
            double x = d_E(a + 3 * i, b + 3 * rev(i));
            if (x > mr) mr = x;
            if (x > th) alive_r = 0;
        }
        if (!alive_d && !alive_r) continue;
        double ed;
        int o;
        if (alive_d && alive_r) {
            ed = md <= mr ? md : mr;
            o = md <= mr ? 0 : 1;
        } else if (alive_d) {
            ed = md;
            o = 0;
        } else {
            ed = mr;
            o = 1;
        }
        if (ed < r->dist) { /* Algorithm 1: strict decrease only */
            r->dist = ed;
            r->label = bundle_of[c];
            r->cidx = c;
            r->orient = o;
        }
    }
}

static int label_impl(int cascade, const double *fibd_or_null, const float *fib, int64_t n,
                      const float *cen, const int32_t *bundle_of, int64_t M, const float *thr,
                      int32_t B, int32_t *labels, double *dist, int32_t *cidx, uint8_t *orient,
                      int32_t *argmax, int64_t *counts, int nthreads) {
    int64_t *ord = bundle_order(bundle_of, M, B);
    double *C = malloc((size_t)(M > 0 ? M : 1) * NC * sizeof(double));
    double *T = malloc((size_t)(B > 0 ? B : 1) * sizeof(double));
    if (!ord || !C || !T) {
        free(ord);
        free(C);
        free(T);
        return 1;
    }
    promote(cen, C, M * NC);
    for (int32_t j = 0; j < B; ++j) T[j] = (double)thr[j];
    int64_t tot[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    set_threads(nthreads);
#pragma omp parallel
    {
        int64_t loc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
#pragma omp for schedule(dynamic, 64)
        for (int64_t f = 0; f < n; ++f) {
            double a[NC];
            if (fibd_or_null)
                memcpy(a, fibd_or_null + f * NC, sizeof(a));
            else
                promote(fib + f * NC, a, NC);
            result_t r;
            if (!all_finite(a)) {
                result_none(&r);
                r.dist = NAN;
            } else if (cascade) {
                label_cascade_one(a, C, bundle_of, T, ord, M, &r, loc);
            } else {
                label_brute_one(a, C, bundle_of, T, ord, M, &r);
            }
            if (labels) labels[f] = r.label;
            if (dist) dist[f] = r.dist;
            if (cidx) cidx[f] = (int32_t)r.cidx;
            if (orient) orient[f] = (uint8_t)r.orient;
            if (argmax) argmax[f] = r.cidx >= 0 ? argmax_point(a, C + r.cidx * NC, r.orient) : -1;
        }
#pragma omp critical
        for (int s = 0; s < 8; ++s) tot[s] += loc[s];
    }
    if (counts)
        for (int s = 0; s < 8; ++s) counts[s] = tot[s];
    free(ord);
    free(C);
    free(T);
    return 0;
}

int oracle_label_brute(const float *fib, int64_t n, const float *cen, const int32_t *bundle_of,
                       int64_t M, const float *thr, int32_t B, int32_t *labels, double *dist,
                       int32_t *cidx, uint8_t *orient, int32_t *argmax, int nthreads) {
    return label_impl(0, NULL, fib, n, cen, bundle_of, M, thr, B, labels, dist, cidx, orient,
                      argmax, NULL, nthreads);
}

int oracle_label_cascade(const float *fib, int64_t n, const float *cen,
                         const int32_t *bundle_of, int64_t M, const float *thr, int32_t B,
                         int32_t *labels, double *dist, int32_t *cidx, uint8_t *orient,
                         int32_t *argmax, int64_t *counts, int nthreads) {
    return label_impl(1, NULL, fib, n, cen, bundle_of, M, thr, B, labels, dist, cidx, orient,
                      argmax, counts, nthreads);
}

/* Decidability of each fiber's label at tolerance tol (mm), given the oracle's own result.
 * flag[f] = 1 (near-tie) when (i) a centroid within tol of the best distance (any centroid if
 * unlabelled) lies within tol of its threshold, or (ii) a centroid of another bundle passes its
 * threshold + tol and lies within tol of the best distance. */
int oracle_near_tie(const float *fib, int64_t n, const float *cen, const int32_t *bundle_of,
                    int64_t M, const float *thr, int32_t B, const int32_t *labels,
                    const double *dist, double tol, uint8_t *flag, int nthreads) {
    double *C = malloc((size_t)(M > 0 ? M : 1) * NC * sizeof(double));
    if (!C) return 1;
    promote(cen, C, M * NC);
    (void)B;
    set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t f = 0; f < n; ++f) {
        double a[NC];
        promote(fib + f * NC, a, NC);
        uint8_t fl = 0;
        if (all_finite(a)) {
            double D = dist[f];
            for (int64_t c = 0; c < M && !fl; ++c) {
                double dd, dr;
                dme_both(a, C + c * NC, &dd, &dr);
                double d = dd <= dr ? dd : dr;
                double th = (double)thr[bundle_of[c]];
                if ((labels[f] < 0 || d <= D + tol) && fabs(d - th) <= tol) fl = 1;
                if (bundle_of[c] != labels[f] && d <= th + tol && fabs(d - D) <= tol) fl = 1;
            }
        }
        flag[f] = fl;
    }
    free(C);
    return 0;
}

/* The same flags as oracle_near_tie, with centroids that cannot matter skipped. Both conditions
 * need d(f,c) <= theta_b(c) + tol, and each orientation's running maximum of point distances is
 * a lower bound of its full maximum, so a centroid is skipped as soon as both running maxima
 * exceed theta + tol (centre point first, then the end points, then the rest, as in the
 * progressive discarding of Section 2.3). Every centroid that is not skipped gets the full
 * d_ME of Eq. 2, and the flag is decided exactly as in oracle_near_tie. */
int oracle_near_tie_pruned(const float *fib, int64_t n, const float *cen,
                           const int32_t *bundle_of, int64_t M, const float *thr, int32_t B,
                           const int32_t *labels, const double *dist, double tol,
                           uint8_t *flag, int nthreads) {
    double *C = malloc((size_t)(M > 0 ? M : 1) * NC * sizeof(double));
    if (!C) return 1;
    promote(cen, C, M * NC);
    (void)B;
    /* point visiting order: centre, ends, the test3 points, then the rest */
    int order[NPTS];
    int k = 0;
    order[k++] = CENTRE;
    order[k++] = 0;
    order[k++] = NPTS - 1;
    for (int q = 0; q < 4; ++q) order[k++] = TEST3[q];
    for (int i = 1; i < NPTS - 1; ++i)
        if (i != CENTRE && i != 5 && i != 15 && i != 3 && i != 17) order[k++] = i;
    set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t f = 0; f < n; ++f) {
        double a[NC];
        promote(fib + f * NC, a, NC);
        uint8_t fl = 0;
        if (all_finite(a)) {
            double D = dist[f];
            for (int64_t c = 0; c < M && !fl; ++c) {
                const double *b = C + c * NC;
                double th = (double)thr[bundle_of[c]];
                double lim = th + tol;
                double md = 0.0, mr = 0.0;
                for (int q = 0; q < NPTS && (md <= lim || mr <= lim); ++q) {
                    int i = order[q];
                    double e = d_E(a + 3 * i, b + 3 * i);
                    double g = d_E(a + 3 * i, b + 3 * rev(i));
                    if (e > md) md = e;
                    if (g > mr) mr = g;
                }
                if (md > lim && mr > lim) continue; /* d > theta + tol: neither condition */
                double d = md <= mr ? md : mr;
                if ((labels[f] < 0 || d <= D + tol) && fabs(d - th) <= tol) fl = 1;
                if (bundle_of[c] != labels[f] && d <= th + tol && fabs(d - D) <= tol) fl = 1;
            }
        }
        flag[f] = fl;
    }
    free(C);
    return 0;
}

/* d_ME and both orientation maxima of fiber f against centroid idx[f] (Eq. 1, Eq. 2): one pair
 * per fiber; idx[f] < 0 gives NaN. */
int oracle_dme_pairs(const float *fib, int64_t n, const float *cen, int64_t M,
                     const int32_t *idx, double *dme, double *dd, double *dr, int nthreads) {
    set_threads(nthreads);
#pragma omp parallel for schedule(static)
    for (int64_t f = 0; f < n; ++f) {
        double x = NAN, y = NAN;
        if (idx[f] >= 0 && idx[f] < M) {
            double a[NC], b[NC];
            promote(fib + f * NC, a, NC);
            promote(cen + (int64_t)idx[f] * NC, b, NC);
            dme_both(a, b, &x, &y);
        }
        if (dd) dd[f] = x;
        if (dr) dr[f] = y;
        if (dme) dme[f] = x < y ? x : y;
    }
    return 0;
}

/* ---- paper-faithful classification (Section 2.3 Eq. 3, Section 2.4) ------------------------ */

/* Arc length of a 21-point polyline: the sum of its 20 segment lengths (Eq. 1 between
 * consecutive points). Read as the fiber length l_S / centroid length l_C of Eq. 3. */
static double poly_length(const double *a) {
    double l = 0.0;
    for (int i = 0; i + 1 < NPTS; ++i) l += d_E(a + 3 * i, a + 3 * (i + 1));
    return l;
}

/* Eq. 3: TN = (|l_S - l_C| / max(l_S, l_C) + 1)^2 - 1; two zero lengths give 0. */
static double tn_term(double ls, double lc) {
    double m = ls > lc ? ls : lc;
    if (!(m > 0.0)) return 0.0;
    double r = fabs(ls - lc) / m;
    return (r + 1.0) * (r + 1.0) - 1.0;
}

/* Classification distance of one pair, or +inf when the pair is discarded.
 * cls 1 (Eq. 2 + TN, lazy): d = min(dd, dr) of Eq. 2; a pair with d > theta is discarded
 *   before TN is computed (Section 2.4, the new algorithm's last optimization); else
 *   D = d + TN, and the pair passes when D <= theta.
 * cls 2 (the paper's new algorithm, Section 2.4): test1 on the centre point; test2 computes both
 *   orientations' end-point distances and infers the direction as the orientation with the
 *   smaller partial maximum (ties: direct); test3 and test4 then run in that orientation only,
 *   each distance checked against theta at once; D = that orientation's maximum + TN (lazy). */
static double cls_distance(int cls, const double *a, const double *b, double th, double ls,
                           double lc, int *orient) {
    if (cls == 1) {
        double dd, dr;
        dme_both(a, b, &dd, &dr);
        double d = dd <= dr ? dd : dr;
        *orient = dd <= dr ? 0 : 1;
        if (d > th) return INFINITY;
        return d + tn_term(ls, lc);
    }
    double m = d_E(a + 3 * CENTRE, b + 3 * CENTRE); /* test1 */
    if (m > th) return INFINITY;
    double ed = m, er = m; /* test2, both orientations */
    double x;
    x = d_E(a, b);                                  if (x > ed) ed = x;
    x = d_E(a + 3 * (NPTS - 1), b + 3 * (NPTS - 1)); if (x > ed) ed = x;
    x = d_E(a, b + 3 * (NPTS - 1));                 if (x > er) er = x;
    x = d_E(a + 3 * (NPTS - 1), b);                 if (x > er) er = x;
    if (ed > th && er > th) return INFINITY;
    int o = ed <= er ? 0 : 1; /* direction inference */
    *orient = o;
    m = o ? er : ed;
    for (int q = 0; q < 4; ++q) { /* test3 */
        x = d_E(a + 3 * TEST3[q], b + 3 * (o ? rev(TEST3[q]) : TEST3[q]));
        if (x > th) return INFINITY;
        if (x > m) m = x;
    }
    for (int i = 1; i < NPTS - 1; ++i) { /* test4 */
        if (i == CENTRE || i == 5 || i == 15 || i == 3 || i == 17) continue;
        x = d_E(a + 3 * i, b + 3 * (o ? rev(i) : i));
        if (x > th) return INFINITY;
        if (x > m) m = x;
    }
    if (m > th) return INFINITY;
    return m + tn_term(ls, lc); /* lazy TN: only for a pair that got this far */
}

/* Labelling with classification cls (1 or 2, see cls_distance): a pair passes when D <= theta;
 * the fiber takes the bundle of the passing centroid with the smallest D, visiting bundles in
 * increasing index and replacing the best only on a strict decrease (Algorithm 1). dist = D. */
int oracle_label_cls(const float *fib, int64_t n, const float *cen, const int32_t *bundle_of,
                     int64_t M, const float *thr, int32_t B, int cls, int32_t *labels,
                     double *dist, int32_t *cidx, uint8_t *orient, int nthreads) {
    if (cls != 1 && cls != 2) return 2;
    int64_t *ord = bundle_order(bundle_of, M, B);
    double *C = malloc((size_t)(M > 0 ? M : 1) * NC * sizeof(double));
    double *L = malloc((size_t)(M > 0 ? M : 1) * sizeof(double));
    if (!ord || !C || !L) {
        free(ord);
        free(C);
        free(L);
        return 1;
    }
    promote(cen, C, M * NC);
    for (int64_t c = 0; c < M; ++c) L[c] = poly_length(C + c * NC);
    set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t f = 0; f < n; ++f) {
        double a[NC];
        promote(fib + f * NC, a, NC);
        result_t r;
        result_none(&r);
        if (!all_finite(a)) {
            r.dist = NAN;
        } else {
            double ls = poly_length(a);
            for (int64_t k = 0; k < M; ++k) {
                int64_t c = ord[k];
                double th = (double)thr[bundle_of[c]];
                int o = 0;
                double D = cls_distance(cls, a, C + c * NC, th, ls, L[c], &o);
                if (D <= th && D < r.dist) {
                    r.dist = D;
                    r.label = bundle_of[c];
                    r.cidx = c;
                    r.orient = o;
                }
            }
        }
        if (labels) labels[f] = r.label;
        if (dist) dist[f] = r.dist;
        if (cidx) cidx[f] = (int32_t)r.cidx;
        if (orient) orient[f] = (uint8_t)r.orient;
    }
    free(ord);
    free(C);
    free(L);
    return 0;
}

/* Decidability of oracle_label_cls's result at tolerance tol (mm), on the classification
 * distance D. A pair's candidate values: D itself (cls 1; D = min(dd, dr) + TN); for cls 2 the
 * value D_o = max_o + TN of every orientation o whose test2 maximum is within tol of the smaller
 * one (an FP32 implementation may infer either). flag[f] = 1 when (i) a candidate within tol of
 * the best D (any, if unlabelled) lies within tol of its threshold, (ii) a candidate of another
 * bundle passes its threshold + tol within tol of the best D, or (iii) (cls 2) a centroid with
 * two possible orientations has a candidate that passes its threshold + tol within tol of the
 * best D or below it. Candidates whose centre-point distance exceeds theta + tol are skipped. */
int oracle_near_tie_cls(const float *fib, int64_t n, const float *cen, const int32_t *bundle_of,
                        int64_t M, const float *thr, int32_t B, int cls, const int32_t *labels,
                        const double *dist, double tol, uint8_t *flag, int nthreads) {
    (void)B;
    double *C = malloc((size_t)(M > 0 ? M : 1) * NC * sizeof(double));
    double *L = malloc((size_t)(M > 0 ? M : 1) * sizeof(double));
    if (!C || !L) {
        free(C);
        free(L);
        return 1;
    }
    promote(cen, C, M * NC);
    for (int64_t c = 0; c < M; ++c) L[c] = poly_length(C + c * NC);
    set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t f = 0; f < n; ++f) {
        double a[NC];
        promote(fib + f * NC, a, NC);
        uint8_t fl = 0;
        if (all_finite(a)) {
            const double Db = dist[f], ls = poly_length(a);
            const int unl = labels[f] < 0;
            for (int64_t c = 0; c < M && !fl; ++c) {
                const double *b = C + c * NC;
                const double th = (double)thr[bundle_of[c]];
                if (d_E(a + 3 * CENTRE, b + 3 * CENTRE) > th + tol) continue;
                double dd, dr;
                dme_both(a, b, &dd, &dr);
                const double tn = tn_term(ls, L[c]);
                double cand[2];
                int nc = 0;
                if (cls == 1) {
                    cand[nc++] = (dd <= dr ? dd : dr) + tn;
                } else {
                    double m = d_E(a + 3 * CENTRE, b + 3 * CENTRE), ed = m, er = m, x;
                    x = d_E(a, b);                                  if (x > ed) ed = x;
                    x = d_E(a + 3 * (NPTS - 1), b + 3 * (NPTS - 1)); if (x > ed) ed = x;
                    x = d_E(a, b + 3 * (NPTS - 1));                 if (x > er) er = x;
                    x = d_E(a + 3 * (NPTS - 1), b);                 if (x > er) er = x;
                    const double lo = ed <= er ? ed : er;
                    if (ed <= lo + tol) cand[nc++] = dd + tn;
                    if (er <= lo + tol) cand[nc++] = dr + tn;
                }
                for (int k = 0; k < nc && !fl; ++k) {
                    const double D = cand[k];
                    if (D > th + tol) continue;
                    if ((unl || D <= Db + tol) && fabs(D - th) <= tol) fl = 1;
                    if (bundle_of[c] != labels[f] && fabs(D - Db) <= tol) fl = 1;
                    if (nc == 2 && (unl || D <= Db + tol)) fl = 1;
                }
            }
        }
        flag[f] = fl;
    }
    free(C);
    free(L);
    return 0;
}

/* Fiber polyline lengths (for tests of Eq. 3's l_S). */
int oracle_lengths(const float *fib, int64_t n, double *len) {
    for (int64_t f = 0; f < n; ++f) {
        double a[NC];
        promote(fib + f * NC, a, NC);
        len[f] = poly_length(a);
    }
    return 0;
}

/* ---- resampling of raw streamlines (Section 2.3) ----------------------------------------- */

/* Section 2.3 works on subject fibers of 21 equidistant points; read here as equidistant
 * in arc length along the streamline's polyline: with cumulative lengths c_0 = 0 <= c_1 <= ...
 * <= c_(m-1) = L over its m points, output point k (0 <= k <= 20) is the point at arc length
 * s_k = k L / 20, linearly interpolated inside the first segment (j, j+1) with c_j < s_k <=
 * c_(j+1) (zero-length segments never hold one); point 0 is the first point and point 20 the
 * last. A streamline with a single point, or of zero length, gives 21 copies of its first
 * point; one with no points gives NaN. points [P][3], offsets [n+1] (fiber f has points
 * offsets[f] .. offsets[f+1]-1), out [n][21][3] in double. */
int oracle_resample(const float *points, const int64_t *offsets, int64_t n, double *out,
                    int nthreads) {
    set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t f = 0; f < n; ++f) {
        const int64_t p0 = offsets[f], m = offsets[f + 1] - offsets[f];
        double *o = out + f * NC;
        if (m <= 0) {
            for (int k = 0; k < NC; ++k) o[k] = NAN;
            continue;
        }
        double *q = malloc((size_t)m * 3 * sizeof(double));
        double *c = malloc((size_t)m * sizeof(double));
        promote(points + 3 * p0, q, 3 * m);
        c[0] = 0.0;
        for (int64_t j = 0; j + 1 < m; ++j) c[j + 1] = c[j] + d_E(q + 3 * j, q + 3 * (j + 1));
        const double L = c[m - 1];
        for (int r = 0; r < 3; ++r) {
            o[r] = q[r];
            o[3 * (NPTS - 1) + r] = q[3 * (m - 1) + r];
        }
        int64_t j = 0;
        for (int k = 1; k < NPTS - 1; ++k) {
            if (!(L > 0.0)) {
                for (int r = 0; r < 3; ++r) o[3 * k + r] = q[r];
                continue;
            }
            const double sk = k * L / (NPTS - 1);
            while (j + 1 < m - 1 && !(c[j] < sk && sk <= c[j + 1])) ++j;
            const double w = (sk - c[j]) / (c[j + 1] - c[j]);
            for (int r = 0; r < 3; ++r)
                o[3 * k + r] = q[3 * j + r] + w * (q[3 * (j + 1) + r] - q[3 * j + r]);
        }
        free(q);
        free(c);
    }
    return 0;
}

/* ---- multi-label output (Section 2.4, on classifying fibers) ----------------------------- */

/* Every bundle a fiber passes: bit b of fiber f's row (words uint32 words) is set when some
 * centroid of bundle b passes its threshold under classification cls (0 Eq. 2: d_ME <= theta;
 * 1 and 2: D <= theta as in oracle_label_cls), which is how the paper's original algorithm could
 * assign a fiber to several bundles. amb (optional, same shape) marks the bundles whose bit is
 * not decidable at tolerance tol: no centroid of the bundle is below theta - tol but one is
 * within tol of theta. Non-finite fibers get no bit. */
int oracle_label_multi(const float *fib, int64_t n, const float *cen, const int32_t *bundle_of,
                       int64_t M, const float *thr, int32_t B, int cls, int64_t words,
                       uint32_t *bits, uint32_t *amb, double tol, int nthreads) {
    if (cls < 0 || cls > 2 || words * 32 < B) return 2;
    double *C = malloc((size_t)(M > 0 ? M : 1) * NC * sizeof(double));
    double *L = malloc((size_t)(M > 0 ? M : 1) * sizeof(double));
    if (!C || !L) {
        free(C);
        free(L);
        return 1;
    }
    promote(cen, C, M * NC);
    for (int64_t c = 0; c < M; ++c) L[c] = poly_length(C + c * NC);
    set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t f = 0; f < n; ++f) {
        uint32_t *row = bits + f * words, *arow = amb ? amb + f * words : NULL;
        for (int64_t w = 0; w < words; ++w) {
            row[w] = 0;
            if (arow) arow[w] = 0;
        }
        double a[NC];
        promote(fib + f * NC, a, NC);
        if (!all_finite(a)) continue;
        const double ls = poly_length(a);
        /* per bundle: the smallest classification distance minus theta */
        double *best = malloc((size_t)B * sizeof(double));
        for (int32_t b = 0; b < B; ++b) best[b] = INFINITY;
        for (int64_t c = 0; c < M; ++c) {
            const double th = (double)thr[bundle_of[c]];
            double D;
            if (cls == 0) {
                double dd, dr;
                dme_both(a, C + c * NC, &dd, &dr);
                D = dd <= dr ? dd : dr;
            } else {
                int o = 0;
                /* with TN the gate is D itself; a large threshold keeps cls_distance from
                 * discarding pairs just above theta, which the ambiguity test needs */
                D = cls_distance(cls, a, C + c * NC, th + tol, ls, L[c], &o);
            }
            if (D - th < best[bundle_of[c]]) best[bundle_of[c]] = D - th;
        }
        for (int32_t b = 0; b < B; ++b) {
            if (best[b] <= 0.0) row[b >> 5] |= 1u << (b & 31);
            if (arow && fabs(best[b]) <= tol) arow[b >> 5] |= 1u << (b & 31);
        }
        free(best);
    }
    free(C);
    free(L);
    return 0;
}

/* y = M x + t for every point, in double. aff = M row-major (9) then t (3). */
static void apply_affine(const double *aff, const double *x, double *y) {
    for (int p = 0; p < NPTS; ++p) {
        const double *q = x + 3 * p;
        for (int r = 0; r < 3; ++r)
            y[3 * p + r] = aff[3 * r] * q[0] + aff[3 * r + 1] * q[1] + aff[3 * r + 2] * q[2] +
                           aff[9 + r];
    }
}

/* Cost, structure and gradient of C(T) = sum_f d_ME(T f, c_sigma(f)) over labelled fibers.
 * The structure (sigma, orientation, argmax) comes from the oracle's own brute labelling of the
 * transformed fibers unless frozen arrays are given (cidx_in/orient_in/argmax_in non-NULL), in
 * which case every fiber with cidx_in >= 0 contributes through that structure.
 * mask (optional) selects the fibers that count. gap[f] (optional) returns the smaller of the
 * argmax margin (max minus second max point distance) and the orientation margin |dd - dr|.
 * grad_cen is [M][21][3] in the caller's centroid order. */
int oracle_grad(const float *fib, int64_t n, const double *aff, const float *cen,
                const int32_t *bundle_of, int64_t M, const float *thr, int32_t B,
                const uint8_t *mask, const int32_t *cidx_in, const uint8_t *orient_in,
                const int32_t *argmax_in, double *cost, double *grad_aff, double *grad_cen,
                int32_t *cidx_out, uint8_t *orient_out, int32_t *argmax_out, double *gap,
                int nthreads) {
    int64_t *ord = bundle_order(bundle_of, M, B);
    double *C = malloc((size_t)(M > 0 ? M : 1) * NC * sizeof(double));
    double *T = malloc((size_t)(B > 0 ? B : 1) * sizeof(double));
    if (!ord || !C || !T) {
        free(ord);
        free(C);
        free(T);
        return 1;
    }
    promote(cen, C, M * NC);
    for (int32_t j = 0; j < B; ++j) T[j] = (double)thr[j];
    set_threads(nthreads);
    int nt = oracle_max_threads();
    double *pg = calloc((size_t)nt * 13, sizeof(double));
    double *pc = grad_cen ? calloc((size_t)nt * (size_t)M * NC, sizeof(double)) : NULL;
    if (!pg || (grad_cen && !pc)) {
        free(ord);
        free(C);
        free(T);
        free(pg);
        free(pc);
        return 1;
    }
#pragma omp parallel
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double *g = pg + 13 * tid;
        double *gc = pc ? pc + (size_t)tid * (size_t)M * NC : NULL;
#pragma omp for schedule(static)
        for (int64_t f = 0; f < n; ++f) {
            double x[NC], y[NC];
            promote(fib + f * NC, x, NC);
            apply_affine(aff, x, y);
            int64_t sig;
            int o, is;
            if (cidx_in) {
                sig = cidx_in[f];
                o = orient_in[f];
                is = argmax_in[f];
            } else {
                result_t r;
                if (!all_finite(y))
                    result_none(&r);
                else
                    label_brute_one(y, C, bundle_of, T, ord, M, &r);
                sig = r.cidx;
                o = r.orient;
                is = sig >= 0 ? argmax_point(y, C + sig * NC, o) : -1;
            }
            if (cidx_out) cidx_out[f] = (int32_t)sig;
            if (orient_out) orient_out[f] = (uint8_t)o;
            if (argmax_out) argmax_out[f] = is;
            if (gap) {
                if (sig >= 0) {
                    double dd, dr;
                    dme_both(y, C + sig * NC, &dd, &dr);
                    double m1 = o ? dr : dd;
                    double m2 = second_max(y, C + sig * NC, o, is);
                    double g1 = m1 - m2, g2 = fabs(dd - dr);
                    gap[f] = g1 < g2 ? g1 : g2;
                } else {
                    gap[f] = INFINITY;
                }
            }
            if (sig < 0 || (mask && !mask[f])) continue;
            int pi = o ? rev(is) : is;
            const double *cp = C + sig * NC + 3 * pi;
            double r0 = y[3 * is] - cp[0], r1 = y[3 * is + 1] - cp[1], r2 = y[3 * is + 2] - cp[2];
            double d = sqrt(r0 * r0 + r1 * r1 + r2 * r2);
            g[12] += d;
            if (d > 0.0) {
                double u[3] = {r0 / d, r1 / d, r2 / d};
                for (int r = 0; r < 3; ++r) {
                    for (int c = 0; c < 3; ++c) g[3 * r + c] += u[r] * x[3 * is + c];
                    g[9 + r] += u[r];
                    if (gc) gc[sig * NC + 3 * pi + r] -= u[r];
                }
            }
        }
    }
    double acc[13] = {0};
    for (int t = 0; t < nt; ++t)
        for (int k = 0; k < 13; ++k) acc[k] += pg[13 * t + k];
    if (cost) *cost = acc[12];
    if (grad_aff)
        for (int k = 0; k < 12; ++k) grad_aff[k] = acc[k];
    if (grad_cen) {
        memset(grad_cen, 0, (size_t)M * NC * sizeof(double));
        for (int t = 0; t < nt; ++t)
            for (int64_t k = 0; k < M * NC; ++k) grad_cen[k] += pc[(size_t)t * M * NC + k];
    }
    free(ord);
    free(C);
    free(T);
    free(pg);
    free(pc);
    return 0;
}
