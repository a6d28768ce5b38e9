/*
 * Plain FP64 all-pairs distortion certificate -- TEST INFRASTRUCTURE ONLY.
 *
 * This file is part of the CPU oracle.  Only the tests, the smoke check and the
 * CPU-baseline leg of the benchmark may load it; the library never does.  It
 * shares no code, header or constant with the CUDA path.
 *
 * What it computes (the paper's definitions, written out directly):
 *   pair distortion   dist(x, y) = | ||f(x) - f(y)|| / ||x - y|| - 1 |      (Eq. 2)
 *   embedding distortion          max over all pairs of dist(x, y)        (Eq. 3)
 * with f(x_i) given as row i of Y (inputs are FP64; float32 data widen
 * exactly).  Every unordered pair i < j is visited once;
 * both squared distances are formed from coordinate differences, never from a
 * Gram matrix, and everything is accumulated in double precision.
 *
 * Readings of the paper used here:
 *   - a pair with ||x_i - x_j|| = 0 has no defined distortion (Eq. 2 divides by
 *     it); it is counted as "degenerate" and left out of every statistic;
 *   - "distortion at most delta" (Sec. 4.3) is read as <=: a pair with
 *     distortion exactly eps is not a violation (violation means > eps);
 *   - the histogram has nbins uniform bins [lo + b*w, lo + (b+1)*w) with
 *     w = (hi - lo) / nbins; values outside [lo, hi) count as overflow;
 *   - the maximum's argmax is the lexicographically smallest (i, j) among ties;
 *   - the mean is the Neumaier-compensated sum of distortions over the
 *     non-degenerate pairs divided by their number.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_MAX_BINS 256

typedef struct {
    uint64_t pairs;        /* pairs visited (including degenerate ones)          */
    uint64_t degenerate;   /* pairs with ||x_i - x_j|| == 0                      */
    uint64_t violations;   /* pairs with distortion > eps                        */
    uint64_t overflow;     /* non-degenerate pairs outside [lo, hi)              */
    uint64_t hist[ORACLE_MAX_BINS];
    double max;            /* largest distortion (0 if no non-degenerate pair)   */
    int64_t argmax_i, argmax_j;
    double sum;            /* Neumaier sum of distortions                        */
    double sum_c;          /* its compensation term                              */
    uint64_t near_edge;    /* pairs within edge_tol of a bin edge or of eps      */
} oracle_cert_t;

typedef struct {
    const double *X, *Y;
    int64_t ldx, ldy, n, row_begin, row_end;
    int d, m, nbins, tid, nthreads;
    double eps, lo, hi, edge_tol;
    oracle_cert_t res;
} job_t;

static void neumaier_add(double *sum, double *c, double v) {
    double t = *sum + v;
    if (fabs(*sum) >= fabs(v))
        *c += (*sum - t) + v;
    else
        *c += (v - t) + *sum;
    *sum = t;
}

static double sqdist(const double *a, const double *b, int len) {
    double acc = 0.0;
    for (int k = 0; k < len; ++k) {
        double t = a[k] - b[k];
        acc += t * t;
    }
    return acc;
}

static void record(oracle_cert_t *r, int64_t i, int64_t j, double dx2, double dy2,
                   double eps, double lo, double hi, int nbins, double edge_tol) {
    r->pairs++;
    if (dx2 == 0.0) {
        r->degenerate++;
        return;
    }
    double delta = fabs(sqrt(dy2 / dx2) - 1.0);
    if (delta > r->max || (r->argmax_i < 0)) {
        r->max = delta;
        r->argmax_i = i;
        r->argmax_j = j;
    }
    neumaier_add(&r->sum, &r->sum_c, delta);
    if (delta > eps) r->violations++;
    if (edge_tol > 0.0) {
        /* bookkeeping for comparisons: distance to the nearest edge lo + b*w */
        double w = (hi - lo) / (double)nbins;
        double t = (delta - lo) / w;
        double tn = floor(t + 0.5);
        int near = fabs(delta - eps) < edge_tol;
        if (tn >= 0.0 && tn <= (double)nbins && fabs(delta - (lo + tn * w)) < edge_tol) near = 1;
        if (near) r->near_edge++;
    }
    if (delta < lo || delta >= hi) {
        r->overflow++;
    } else {
        int b = (int)floor((delta - lo) / (hi - lo) * (double)nbins);
        if (b >= nbins) b = nbins - 1;
        if (b < 0) b = 0;
        r->hist[b]++;
    }
}

static void *worker(void *arg) {
    job_t *jb = (job_t *)arg;
    oracle_cert_t *r = &jb->res;
    memset(r, 0, sizeof(*r));
    r->argmax_i = r->argmax_j = -1;
    /* rows are dealt round-robin so that threads get similar pair counts */
    for (int64_t i = jb->row_begin + jb->tid; i < jb->row_end; i += jb->nthreads) {
        const double *xi = jb->X + i * jb->ldx;
        const double *yi = jb->Y + i * jb->ldy;
        for (int64_t j = i + 1; j < jb->n; ++j) {
            double dx2 = sqdist(xi, jb->X + j * jb->ldx, jb->d);
            double dy2 = sqdist(yi, jb->Y + j * jb->ldy, jb->m);
            record(r, i, j, dx2, dy2, jb->eps, jb->lo, jb->hi, jb->nbins, jb->edge_tol);
        }
    }
    return NULL;
}

/*
 * Certificate over the pairs (i, j) with row_begin <= i < row_end and
 * i < j < n.  row_begin = 0, row_end = n gives the full certificate.
 * Returns 0 on success, -1 on bad arguments.
 */
int oracle_certificate(const double *X, int64_t ldx, const double *Y, int64_t ldy,
                       int64_t n, int d, int m, double eps, double lo, double hi,
                       int nbins, int64_t row_begin, int64_t row_end, int nthreads,
                       double edge_tol, oracle_cert_t *out) {
    if (!X || !Y || !out || n < 0 || d < 1 || m < 1 || nbins < 1 ||
        nbins > ORACLE_MAX_BINS || !(hi > lo) || row_begin < 0 || row_end > n ||
        row_begin > row_end || ldx < d || ldy < m)
        return -1;
    if (nthreads < 1) nthreads = 1;
    job_t *jobs = (job_t *)calloc((size_t)nthreads, sizeof(job_t));
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    if (!jobs || !th) {
        free(jobs);
        free(th);
        return -1;
    }
    for (int t = 0; t < nthreads; ++t) {
        job_t *jb = &jobs[t];
        jb->X = X; jb->Y = Y; jb->ldx = ldx; jb->ldy = ldy; jb->n = n;
        jb->row_begin = row_begin; jb->row_end = row_end;
        jb->d = d; jb->m = m; jb->nbins = nbins; jb->tid = t; jb->nthreads = nthreads;
        jb->eps = eps; jb->lo = lo; jb->hi = hi; jb->edge_tol = edge_tol;
    }
    for (int t = 1; t < nthreads; ++t) pthread_create(&th[t], NULL, worker, &jobs[t]);
    worker(&jobs[0]);
    for (int t = 1; t < nthreads; ++t) pthread_join(th[t], NULL);

    memset(out, 0, sizeof(*out));
    out->argmax_i = out->argmax_j = -1;
    for (int t = 0; t < nthreads; ++t) {
        oracle_cert_t *r = &jobs[t].res;
        out->pairs += r->pairs;
        out->degenerate += r->degenerate;
        out->violations += r->violations;
        out->overflow += r->overflow;
        out->near_edge += r->near_edge;
        for (int b = 0; b < nbins; ++b) out->hist[b] += r->hist[b];
        neumaier_add(&out->sum, &out->sum_c, r->sum);
        neumaier_add(&out->sum, &out->sum_c, r->sum_c);
        if (r->argmax_i >= 0) {
            int better = out->argmax_i < 0 || r->max > out->max ||
                         (r->max == out->max &&
                          (r->argmax_i < out->argmax_i ||
                           (r->argmax_i == out->argmax_i && r->argmax_j < out->argmax_j)));
            if (better) {
                out->max = r->max;
                out->argmax_i = r->argmax_i;
                out->argmax_j = r->argmax_j;
            }
        }
    }
    out->sum += out->sum_c;
    out->sum_c = 0.0;
    free(jobs);
    free(th);
    return 0;
}

/* One row's pairs of a tile range: (i, j) for j in [jb, je). */
typedef struct {
    int64_t i, jb, je;
} segment_t;

typedef struct {
    const double *X, *Y;
    int64_t ldx, ldy;
    const segment_t *seg;
    int64_t nseg;
    int d, m, nbins, tid, nthreads;
    double eps, lo, hi, edge_tol;
    oracle_cert_t res;
} seg_job_t;

static void *seg_worker(void *arg) {
    seg_job_t *jb = (seg_job_t *)arg;
    oracle_cert_t *r = &jb->res;
    memset(r, 0, sizeof(*r));
    r->argmax_i = r->argmax_j = -1;
    for (int64_t q = jb->tid; q < jb->nseg; q += jb->nthreads) {
        const segment_t *sg = &jb->seg[q];
        const double *xi = jb->X + sg->i * jb->ldx;
        const double *yi = jb->Y + sg->i * jb->ldy;
        for (int64_t j = sg->jb; j < sg->je; ++j) {
            double dx2 = sqdist(xi, jb->X + j * jb->ldx, jb->d);
            double dy2 = sqdist(yi, jb->Y + j * jb->ldy, jb->m);
            record(r, sg->i, j, dx2, dy2, jb->eps, jb->lo, jb->hi, jb->nbins, jb->edge_tol);
        }
    }
    return NULL;
}

/*
 * Certificate over the pairs held by the tiles [t0, t1) of the upper triangle
 * of `tile` x `tile` blocks of the points, numbered row by row: with T block
 * rows (blocks <= 0: ceil(n / tile); more rows than that are blocks past n),
 * block row I holds the tiles (I, J), J = I .. T - 1, and tile (I, J) holds
 * the pairs (i, j) with i in block I, j in block J and i < j < n.  This is
 * the pair set of one shard of the GPU library's sharded certificate; the
 * definitions of every statistic are those of oracle_certificate.
 */
int oracle_certificate_tiles(const double *X, int64_t ldx, const double *Y, int64_t ldy,
                             int64_t n, int d, int m, double eps, double lo, double hi,
                             int nbins, int64_t tile, int64_t blocks, int64_t t0, int64_t t1,
                             int nthreads, double edge_tol, oracle_cert_t *out) {
    if (!X || !Y || !out || n < 0 || d < 1 || m < 1 || nbins < 1 || nbins > ORACLE_MAX_BINS ||
        !(hi > lo) || tile < 1 || t0 < 0 || t1 < t0 || ldx < d || ldy < m)
        return -1;
    if (nthreads < 1) nthreads = 1;
    const int64_t T = blocks > 0 ? blocks : (n + tile - 1) / tile;
    if (T * tile < n || t1 > T * (T + 1) / 2) return -1;
    /* the row segments: for each block row I, the block columns [Ja, Jb) of
       the range, hence j in [max(i + 1, Ja tile), min(n, Jb tile)) */
    int64_t cap = 0;
    for (int64_t I = 0, off = 0; I < T; off += T - I, ++I) {
        int64_t a = t0 > off ? t0 : off, b = t1 < off + (T - I) ? t1 : off + (T - I);
        if (a < b) cap += tile;
    }
    segment_t *seg = (segment_t *)calloc((size_t)(cap > 0 ? cap : 1), sizeof(segment_t));
    seg_job_t *jobs = (seg_job_t *)calloc((size_t)nthreads, sizeof(seg_job_t));
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    if (!seg || !jobs || !th) {
        free(seg);
        free(jobs);
        free(th);
        return -1;
    }
    int64_t nseg = 0;
    for (int64_t I = 0, off = 0; I < T; off += T - I, ++I) {
        int64_t a = t0 > off ? t0 : off, b = t1 < off + (T - I) ? t1 : off + (T - I);
        if (a >= b) continue;
        const int64_t Ja = I + (a - off), Jb = I + (b - off);
        for (int64_t i = I * tile; i < (I + 1) * tile && i < n; ++i) {
            int64_t jb = Ja * tile > i + 1 ? Ja * tile : i + 1;
            int64_t je = Jb * tile < n ? Jb * tile : n;
            if (jb < je) {
                seg[nseg].i = i;
                seg[nseg].jb = jb;
                seg[nseg].je = je;
                ++nseg;
            }
        }
    }
    for (int t = 0; t < nthreads; ++t) {
        seg_job_t *jb = &jobs[t];
        jb->X = X; jb->Y = Y; jb->ldx = ldx; jb->ldy = ldy; jb->seg = seg; jb->nseg = nseg;
        jb->d = d; jb->m = m; jb->nbins = nbins; jb->tid = t; jb->nthreads = nthreads;
        jb->eps = eps; jb->lo = lo; jb->hi = hi; jb->edge_tol = edge_tol;
    }
    for (int t = 1; t < nthreads; ++t) pthread_create(&th[t], NULL, seg_worker, &jobs[t]);
    seg_worker(&jobs[0]);
    for (int t = 1; t < nthreads; ++t) pthread_join(th[t], NULL);
    memset(out, 0, sizeof(*out));
    out->argmax_i = out->argmax_j = -1;
    for (int t = 0; t < nthreads; ++t) {
        oracle_cert_t *r = &jobs[t].res;
        out->pairs += r->pairs;
        out->degenerate += r->degenerate;
        out->violations += r->violations;
        out->overflow += r->overflow;
        out->near_edge += r->near_edge;
        for (int b = 0; b < nbins; ++b) out->hist[b] += r->hist[b];
        neumaier_add(&out->sum, &out->sum_c, r->sum);
        neumaier_add(&out->sum, &out->sum_c, r->sum_c);
        if (r->argmax_i >= 0) {
            int better = out->argmax_i < 0 || r->max > out->max ||
                         (r->max == out->max &&
                          (r->argmax_i < out->argmax_i ||
                           (r->argmax_i == out->argmax_i && r->argmax_j < out->argmax_j)));
            if (better) {
                out->max = r->max;
                out->argmax_i = r->argmax_i;
                out->argmax_j = r->argmax_j;
            }
        }
    }
    out->sum += out->sum_c;
    out->sum_c = 0.0;
    free(seg);
    free(jobs);
    free(th);
    return 0;
}

typedef struct {
    const double *X, *Y;
    int64_t ldx, ldy;
    int d, m;
    const int64_t *I, *J;
    int64_t begin, end;
    double *dx2, *dy2;
} pairs_job_t;

static void *pairs_worker(void *arg) {
    pairs_job_t *jb = (pairs_job_t *)arg;
    for (int64_t p = jb->begin; p < jb->end; ++p) {
        jb->dx2[p] = sqdist(jb->X + jb->I[p] * jb->ldx, jb->X + jb->J[p] * jb->ldx, jb->d);
        jb->dy2[p] = sqdist(jb->Y + jb->I[p] * jb->ldy, jb->Y + jb->J[p] * jb->ldy, jb->m);
    }
    return NULL;
}

/*
 * Squared distances ||x_i - x_j||^2 and ||y_i - y_j||^2 (FP64, direct
 * differences) for an explicit list of pairs; used to check sampled outputs of
 * full-size runs one pair at a time.  The list is split evenly over nthreads.
 */
int oracle_pair_sqdist(const double *X, int64_t ldx, const double *Y, int64_t ldy,
                       int d, int m, const int64_t *I, const int64_t *J,
                       int64_t npairs, double *dx2, double *dy2, int nthreads) {
    if (!X || !Y || !I || !J || !dx2 || !dy2 || d < 1 || m < 1) return -1;
    if (nthreads < 1) nthreads = 1;
    pairs_job_t *jobs = (pairs_job_t *)calloc((size_t)nthreads, sizeof(pairs_job_t));
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    if (!jobs || !th) {
        free(jobs);
        free(th);
        return -1;
    }
    for (int t = 0; t < nthreads; ++t) {
        pairs_job_t *jb = &jobs[t];
        jb->X = X; jb->Y = Y; jb->ldx = ldx; jb->ldy = ldy; jb->d = d; jb->m = m;
        jb->I = I; jb->J = J; jb->dx2 = dx2; jb->dy2 = dy2;
        jb->begin = npairs * t / nthreads;
        jb->end = npairs * (t + 1) / nthreads;
    }
    for (int t = 1; t < nthreads; ++t) pthread_create(&th[t], NULL, pairs_worker, &jobs[t]);
    pairs_worker(&jobs[0]);
    for (int t = 1; t < nthreads; ++t) pthread_join(th[t], NULL);
    free(jobs);
    free(th);
    return 0;
}
