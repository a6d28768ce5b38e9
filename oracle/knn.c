/*
 * Plain FP64 k-nearest-neighbour search -- TEST INFRASTRUCTURE ONLY.
 *
 * Part of the CPU oracle; only the tests and the benchmark's CPU legs load it,
 * never the library.  It shares no code with the CUDA path.
 *
 * What it computes (the applications of Sec. 4.6 and Sec. 4.7 of the paper:
 * a 10-nearest-neighbour vote on embedded descriptors, and a k = 30
 * nearest-neighbour graph of the embedded points): for every query q, the k
 * base points b with the smallest Euclidean distance ||q - b||, found by
 * computing every distance from coordinate differences in double precision
 * (inputs are FP64; float32 data widen exactly) and keeping the k smallest.
 * Readings used here:
 *   - order: by squared distance, ties (equal FP64 values) by the smaller base
 *     index, so the answer is unique;
 *   - exclude_self (the k-NN graph of one point set): base point i is not a
 *     neighbour of query i.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>

typedef struct {
    const double *Q, *B;
    int64_t ldq, ldb, nq, nb;
    int m, k, exclude_self, tid, nthreads;
    int64_t *idx;
    double *d2;
} knn_job_t;

/* (d, j) comes before (e, l) */
static int before(double d, int64_t j, double e, int64_t l) { return d < e || (d == e && j < l); }

static void *knn_worker(void *arg) {
    knn_job_t *jb = (knn_job_t *)arg;
    const int k = jb->k;
    for (int64_t q = jb->tid; q < jb->nq; q += jb->nthreads) {
        const double *x = jb->Q + q * jb->ldq;
        int64_t *bi = jb->idx + q * k;
        double *bd = jb->d2 + q * k;
        int have = 0;
        for (int64_t j = 0; j < jb->nb; ++j) {
            if (jb->exclude_self && j == q) continue;
            const double *y = jb->B + j * jb->ldb;
            double acc = 0.0;
            for (int c = 0; c < jb->m; ++c) {
                const double t = x[c] - y[c];
                acc += t * t;
            }
            /* insert into the sorted list of the best `have` (at most k) */
            if (have == k && !before(acc, j, bd[k - 1], bi[k - 1])) continue;
            int pos = have < k ? have : k - 1;
            while (pos > 0 && before(acc, j, bd[pos - 1], bi[pos - 1])) {
                bd[pos] = bd[pos - 1];
                bi[pos] = bi[pos - 1];
                --pos;
            }
            bd[pos] = acc;
            bi[pos] = j;
            if (have < k) ++have;
        }
        for (int r = have; r < k; ++r) {
            bi[r] = -1;
            bd[r] = -1.0;
        }
    }
    return NULL;
}

/*
 * idx (nq x k) and d2 (nq x k): the k nearest base points of every query
 * and their squared distances, nearest first.  Returns 0, or -1 on bad
 * arguments.
 */
int oracle_knn(const double *Q, int64_t ldq, int64_t nq, const double *B, int64_t ldb, int64_t nb,
               int m, int k, int exclude_self, int nthreads, int64_t *idx, double *d2) {
    if (!Q || !B || !idx || !d2 || m < 1 || k < 1 || nq < 0 || nb < 0 || ldq < m || ldb < m)
        return -1;
    if (nthreads < 1) nthreads = 1;
    knn_job_t *jobs = (knn_job_t *)calloc((size_t)nthreads, sizeof(knn_job_t));
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    if (!jobs || !th) {
        free(jobs);
        free(th);
        return -1;
    }
    for (int t = 0; t < nthreads; ++t) {
        knn_job_t *jb = &jobs[t];
        jb->Q = Q; jb->B = B; jb->ldq = ldq; jb->ldb = ldb; jb->nq = nq; jb->nb = nb;
        jb->m = m; jb->k = k; jb->exclude_self = exclude_self; jb->tid = t; jb->nthreads = nthreads;
        jb->idx = idx; jb->d2 = d2;
    }
    for (int t = 1; t < nthreads; ++t) pthread_create(&th[t], NULL, knn_worker, &jobs[t]);
    knn_worker(&jobs[0]);
    for (int t = 1; t < nthreads; ++t) pthread_join(th[t], NULL);
    free(jobs);
    free(th);
    return 0;
}
