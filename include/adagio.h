/*
 * adagio.h -- C ABI of the GB300-native ADAGIO library.
 *
 * ADAGIO (Blasiok & Tsourakakis, arXiv 1609.05388) embeds a point cloud
 * T = {x_1..x_n} in R^d linearly into R^m by
 *     f(w) = (P w, S (w - P^T P w))                              (Algorithm 1)
 * where P (s x d, orthonormal rows) spans the top-s principal subspace of the
 * zero-centred data (Sec. 2, "PCA") and S (k x d) has iid entries
 * +-1/sqrt(k) (Algorithm 1; Lemma 2), m = s + k.  For a target dimension m
 * the library uses s = floor(m/2), k = ceil(m/2) (Sec. 4.1) unless told
 * otherwise.  The map is stored as the m x d matrix A = [P ; S (I - P^T P)],
 * so that Y = X A^T.
 *
 * Quality is certified exhaustively: for every unordered pair i < j the
 * pair distortion  | ||y_i - y_j|| / ||x_i - x_j|| - 1 |  (Eq. 2) is formed,
 * and the certificate reports its maximum (Eq. 3, the embedding's distortion),
 * mean, a histogram and the number of pairs above eps.
 *
 * Conventions for every entry point:
 *  - Matrices are float32, row-major, one point per row, with an explicit
 *    leading dimension (elements between consecutive rows, >= the row length).
 *  - Array arguments may be DEVICE pointers (on the context's device) or HOST
 *    pointers (pageable or pinned).  Host inputs are copied to the device and
 *    host outputs copied back inside the call; this is the end-to-end path.
 *    Arrays are owned by the caller and never retained after the call.
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream).  Work is
 *    enqueued on it.  Entry points that return a host-side result (a
 *    certificate, a chosen dimension) synchronise that stream before
 *    returning; the others return as soon as the work is enqueued, unless a
 *    host output array forces a synchronising copy.
 *  - A context owns a device workspace and must not be used by two calls at
 *    the same time (calls on one context are serialised by the caller).
 *  - Every function returns ADAGIO_OK (0) or a negative status; no exception
 *    crosses the ABI and the library never exits or traps.  The message of
 *    the last failure on a context is returned by adagio_last_error().
 */
#ifndef ADAGIO_H
#define ADAGIO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ status */
#define ADAGIO_OK                  0
#define ADAGIO_E_INVALID_ARG      -1  /* a size, pointer or option is out of range   */
#define ADAGIO_E_NONFINITE        -2  /* an input holds NaN or Inf                   */
#define ADAGIO_E_CUDA             -3  /* a CUDA runtime call failed                  */
#define ADAGIO_E_WORKSPACE        -4  /* the workspace limit would be exceeded       */
#define ADAGIO_E_QUEUE_OVERFLOW   -5  /* recompute queue full even after a retry     */
#define ADAGIO_E_TIMEOUT          -6  /* a bounded device-side wait gave up          */
#define ADAGIO_E_NOT_CERTIFIABLE  -7  /* eps not reached at the largest allowed m    */
#define ADAGIO_E_UNSUPPORTED      -8  /* the device is not sm_103 or a mode is absent */

#define ADAGIO_HIST_BINS 64

/* Arithmetic of the all-pairs Gram tiles (the recompute of flagged
 * pairs is the same in every mode). */
#define ADAGIO_PREC_FP32     0  /* plain FP32 SIMT Gram tiles                       */
#define ADAGIO_PREC_FP16X3   1  /* tensor cores: 2-term FP16 split, 3 products,     */
                                /* FP32 accumulate (power-of-two scaled)            */
#define ADAGIO_PREC_BF16X3   2  /* tensor cores: 2-term BF16 split, 3 products      */

#define ADAGIO_JL_RADEMACHER 0  /* entries +-1/sqrt(k) (Algorithm 1)                */
#define ADAGIO_JL_GAUSSIAN   1  /* entries N(0, 1/k) (Box-Muller)                   */

typedef struct adagio_ctx adagio_ctx;

/*
 * Certificate of an embedding (Eq. 2 and Eq. 3 over all n(n-1)/2 pairs).
 *  pairs        n(n-1)/2
 *  degenerate   pairs with x_i == x_j (Eq. 2 undefined); excluded from all
 *               statistics below
 *  violations   pairs with distortion > eps (distortion == eps is allowed)
 *  overflow     pairs outside [hist_lo, hist_hi)
 *  recomputed   pairs whose fast tensor/SIMT value was too close to a bin
 *               edge, to eps, or too ill-conditioned, and were recomputed
 *               from coordinate differences (to within 1e-6, or exactly
 *               where that still leaves a bin edge or eps within reach)
 *  hist[b]      pairs with hist_lo + b*w <= distortion < hist_lo + (b+1)*w,
 *               w = (hist_hi - hist_lo) / 64
 *  max          largest distortion, at pair (argmax_i, argmax_j), i < j
 *  mean         mean distortion over the non-degenerate pairs
 *  max_err_bound   bound on |max - exact max| implied by the per-pair error
 *                  bounds (<= 1e-5 by construction)
 *  mean_err_bound  bound on |mean - exact mean|: the per-pair error bounds
 *                  averaged over the non-degenerate pairs (the tensor-core
 *                  tiles take each tile row's largest bound for its pairs)
 *  Histogram and violation counts are exact except possibly for pairs whose
 *  exact distortion lies within 1e-6 of a bin edge or of eps.
 */
typedef struct {
    uint64_t pairs, degenerate, violations, overflow, recomputed;
    uint64_t hist[ADAGIO_HIST_BINS];
    double max, mean, max_err_bound, mean_err_bound;
    int64_t argmax_i, argmax_j;
    double hist_lo, hist_hi, eps;
} adagio_cert;

/*
 * One shard's part of a certificate (adagio_distortion_shard): the raw sums
 * that adagio_cert_merge combines.  Fields as in adagio_cert, except
 *  pairs        the pairs of this shard's tiles
 *  sum          sum of the distortions of its non-degenerate pairs
 *  bound_sum    sum of their error bounds
 *  max          -1 when the shard has no non-degenerate pair
 *  max_bound    largest per-pair error bound
 *  shard, nshards   which part of how many
 */
typedef struct {
    uint64_t pairs, degenerate, violations, overflow, recomputed;
    uint64_t hist[ADAGIO_HIST_BINS];
    double sum, bound_sum, max, max_bound;
    int64_t argmax_i, argmax_j;
    double hist_lo, hist_hi, eps;
    int32_t shard, nshards;
} adagio_cert_part;

/*
 * Options of adagio_fit.  Fill with adagio_default_fit_opts() first.
 *  eps         > 0: search the smallest certified target dimension m (the
 *              exhaustive certificate's maximum distortion <= eps) by
 *              galloping (m = 16, 32, 64, ... capped at m_cap) and bisection;
 *              <= 0: fit at the fixed dimension `m`
 *  m           target dimension when eps <= 0
 *  s           number of principal rows; -1 = floor(m/2) (Sec. 4.1).  In a
 *              search, probe r uses min(s, r) of them: s = 0 is the JL-only
 *              map and s >= m_cap the PCA-only map, the two baselines Table 3
 *              compares ADAGIO with
 *  seed        seed of the JL matrix and of the randomized PCA start block
 *  jl_dist     ADAGIO_JL_RADEMACHER (default) or ADAGIO_JL_GAUSSIAN
 *  precision   arithmetic of the certificate tiles (ADAGIO_PREC_*)
 *  use_predictor  1: start from the dimension predictor's guess (needs a
 *              trained predictor on the context), verify it with the
 *              exhaustive certificate, and fall back to the search
 *  hist_lo/hi  histogram range; hi <= lo selects [0, 2 eps) (or [0, 1))
 *  max_iter, tol   subspace iteration stops when every Ritz residual
 *              ||C v - theta v|| <= tol * theta_1 for the kept vectors
 *  oversample  extra block columns of the subspace iteration (default 32)
 */
typedef struct {
    double eps;
    int m;
    int s;
    uint64_t seed;
    int jl_dist;
    int precision;
    int use_predictor;
    double hist_lo, hist_hi;
    int max_iter;
    double tol;
    int oversample;
} adagio_fit_opts;

void adagio_default_fit_opts(adagio_fit_opts *opts);

/* ----------------------------------------------------------------- context */
/* Creates a context on CUDA device `device`.  workspace_limit = 0 means no
 * limit; otherwise a call that would need more device workspace fails with
 * ADAGIO_E_WORKSPACE.  Fails with ADAGIO_E_UNSUPPORTED on a device that is
 * not compute capability 10.3.  *out is NULL on failure. */
int adagio_ctx_create(int device, size_t workspace_limit, adagio_ctx **out);
int adagio_ctx_destroy(adagio_ctx *ctx);
/* Message of the last failure on ctx ("" if none).  The pointer stays valid
 * until the next call on ctx.  NULL ctx gives the message of the last failed
 * adagio_ctx_create on this thread. */
const char *adagio_last_error(const adagio_ctx *ctx);
/* Bytes of device workspace currently held by ctx. */
size_t adagio_workspace_bytes(const adagio_ctx *ctx);

/* ------------------------------------------------------------- certificate */
/*
 * Exhaustive distortion certificate of the map x_i -> y_i (Eq. 2, Eq. 3).
 *  X  n x d (leading dimension ldx), Y  n x m (leading dimension ldy).
 *  eps in (0, 1): violation threshold.  hist_hi <= hist_lo selects [0, 2 eps).
 *  precision  ADAGIO_PREC_*.
 * Never materialises the n x n matrix.  Synchronises `stream`.
 * Errors: INVALID_ARG (n < 2, d < 1, m < 1, bad eps/range/pointers),
 * NONFINITE, WORKSPACE, QUEUE_OVERFLOW, CUDA.
 */
int adagio_distortion(adagio_ctx *ctx, const float *X, int64_t n, int d, int64_t ldx,
                      const float *Y, int m, int64_t ldy, double eps, double hist_lo,
                      double hist_hi, int precision, adagio_cert *out, void *stream);

/*
 * Shard `shard` of `nshards` of the certificate of adagio_distortion (the
 * same pairs, Eq. 2 and Eq. 3, split so that several GPUs or calls can each
 * take a part: the introduction's list of contributions and the conclusion
 * call the method amenable to distributed implementation).
 * The pairs are grouped in 128 x 128 tiles of the upper triangle, numbered
 * row by row: with B = 2 ceil(n / 256) block rows of 128 points (the last
 * ones partly or wholly past n), block row I holds the tiles (I, J),
 * J = I .. B - 1, and tile (I, J) the pairs (i, j), i in block I, j in block
 * J, i < j < n.  Shard s takes the tiles [T s / nshards, T (s + 1) / nshards)
 * of the T = B (B + 1) / 2 tiles.  The partition depends only on n, so shards computed on
 * different GPUs (whatever their tuned tile configuration) cover every pair
 * exactly once.  Arguments as adagio_distortion; 0 <= shard < nshards.
 * Writes `out`; synchronises `stream`.  ADAGIO_E_INVALID_ARG on bad sizes or
 * shard numbers.
 */
int adagio_distortion_shard(adagio_ctx *ctx, const float *X, int64_t n, int d, int64_t ldx,
                            const float *Y, int m, int64_t ldy, double eps, double hist_lo,
                            double hist_hi, int precision, int shard, int nshards,
                            adagio_cert_part *out, void *stream);

/*
 * Combines the `count` parts of one sharded certificate (host only, no GPU
 * work): counts and histograms add, the maximum is the largest (ties: the
 * lexicographically smallest pair, as in one call), the mean is the summed
 * distortions over the non-degenerate pairs.  Counts, histogram, maximum and
 * its pair equal those of adagio_distortion; the mean agrees to rounding.
 * ADAGIO_E_INVALID_ARG unless the parts are shards 0 .. count - 1 of count with
 * the same eps and histogram range.
 */
int adagio_cert_merge(const adagio_cert_part *parts, int count, adagio_cert *out);

/*
 * Verdict of one JL prefix in adagio_distortion_prefixes.
 *  k            JL rows the candidate keeps (kc)
 *  verdict      1: the candidate is certified (no pair's distortion exceeds
 *               eps); 0: some pair's distortion exceeds eps; -1: undecided
 *               (no violation found, but unsettled_pairs > 0)
 *  violations   pairs whose distortion exceeds eps: the exact count when
 *               unsettled_pairs = 0, else a lower bound
 *  recomputed   pairs the per-pair bounds left open (near eps, or possibly
 *               x_i == x_j), decided by an exact FP64 recompute of their rows
 *  unsettled_pairs  open pairs beyond the recompute queue's capacity (2^18
 *               pairs per call, shared by the candidates); 0 in practice
 *  max_lower, max_upper the candidate's largest distortion lies in
 *               [max_lower, max_upper] (bounds of the pairs' intervals and
 *               the exact values of the recomputed pairs); max_upper is +inf
 *               when an unsettled pair may have x_i == x_j
 *  Pairs with x_i == x_j are excluded, as in the certificate.
 */
typedef struct {
    int32_t k;
    int32_t verdict;
    uint64_t violations, unsettled_pairs, recomputed;
    double max_lower, max_upper;
} adagio_prefix_cert;

/*
 * Several target dimensions of the search of Algorithm 1 checked in one pass
 * over the pairs.  Y (n x (s + k), leading dimension ldy) is the embedding of
 * the map with s PCA rows and k JL rows (Lemma 2), the PCA coordinates first.
 * Candidate c keeps the PCA rows and the first kc[c] JL rows, rescaled to the
 * JL map with kc[c] rows (entries +-1/sqrt(kc[c]), so its squared distances
 * are |dP|^2 + (k / kc[c]) |dJ[:kc[c]]|^2).  Either every kc[c] is a multiple
 * of 64 or equal to k, or every k - kc[c] is a multiple of 64 (k, k - 64,
 * k - 128, ...: the prefixes below a dimension already fitted);
 * 1 <= kc[c] <= k; 1 <= count <= 4.  The pass computes `full`, the certificate of
 * the whole map (as adagio_distortion with hist [0, 2 eps)), and out[c], the
 * verdict of each candidate against eps: from per-pair bounds on its
 * distortion on the shared tensor-core Gram sums, and for the few pairs those
 * bounds leave open, from an exact recompute.
 *  precision    ADAGIO_PREC_FP16X3 or ADAGIO_PREC_BF16X3.
 * X, Y host or device; full and out host.  Synchronises `stream`.
 * Errors: INVALID_ARG (sizes, kc, count, eps in (0, 1), precision),
 * NONFINITE, WORKSPACE, QUEUE_OVERFLOW, UNSUPPORTED, CUDA.
 */
int adagio_distortion_prefixes(adagio_ctx *ctx, const float *X, int64_t n, int d, int64_t ldx,
                               const float *Y, int s, int k, int64_t ldy, double eps, const int *kc,
                               int count, int precision, adagio_cert *full, adagio_prefix_cert *out,
                               void *stream);

/*
 * Allocation-free certificate (the paper has no counterpart; this is a
 * deployment variant of adagio_distortion).  For callers that cannot let a
 * library allocate device memory during a call -- a service whose device
 * memory all belongs to its own pool, or a loop that cannot afford the
 * device-wide synchronisation of cudaMalloc/cudaFree -- it computes the same
 * certificate as adagio_distortion with precision ADAGIO_PREC_FP32, using
 * only a fixed 8 MiB scratch array that the library keeps in static device
 * memory (held by every GPU that loads the library until the process exits).
 *  Limits: n <= 1024, d <= 512, m <= 256, on a GPU of any SM count (the
 *          call uses at most 160 SMs' worth of CTAs); larger inputs fail with
 *          ADAGIO_E_INVALID_ARG.  X and Y must be device pointers; out is host.
 *  The first call on a device looks up the scratch array's device address;
 *  make that first call before capturing any stream on the device.
 *  All calls share the scratch array (it keeps the last call's contents and
 *  each call clears what must start at zero); overlapping calls would race, so
 *  calls are serialised by a host lock and the stream is synchronised before
 *  returning, on failure too.  No cudaMalloc, cudaFree or allocating library
 *  call is made.  adagio_last_cert_stats then reports this call.
 */
int adagio_distortion_noalloc(adagio_ctx *ctx, const float *X, int64_t n, int d, int64_t ldx,
                              const float *Y, int m, int64_t ldy, double eps, double hist_lo,
                              double hist_hi, adagio_cert *out, void *stream);

/* ------------------------------------------------------------------- embed */
/*
 * Y = X A^T: row i of Y is f(x_i) = A x_i (Algorithm 1's output for every w).
 *  A  m x d (lda), X  n x d (ldx), Y  n x m (ldy), written in full; n <= 2^30.
 * Computed on tcgen05 tensor cores from per-row power-of-two FP16 splits of X
 * and A (hi + lo, three products per term), FP32 accumulation: about 1e-7
 * relative to |A| |x| per entry.
 * Errors: INVALID_ARG, CUDA, WORKSPACE (host arrays need staging), TIMEOUT
 * (reported when Y is a host array; a device-array call does not synchronise,
 * and a later synchronising call on the context reports it).
 */
int adagio_embed(adagio_ctx *ctx, const float *A, int m, int d, int64_t lda,
                 const float *X, int64_t n, int64_t ldx, float *Y, int64_t ldy,
                 void *stream);

/* --------------------------------------------------------------- fit steps */
/*
 * JL matrix S (k x d, lds >= d): entry (i, j) is +-1/sqrt(k) by the top bit of
 * output number c = i*2^32 + 2j of the SplitMix64 stream seeded with `seed`
 * (Steele, Lea & Flood 2014); Gaussian: Box-Muller from outputs c and c + 1.
 * Row i does not depend on k except for the scale (Algorithm 1; Lemma 2).
 */
int adagio_jl_matrix(adagio_ctx *ctx, uint64_t seed, int k, int d, int jl_dist,
                     float *S, int64_t lds, void *stream);

/*
 * Top-s principal directions of X (Sec. 2 "PCA"; randomized PCA, Sec. 4.5):
 * randomized block subspace iteration on the covariance C = Xc^T Xc of the
 * centred data, shifted CholeskyQR2 orthonormalisation and Rayleigh-Ritz.
 *  P      s x d (ldp) orthonormal rows by decreasing eigenvalue; the entry of
 *         largest magnitude of each row is positive
 *  theta  s eigenvalue estimates of C (host or device, may be NULL)
 *  opts   seed, max_iter, tol, oversample are used (NULL = defaults)
 * Synchronises `stream`.  Errors: INVALID_ARG (s < 1 or s > d), NONFINITE,
 * WORKSPACE, CUDA.
 */
int adagio_pca(adagio_ctx *ctx, const float *X, int64_t n, int d, int64_t ldx, int s,
               const adagio_fit_opts *opts, float *P, int64_t ldp, double *theta,
               void *stream);

/*
 * A = [P ; S (I - P^T P)] (m = s + k rows, d columns, lda >= d): the matrix
 * of Algorithm 1's map w -> (P w, S (w - P^T P w)).  s or k may be 0.
 */
int adagio_assemble(adagio_ctx *ctx, const float *P, int s, int64_t ldp, const float *S,
                    int k, int64_t lds, int d, float *A, int64_t lda, void *stream);

/* --------------------------------------------------------------------- fit */
/*
 * Fits the ADAGIO map of X.  With opts->eps > 0 the smallest certified target
 * dimension found by the search is used (the paper's Table 3 question: how
 * many dimensions reach distortion eps); otherwise opts->m.
 *  A       output, m_cap x d (row-major, leading dimension d); the first
 *          *m_out rows hold the map
 *  m_cap   largest m allowed (<= d when eps > 0)
 *  m_out, s_out   chosen m and its number of principal rows
 *  cert    certificate of the returned map (may be NULL when eps <= 0)
 * Synchronises `stream`.  Errors: INVALID_ARG, NONFINITE, WORKSPACE, CUDA,
 * NOT_CERTIFIABLE (eps not reached at m_cap: A, m_out and cert still hold
 * the map at m_cap and its certificate).
 */
int adagio_fit(adagio_ctx *ctx, const float *X, int64_t n, int d, int64_t ldx,
               const adagio_fit_opts *opts, float *A, int m_cap, int *m_out, int *s_out,
               adagio_cert *cert, void *stream);

/* ------------------------------------------------------------- batched fit */
/*
 * One data set of a batched fit.  Inputs are set by the caller; the fields
 * marked "out" are written by adagio_fit_batched.
 */
typedef struct {
    const float *X;     /* device: n x d rows (row-major), leading dimension ldx >= d */
    int64_t n;          /* points, >= 2 */
    int d;              /* dimensions, >= 1 */
    int64_t ldx;
    double eps;         /* target maximum distortion in (0, 1); <= 0: fixed m */
    int m;              /* the fixed target dimension when eps <= 0 */
    int m_cap;          /* rows A can hold; the search probes up to min(m_cap, d) */
    float *A;           /* device: m_cap x d (leading dimension d); out: first m_out rows */
    int m_out, s_out;   /* out: chosen m and its number of principal rows */
    int status;         /* out: ADAGIO_OK or ADAGIO_E_NOT_CERTIFIABLE */
    int probes;         /* out: certificates the search ran */
    int full_certs;     /* out: of those, the ones that ran to completion */
    adagio_cert cert;   /* out: certificate of the returned map */
    float *feats;       /* device, 68 floats, or NULL: out: the predictor's
                           features of X (see adagio_features), taken from
                           this fit's own PCA */
} adagio_instance;

/* Capture each lock-step round as one CUDA graph (instantiated and launched
 * once) instead of launching its kernels one by one. */
#define ADAGIO_BATCH_GRAPH 1

/*
 * Fits `count` independent data sets of uneven n and d.  The paper has no
 * batched form: every instance gets exactly the fit adagio_fit computes for
 * it with the same opts (Algorithm 1 with the Sec. 4.1 split, the certified
 * search for the smallest m reaching eps), bit for bit.  The instances run in
 * lock-step rounds: each round enqueues, on one stream per instance, the next
 * piece of every unfinished instance (subspace iterations up to the next
 * convergence test, or one probe of the search: JL rows, A, Y = X A^T and the
 * exhaustive certificate), then synchronises once and takes every instance's
 * host decision.  Small instances therefore share the GPU instead of running
 * one after another, and a round costs one synchronisation for all of them.
 *  count  1 .. 4096 instances; inst[i] as described above (X and A on the
 *         device of ctx)
 *  opts   shared options: s (-1 = floor(m/2)), seed, jl_dist, precision,
 *         use_predictor (one batched network call after the first 64
 *         principal directions), hist_lo/hist_hi, max_iter, tol, oversample;
 *         opts->eps and opts->m are ignored (each instance has its own)
 *  flags  0 or ADAGIO_BATCH_GRAPH
 * The recompute queues and the workspace for all instances are reserved
 * before the first round.  Synchronises `stream`.  Returns ADAGIO_OK when
 * every instance has a map (an instance whose eps is not reached at its cap
 * gets status ADAGIO_E_NOT_CERTIFIABLE and the map at the cap, as adagio_fit
 * does); errors: INVALID_ARG, NONFINITE (in any instance), WORKSPACE,
 * QUEUE_OVERFLOW, TIMEOUT, CUDA.
 */
int adagio_fit_batched(adagio_ctx *ctx, int count, adagio_instance *inst,
                       const adagio_fit_opts *opts, int flags, void *stream);

/*
 * Statistics of the most recent adagio_fit_batched on ctx.
 *  rounds       lock-step rounds (one synchronisation each)
 *  graphs       rounds that ran as a captured CUDA graph
 *  pca_rounds   rounds that advanced some instance's subspace iteration
 *  total_ms     wall time of the call
 */
typedef struct {
    int rounds, graphs, pca_rounds;
    double total_ms;
} adagio_batch_stats;

int adagio_last_batch_stats(const adagio_ctx *ctx, adagio_batch_stats *out);

/* ----------------------------------------------------- dimension predictor */
/*
 * A small network predicts the target dimension the certified search would
 * return, so that adagio_fit (opts->use_predictor = 1) can start from the
 * prediction: the predicted m is verified with the exhaustive certificate and
 * returned if it passes; otherwise the search continues above it.  The paper
 * has no learned component; the certificate keeps every returned map exact.
 *  Features (68 floats): 0.5 log(theta_i / tr C) for the 64 leading eigenvalues
 *  of the centred covariance C (missing ones: 0.5 log 1e-12), log n, log d,
 *  eps, 1.  Network: 68 -> 256 -> 256 -> 1, exact GELU, output y = log m,
 *  BF16 weights with FP32 accumulation and activations; m = ceil(1.05 e^y).
 *  Parameters (adagio_mlp_num_params() floats): W1 [256][68], b1 [256],
 *  W2 [256][256], b2 [256], w3 [256], b3 [1] (FP32 master copy).
 *  Training: mean squared error on y, Adam (beta 0.9 / 0.999, eps 1e-8) with
 *  bias correction.  Arrays may be host or device pointers.
 */
int64_t adagio_mlp_num_params(void);
int adagio_mlp_init(adagio_ctx *ctx, uint64_t seed);
int adagio_mlp_set_params(adagio_ctx *ctx, const float *params, int64_t count);
int adagio_mlp_get_params(adagio_ctx *ctx, float *params, int64_t count);
/* y (count floats) = network output for `count` feature rows (count x 68). */
int adagio_mlp_forward(adagio_ctx *ctx, const float *feats, int count, float *y, void *stream);
/* Loss (mean squared error against target y) and its gradient, no update. */
int adagio_mlp_grad(adagio_ctx *ctx, const float *feats, const float *target, int count,
                    double *loss, float *grads, void *stream);
/* One Adam step on a batch; *loss (may be NULL) gets the batch loss before it. */
int adagio_mlp_train_step(adagio_ctx *ctx, const float *feats, const float *target, int count,
                          float lr, double *loss, void *stream);
/* m_out[i] = ceil(1.05 exp(y_i)) for each feature row. */
int adagio_predict_m(adagio_ctx *ctx, const float *feats, int count, int *m_out, void *stream);
/* Spectrum features of X for the predictor (68 floats, host or device). */
int adagio_features(adagio_ctx *ctx, const float *X, int64_t n, int d, int64_t ldx, double eps,
                    const adagio_fit_opts *opts, float *feats, void *stream);
/* Weights, Adam moments and step count to / from a file. */
int adagio_mlp_save(adagio_ctx *ctx, const char *path);
int adagio_mlp_load(adagio_ctx *ctx, const char *path);

/* ------------------------------------------------------------- diagnostics */
/*
 * Timing of the most recent certificate on ctx, taken with CUDA events on the
 * caller's stream around each stage when timing is enabled
 * (adagio_set_timing(ctx, 1); off by default, it adds one event pair per
 * stage).  All times in milliseconds; -1 when not measured.
 *  prep_ms       K0 (centring, split planes) of X and Y
 *  tile_ms       K8, the all-pairs tile kernel
 *  recompute_ms  K9 + K10 (recompute of queued pairs, finaliser)
 *  queued        pairs sent to the recompute
 *  grid          CTAs of the tile kernel; tiles = tile pairs it walked
 */
typedef struct {
    double prep_ms, tile_ms, recompute_ms;
    uint64_t queued;
    int grid;
    int64_t tiles;
} adagio_cert_stats;

/*
 * Statistics of the most recent adagio_fit on ctx.
 *  probes          certificates run by the search (early-exit probes included)
 *  full_certs      probes that ran to completion
 *  pca_iterations  subspace iterations over all blocks
 *  s_computed      principal directions computed
 *  pca_ms, total_ms  wall time of the PCA (covariance included) and of the fit
 *  predicted_m     the predictor's guess (0 when the predictor was not used)
 */
typedef struct {
    int probes, full_certs, pca_iterations, s_computed;
    double pca_ms, total_ms;
    int predicted_m;  /* the predictor's guess (0 when the predictor was not used) */
} adagio_fit_stats;

int adagio_last_fit_stats(const adagio_ctx *ctx, adagio_fit_stats *out);

int adagio_set_timing(adagio_ctx *ctx, int enable);
int adagio_last_cert_stats(const adagio_ctx *ctx, adagio_cert_stats *out);

/*
 * Tile configuration of the split-precision certificates (the all-pairs step
 * of Eq. 2 and Eq. 3; the classification of every pair does not depend on it):
 *   variant  ADAGIO_TILES_AUTO    default: the autotuned kernel for n's size
 *                                 class (adagio_autotune_tiles), else SINGLE
 *            ADAGIO_TILES_SINGLE  one CTA per 128 x 128 tile
 *            ADAGIO_TILES_PAIR    a cluster of two CTAs per 256 x 128 tile
 *                                 (SINGLE where such clusters cannot be
 *                                 resident on the device)
 *   band     tile rows (of 128 points) per band of the tile schedule, whose I
 *            tiles stay in L2 while the J tiles stream: 1 to 64, or 0 for the
 *            autotuned value, else 8
 * Returns ADAGIO_E_INVALID_ARG for any other value.  Adopted by the next call.
 */
#define ADAGIO_TILES_AUTO 0
#define ADAGIO_TILES_SINGLE 1
#define ADAGIO_TILES_PAIR 2
int adagio_set_tile_kernel(adagio_ctx *ctx, int variant, int band);

/*
 * Autotuner of the certificate's tile configuration.  Runs the certificate
 * of (X, Y) (host or device arrays, as adagio_distortion takes them) with
 * every candidate: each tile kernel the device runs (single CTA, CTA pair)
 * with schedule bands of 4, 8, 16, 32 and 64 tile rows; times the tile kernel with
 * CUDA events (one warm-up and three timed runs each, the fastest counts);
 * keeps the fastest on ctx for the size class of n (the number of 128-row
 * tile blocks rounded up to a power of two), where later certificates of
 * that class with variant and band left automatic use it.  Writes the chosen
 * configuration to *best.  Synchronises the stream.  Errors: those of
 * adagio_distortion.
 */
typedef struct {
    int variant;     /* ADAGIO_TILES_SINGLE or ADAGIO_TILES_PAIR */
    int band;        /* tile rows per schedule band */
    double tile_ms;  /* its tile-kernel time on the tuned problem */
    int size_class;  /* the size class of n it applies to */
} adagio_tile_config;
int adagio_autotune_tiles(adagio_ctx *ctx, const float *X, int64_t n, int d, int64_t ldx,
                          const float *Y, int m, int64_t ldy, double eps, int precision,
                          adagio_tile_config *best, void *stream);
/* The tuned table as JSON (device name and one entry per size class), and
 * back.  Loading a table of another device name loads nothing and returns
 * ADAGIO_E_INVALID_ARG; a malformed file also returns ADAGIO_E_INVALID_ARG. */
int adagio_tune_save(const adagio_ctx *ctx, const char *path);
int adagio_tune_load(adagio_ctx *ctx, const char *path);
/* The tile kernel that certifies n points on ctx (1 = single, 2 = pair);
 * queries the device on first use.  Negative on error. */
int adagio_tile_kernel_for(adagio_ctx *ctx, int64_t n);

/*
 * Error-model check of the certificate's fast path.  Runs the certificate of
 * (X, Y) like adagio_distortion and, for the 128 x 128 tile pairs number
 * q * stride (q = 0 .. tiles - 1) in the order the tile kernel visits them,
 * writes per pair (local row a, local column b) four floats at
 * out[((q * 128 + a) * 128 + b) * 4]: the fast squared
 * distances dx2 = ||xc_a||^2 + ||xc_b||^2 - 2 xc_a.xc_b and dy2 (likewise)
 * and their error bounds ex, ey; tile_ij[2q], tile_ij[2q+1] receive the tile
 * coordinates (I, J), so the pair is (128 I + a, 128 J + b).  Entries of
 * pairs outside i < j < n are written but meaningless.  Arrays are host or
 * device; `out` holds tiles * 65536 floats.  Synchronises `stream`.
 */
int adagio_debug_tile_bounds(adagio_ctx *ctx, const float *X, int64_t n, int d, int64_t ldx,
                             const float *Y, int m, int64_t ldy, int precision, int64_t tiles,
                             int64_t stride, float *out, int *tile_ij, void *stream);

/*
 * k nearest neighbours in an embedded space: the searches of the paper's
 * applications (Sec. 4.6, a 10-nearest-neighbour vote on embedded
 * descriptors; Sec. 4.7, a k = 30 nearest-neighbour graph of the embedded
 * points).  For every query row q of Q (nq x m, leading dimension ldq), the k
 * rows b of B (nb x m, ldb) with the smallest Euclidean distance ||q - b||
 * of the FP32 values, nearest first; equal distances are ordered by the
 * smaller base index; with exclude_self, base row i is not a neighbour of
 * query row i (the graph of one point set: pass the same array as Q and B).
 *  idx  nq x k base indices (row-major int64), d2  nq x k squared distances
 *       (FP64, from coordinate differences).  Host or device arrays.
 *  1 <= k <= 48, k <= nb (k <= nb - 1 with exclude_self).
 * Computed from tensor-core Gram blocks (split-precision FP16), with the
 * candidates re-ranked by exact FP64 distances; a row whose candidate list
 * cannot be shown complete from the Gram error bound is searched again over
 * every base point (adagio_knn_last_exact_rows counts them).  The answer is
 * the exact one.  Synchronises `stream`.
 * Errors: INVALID_ARG, NONFINITE (NaN or Inf in Q or B), WORKSPACE, CUDA, TIMEOUT.
 */
int adagio_knn(adagio_ctx *ctx, const float *Q, int64_t nq, int64_t ldq, const float *B,
               int64_t nb, int64_t ldb, int m, int k, int exclude_self, int64_t *idx,
               double *d2, void *stream);

/* Query rows of the last adagio_knn on ctx that were searched again over
 * every base point (their candidate list could not be shown complete). */
int64_t adagio_knn_last_exact_rows(const adagio_ctx *ctx);

/* Number of kernels this library has launched in this process (all contexts,
 * all devices); a difference of two readings counts the launches between. */
uint64_t adagio_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* ADAGIO_H */
