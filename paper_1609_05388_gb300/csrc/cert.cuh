// Certificate pipeline: launch descriptors shared by the tile kernels, the
// recompute and the finaliser.
#pragma once

#include "internal.cuh"
#include "cert_common.cuh"
#include "prep.cuh"

namespace adagio {

// JL-prefix candidates of the multi-candidate certificate (one pass of the
// single-CTA tensor tiles): Y holds the PCA part in its first s_pad = pad64(s)
// columns (zeros after s), zeros up to column jo and k JL columns from jo;
// candidate c keeps the first kc[c] JL columns scaled by sqrt(k / kc[c]), and
// jo + kc[c] is a multiple of 64 or kc[c] = k.  The kernel writes one verdict
// record per epilogue warp and candidate into `out` (device); `cs` (device)
// receives the candidates' row statistics.
struct MultiSpec {
    int count = 0;
    int s = 0, s_pad = 0, jo = 0, k = 0;
    int kc[4] = {0, 0, 0, 0};
    double eps = 0.0;          // the candidates' violation threshold (FP64, as given)
    void *cs = nullptr;        // count x n_pad float4
    void *out = nullptr;       // slots x count verdict records (32 B each)
    int slots = 0;             // records per candidate (CTAs x epilogue warps)
    void *cq = nullptr;        // device: int4 (i, j, candidate, 0) of the open pairs
    unsigned long long *cqcount = nullptr;  // device: open pairs offered (zeroed by the caller)
    unsigned long long cqcap = 0;
};

struct CertLaunch {
    adagio_ctx *ctx = nullptr;
    const PrepMat *x = nullptr;
    const PrepMat *y = nullptr;
    CertConst cc{};
    CertPartial *partials = nullptr;  // [grid]
    int grid = 0;
    int2 *queue = nullptr;
    unsigned long long *qcount = nullptr;
    unsigned long long qcap = 0;
    int *stop_flag = nullptr;         // early exit (search probes) or null
    int *status = nullptr;            // device status word (timeouts)
    void *dump = nullptr;             // optional per-pair (dx2, dy2, ex, ey) dump
    long long dump_tiles = 0;         // tile pairs to dump (schedule order)
    long long dump_stride = 1;        // every dump_stride-th tile pair
    void *rs_xy = nullptr;            // tensor path: per-row statistics (2 n_pad float4: by row, by column pair)
    // tiles [t_begin, t_end) of the row-major upper triangle of 128 x 128
    // tiles (a shard); t_end < 0: all of them
    long long t_begin = 0, t_end = -1;
    const MultiSpec *multi = nullptr;  // multi-candidate pass (single-CTA tensor tiles)
    const float *ysrc = nullptr;       // Y as given (the candidates' row statistics)
    int64_t ldy_src = 0;
};

// Device-side result of the finaliser (host copies it back).
struct CertDevResult {
    unsigned long long hist[kBins];
    unsigned long long fast_pairs, queued, recomputed, degenerate, violations, overflow;
    double sum, bound_sum;
    float max, max_bound;
    int argmax_i, argmax_j;
    unsigned flags;
    int status;
    int stopped;  // the early-exit flag fired: statistics are partial
    unsigned long long qlen;  // pairs pushed to the recompute queue (may exceed its capacity)
};

void launch_cert_simt(const CertLaunch &L, cudaStream_t st);
int cert_simt_threads();
// tcgen05 tile kernel; returns false when the shape is not supported
bool launch_cert_tc(const CertLaunch &L, int precision, cudaStream_t st);
void cert_tc_init();
void cert_simt_init();
void recompute_init();
// every certificate kernel's attributes, set once (call before a capture)
void cert_init();
// 128-row block coordinates of 128 x 128 tile unit u of the tensor-core kernel
void tc_tile_coords(adagio_ctx *ctx, int64_t n, long long u, int *I, int *J);
// tensor-core tile kernel for n points: 1 = one CTA per tile, 2 = CTA pairs
int tc_variant(adagio_ctx *ctx, int64_t n);
// the tile configuration (kernel and schedule band) used for n points
TileConfig tc_config(adagio_ctx *ctx, int64_t n);
// size class of n for the tuned table: ceil(log2(128-row tile blocks))
int tc_size_class(int64_t n);
// whether CTA-pair tiles can run on the context's device
bool tc_pair_supported(adagio_ctx *ctx);

// Exact recompute of the queued pairs from the original (uncentred) inputs.
void launch_recompute(const float *X, int64_t ldx, int d, const float *Y, int64_t ldy, int m,
                      const int2 *queue, const unsigned long long *qcount,
                      unsigned long long qcap, CertConst cc, CertPartial *partials, int grid,
                      cudaStream_t st);

void launch_finalize(const CertPartial *fast, int nfast, const CertPartial *rec, int nrec,
                     const unsigned long long *qcount, const unsigned *flags, const int *status,
                     const int *stop_flag, CertDevResult *out, cudaStream_t st);
int cert_tc_ctas(adagio_ctx *ctx, int64_t n);
// partial records one tensor-core tile CTA writes (one per epilogue warp)
int cert_tc_slots_per_cta();

// Full certificate of (X, Y) given device pointers.  Fills `out`; returns the
// status (ADAGIO_OK, ADAGIO_E_NONFINITE, ...).  stop_early: the tile kernels
// stop at the first certain violation (a search probe only needs max > eps),
// in which case the statistics are partial and only out->max > eps is
// meaningful.  Synchronises `st`.
struct CertOptions {
    double eps = 0.1, lo = 0.0, hi = 0.2;
    int precision = ADAGIO_PREC_FP16X3;
    bool stop_early = false;
    void *dump = nullptr;       // per-pair fast values of the first dump_tiles tile pairs
    long long dump_tiles = 0;
    long long dump_stride = 1;
    int shard = 0, nshards = 1;  // this shard of the tiles (adagio_distortion_shard)
    const MultiSpec *multi = nullptr;  // JL-prefix candidates checked in the same pass
};

// Tiles [*t0, *t1) of shard `shard` of `nshards` (row-major upper triangle of
// the 128 x 128 tiles of n points) and the pairs i < j < n they hold.
void shard_range(int64_t n, int shard, int nshards, long long *t0, long long *t1);
unsigned long long shard_pairs(int64_t n, long long t0, long long t1);
// the certificate of one or more shard parts (adagio_cert_merge's arithmetic)
void cert_from_parts(const adagio_cert_part *parts, int count, adagio_cert *out);

// 128-row block coordinates of the t-th 128 x 128 tile the tile kernel of
// `precision` visits for n points (host side, for diagnostics).
void tile_coords(adagio_ctx *ctx, int precision, int64_t n, long long t, int *I, int *J);
// Writes `out` (the certificate), or with part_out the raw part of the shard
// that opt selects (out may then be null).
int certify(adagio_ctx *ctx, const float *X, int64_t ldx, const float *Y, int64_t ldy, int64_t n,
            int d, int m, const CertOptions &opt, adagio_cert *out, cudaStream_t st,
            bool *stopped = nullptr, const PrepMat *px_ready = nullptr,
            adagio_cert_part *part_out = nullptr);
size_t certify_bytes(adagio_ctx *ctx, int64_t n, int d, int m, int precision);

// The certificate as three host steps, so that many can be enqueued before
// one synchronisation (batched fits, graph capture):
//   cert_job_setup    carves the job's device scratch from the workspace
//   cert_job_enqueue  enqueues all device work (no host sync, no allocation)
//   cert_job_collect  interprets the copied-back CertDevResult
struct CertJob {
    const float *X = nullptr, *Y = nullptr;
    int64_t ldx = 0, ldy = 0, n = 0;
    int d = 0, m = 0;
    CertOptions opt;
    const PrepMat *px = nullptr;      // prepared X (owned by the caller, reusable)
    unsigned *flags = nullptr;
    int *stop = nullptr, *status = nullptr;
    unsigned long long *qcount = nullptr;
    CertPartial *partials = nullptr, *rparts = nullptr;
    int nparts = 0, rgrid = 0;
    CertDevResult *dres = nullptr;
    float4 *rs_xy = nullptr;
    int2 *queue = nullptr;
    unsigned long long qcap = 0;
    PrepMat py;                        // Y prep, carved from the workspace by enqueue
    bool clear_flags = true;           // enqueue zeroes `flags` (false: the caller did)
};
size_t cert_job_bytes(adagio_ctx *ctx, int64_t n, int m, int precision);
size_t cert_prep_x_bytes(int64_t n, int d, int precision);
// prepares X for certificates (the split planes or the FP32 copy)
void cert_prepare_x(adagio_ctx *ctx, const float *X, int64_t ldx, int64_t n, int d, int precision,
                    PrepMat &px, unsigned *flags, cudaStream_t st);
void cert_job_setup(adagio_ctx *ctx, CertJob &job, int2 *queue, unsigned long long qcap);
// carves the Y prep from the workspace; `ev` (optional) gets ev[1] after the
// preps and ev[2] after the tile kernel
void cert_job_enqueue(adagio_ctx *ctx, CertJob &job, cudaStream_t st, cudaEvent_t *ev = nullptr);
// 0 = ok; ADAGIO_E_QUEUE_OVERFLOW when the queue was too small (retry with more)
int cert_job_collect(const CertJob &job, const CertDevResult &h, adagio_cert *out, bool *stopped,
                     adagio_cert_part *part_out = nullptr);
unsigned long long cert_queue_capacity(unsigned long long pairs);
void cert_ensure_queue(adagio_ctx *ctx, unsigned long long cap);
// tensor path: makes the tile schedule for n points resident (call before capture)
void tc_prepare(adagio_ctx *ctx, int64_t n);


}  // namespace adagio
