// Certificate orchestration (Eq. 2, Eq. 3): K0 prep of X and Y, K8 tile
// kernel (FP32 SIMT or tcgen05 split precision), K9 recompute of the
// flagged pairs, K10 finaliser, one device->host copy of the result.
#include "internal.cuh"
#include "cert.cuh"

#include <cmath>
#include <cstring>

namespace adagio {

// Initial capacity of the recompute queue: 1/256 of the pairs (at least
// 2^20 entries; split-precision tiles typically queue 0.2 %); it grows to the
// observed need when a run overflows it.
unsigned long long cert_queue_capacity(unsigned long long pairs) {
    unsigned long long q = pairs / 256;
    if (q < (1ull << 20)) q = 1ull << 20;
    if (q > pairs) q = pairs;
    return q;
}

void cert_ensure_queue(adagio_ctx *ctx, unsigned long long cap) {
    if (ctx->qbuf_cap >= cap) return;
    if (ctx->qbuf_fixed)
        fail(ADAGIO_E_QUEUE_OVERFLOW, "recompute queue needs %llu entries, fixed capacity is %llu", cap,
             ctx->qbuf_cap);
    if (ctx->qbuf) {
        ADAGIO_CUDA(cudaDeviceSynchronize());  // a previous certificate may still read it
        ADAGIO_CUDA(cudaFree(ctx->qbuf));
        ctx->qbuf = nullptr;
        ctx->qbuf_cap = 0;
    }
    cudaError_t e = cudaMalloc(&ctx->qbuf, cap * sizeof(int2));
    if (e != cudaSuccess) {
        cudaGetLastError();
        ctx->qbuf = nullptr;
        fail(ADAGIO_E_WORKSPACE, "cudaMalloc of a %llu-entry recompute queue failed: %s", cap,
             cudaGetErrorString(e));
    }
    ctx->qbuf_cap = cap;
}

void cert_init() {
    cert_tc_init();
    cert_simt_init();
    recompute_init();
}

static int partial_slots(adagio_ctx *ctx, int64_t n, int precision) {
    if (precision == ADAGIO_PREC_FP32) return ctx->num_sms;  // 1 CTA / SM (64 KB hist + regs)
    return cert_tc_ctas(ctx, n) * cert_tc_slots_per_cta();    // one slot per epilogue warp
}

static int recompute_grid(adagio_ctx *ctx) { return ctx->num_sms * 3; }  // resident: 3 x 256 threads / SM

size_t cert_prep_x_bytes(int64_t n, int d, int precision) {
    const bool tc = precision != ADAGIO_PREC_FP32;
    return prep_bytes(n, d, !tc, tc);
}

size_t cert_job_bytes(adagio_ctx *ctx, int64_t n, int m, int precision) {
    const bool tc = precision != ADAGIO_PREC_FP32;
    size_t b = prep_bytes(n, m, !tc, tc);
    b += align_up(sizeof(CertPartial) * (partial_slots(ctx, n, precision) + recompute_grid(ctx)), 256);
    b += 4 * 256 + align_up(sizeof(CertDevResult), 256);
    if (tc) b += align_up(2 * (size_t)pad_rows(n) * sizeof(float4), 256);
    return b + 1024;
}

size_t certify_bytes(adagio_ctx *ctx, int64_t n, int d, int m, int precision) {
    return cert_prep_x_bytes(n, d, precision) + cert_job_bytes(ctx, n, m, precision) + 4096;
}

void cert_prepare_x(adagio_ctx *ctx, const float *X, int64_t ldx, int64_t n, int d, int precision,
                    PrepMat &px, unsigned *flags, cudaStream_t st) {
    const bool tc = precision != ADAGIO_PREC_FP32;
    prep_matrix(ctx, X, n, d, ldx, precision, !tc, tc, px, flags, st);
}

void cert_job_setup(adagio_ctx *ctx, CertJob &job, int2 *queue, unsigned long long qcap) {
    job.flags = ws_array<unsigned>(ctx, 1);
    job.stop = ws_array<int>(ctx, 1);
    job.status = ws_array<int>(ctx, 1);
    job.qcount = ws_array<unsigned long long>(ctx, 1);
    job.nparts = partial_slots(ctx, job.n, job.opt.precision);
    job.rgrid = recompute_grid(ctx);
    job.partials = ws_array<CertPartial>(ctx, job.nparts);
    job.rparts = ws_array<CertPartial>(ctx, job.rgrid);
    job.dres = ws_array<CertDevResult>(ctx, 1);
    const bool tc = job.opt.precision != ADAGIO_PREC_FP32;
    const int64_t n_pad = pad_rows(job.n);
    job.rs_xy = tc ? ws_array<float4>(ctx, 2 * (size_t)n_pad) : nullptr;
    job.queue = queue;
    job.qcap = qcap;
}

void cert_job_enqueue(adagio_ctx *ctx, CertJob &job, cudaStream_t st, cudaEvent_t *ev) {
    const bool tc = job.opt.precision != ADAGIO_PREC_FP32;
    const CertOptions &opt = job.opt;
    if (job.clear_flags) ADAGIO_CUDA(cudaMemsetAsync(job.flags, 0, sizeof(unsigned), st));
    ADAGIO_CUDA(cudaMemsetAsync(job.stop, 0, sizeof(int), st));
    ADAGIO_CUDA(cudaMemsetAsync(job.status, 0, sizeof(int), st));
    ADAGIO_CUDA(cudaMemsetAsync(job.qcount, 0, sizeof(unsigned long long), st));
    prep_matrix(ctx, job.Y, job.n, job.m, job.ldy, opt.precision, !tc, tc, job.py, job.flags, st);
    if (ev) ADAGIO_CUDA(cudaEventRecord(ev[1], st));

    CertLaunch L;
    L.ctx = ctx;
    L.x = job.px;
    L.y = &job.py;
    L.cc.lo = (float)opt.lo;
    L.cc.hi = (float)opt.hi;
    L.cc.w = (float)((opt.hi - opt.lo) / kBins);
    L.cc.inv_w = (float)(kBins / (opt.hi - opt.lo));
    L.cc.eps = (float)opt.eps;
    L.cc.c_r = 8.0f * 5.9604645e-08f;
    L.cc.lo_is_floor = opt.lo <= 0.0;
    L.grid = job.nparts;
    L.partials = job.partials;
    L.queue = job.queue;
    L.qcount = job.qcount;
    L.qcap = job.qcap;
    L.stop_flag = opt.stop_early ? job.stop : nullptr;
    L.status = job.status;
    L.dump = opt.dump;
    L.dump_tiles = opt.dump_tiles;
    L.dump_stride = opt.dump_stride;
    L.multi = opt.multi;
    L.ysrc = job.Y;
    L.ldy_src = job.ldy;
    L.rs_xy = job.rs_xy;
    if (opt.nshards > 1) shard_range(job.n, opt.shard, opt.nshards, &L.t_begin, &L.t_end);
    if (tc) {
        if (!launch_cert_tc(L, opt.precision, st))
            fail(ADAGIO_E_UNSUPPORTED, "tensor-core certificate does not support n=%lld",
                 (long long)job.n);
    } else {
        launch_cert_simt(L, st);
    }
    if (ev) ADAGIO_CUDA(cudaEventRecord(ev[2], st));
    launch_recompute(job.X, job.ldx, job.d, job.Y, job.ldy, job.m, job.queue, job.qcount, job.qcap,
                     L.cc, job.rparts, job.rgrid, st);
    launch_finalize(job.partials, job.nparts, job.rparts, job.rgrid, job.qcount, job.flags,
                    job.status, job.stop, job.dres, st);
}

void shard_range(int64_t n, int shard, int nshards, long long *t0, long long *t1) {
    const long long T = pad_rows(n) / kTileRows, ntp = T * (T + 1) / 2;
    *t0 = (long long)((__int128)ntp * shard / nshards);
    *t1 = (long long)((__int128)ntp * (shard + 1) / nshards);
}

unsigned long long shard_pairs(int64_t n, long long t0, long long t1) {
    const long long T = pad_rows(n) / kTileRows;
    auto rows = [&](long long I) {
        return (unsigned long long)std::max<int64_t>(0, std::min<int64_t>(kTileRows, n - I * kTileRows));
    };
    unsigned long long p = 0;
    long long off = 0;
    for (long long I = 0; I < T && off < t1; off += T - I, ++I) {
        // row I holds tiles off .. off + T - I - 1 (J = I .. T - 1)
        const long long lo = std::max(t0, off), hi = std::min(t1, off + T - I);
        const unsigned long long rI = rows(I);
        for (long long t = lo; t < hi; ++t) {
            const long long J = I + (t - off);
            p += J == I ? rI * (rI - (rI > 0)) / 2 : rI * rows(J);
        }
    }
    return p;
}

void cert_from_parts(const adagio_cert_part *parts, int count, adagio_cert *out) {
    std::memset(out, 0, sizeof(*out));
    double sum = 0.0, bsum = 0.0, mxb = 0.0;
    double mx = -1.0;
    int64_t ai = -1, aj = -1;
    for (int q = 0; q < count; ++q) {
        const adagio_cert_part &p = parts[q];
        out->pairs += p.pairs;
        out->degenerate += p.degenerate;
        out->violations += p.violations;
        out->overflow += p.overflow;
        out->recomputed += p.recomputed;
        for (int b = 0; b < kBins; ++b) out->hist[b] += p.hist[b];
        sum += p.sum;
        bsum += p.bound_sum;
        mxb = std::max(mxb, p.max_bound);
        // the larger distortion; on a tie the lexicographically smaller pair
        if (p.max >= 0.0 && (p.max > mx || (p.max == mx && (p.argmax_i < ai || (p.argmax_i == ai &&
                                                                                  p.argmax_j < aj))))) {
            mx = p.max;
            ai = p.argmax_i;
            aj = p.argmax_j;
        }
    }
    const unsigned long long good = out->pairs - out->degenerate;
    if (mx >= 0.0) {
        out->max = mx;
        out->argmax_i = ai;
        out->argmax_j = aj;
    } else {
        out->max = 0.0;
        out->argmax_i = out->argmax_j = -1;
    }
    out->mean = good ? sum / (double)good : 0.0;
    out->max_err_bound = std::max(mxb, 1e-12);
    out->mean_err_bound = good ? bsum / (double)good : 0.0;
    out->hist_lo = parts[0].hist_lo;
    out->hist_hi = parts[0].hist_hi;
    out->eps = parts[0].eps;
}

int cert_job_collect(const CertJob &job, const CertDevResult &h, adagio_cert *out, bool *stopped,
                     adagio_cert_part *part_out) {
    const CertOptions &opt = job.opt;
    unsigned long long pairs = (unsigned long long)job.n * (unsigned long long)(job.n - 1) / 2;
    if (opt.nshards > 1) {
        long long t0, t1;
        shard_range(job.n, opt.shard, opt.nshards, &t0, &t1);
        pairs = shard_pairs(job.n, t0, t1);
    }
    if (h.flags & 1u) fail(ADAGIO_E_NONFINITE, "input holds NaN or Inf");
    if (h.status != 0)
        fail(ADAGIO_E_TIMEOUT, "certificate kernel gave up a bounded wait (status %d)", h.status);
    // a stopped certificate found a certain violation on the fast path: its
    // verdict does not depend on the recompute queue, so an overflow is moot
    if (h.qlen > job.qcap && !h.stopped) return ADAGIO_E_QUEUE_OVERFLOW;
    if (stopped) *stopped = h.stopped != 0;
    if (!h.stopped) {
        if (h.fast_pairs + h.queued != pairs || h.queued != h.qlen ||
            h.recomputed + h.degenerate != h.qlen)
            fail(ADAGIO_E_CUDA,
                 "internal: pair accounting mismatch (fast %llu + queued %llu != %llu, recomputed "
                 "%llu, degenerate %llu)",
                 h.fast_pairs, h.queued, pairs, h.recomputed, h.degenerate);
    }
    adagio_cert_part p;
    std::memset(&p, 0, sizeof(p));
    p.pairs = pairs;
    p.degenerate = h.degenerate;
    p.violations = h.violations;
    p.overflow = h.overflow;
    p.recomputed = h.recomputed + h.degenerate;
    std::memcpy(p.hist, h.hist, sizeof(p.hist));
    p.sum = h.sum;
    p.bound_sum = h.bound_sum;
    p.max = h.max >= 0.0f ? (double)h.max : -1.0;
    p.max_bound = h.max_bound;
    p.argmax_i = h.max >= 0.0f ? h.argmax_i : -1;
    p.argmax_j = h.max >= 0.0f ? h.argmax_j : -1;
    p.hist_lo = opt.lo;
    p.hist_hi = opt.hi;
    p.eps = opt.eps;
    p.shard = opt.shard;
    p.nshards = opt.nshards;
    if (part_out) *part_out = p;
    if (out) cert_from_parts(&p, 1, out);
    return ADAGIO_OK;
}

int certify(adagio_ctx *ctx, const float *X, int64_t ldx, const float *Y, int64_t ldy, int64_t n,
            int d, int m, const CertOptions &opt, adagio_cert *out, cudaStream_t st,
            bool *stopped, const PrepMat *px_ready, adagio_cert_part *part_out) {
    const bool tc = opt.precision != ADAGIO_PREC_FP32;
    const unsigned long long pairs = (unsigned long long)n * (unsigned long long)(n - 1) / 2;
    if (!ctx->qbuf_fixed) cert_ensure_queue(ctx, cert_queue_capacity(pairs));
    if (tc) tc_prepare(ctx, n);
    const size_t mark = ctx->ws.off;
    for (int attempt = 0; attempt < 2; ++attempt) {
        ctx->ws.off = mark;
        cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
        if (ctx->collect_timing) {
            for (auto &e : ev) ADAGIO_CUDA(cudaEventCreate(&e));
            ADAGIO_CUDA(cudaEventRecord(ev[0], st));
        }
        CertJob job;
        job.X = X;
        job.ldx = ldx;
        job.Y = Y;
        job.ldy = ldy;
        job.n = n;
        job.d = d;
        job.m = m;
        job.opt = opt;
        cert_job_setup(ctx, job, ctx->qbuf, ctx->qbuf_cap);
        PrepMat px;
        if (px_ready) {
            job.px = px_ready;
        } else {
            // X's prep reports a non-finite input through the job's flag word
            ADAGIO_CUDA(cudaMemsetAsync(job.flags, 0, sizeof(unsigned), st));
            cert_prepare_x(ctx, X, ldx, n, d, opt.precision, px, job.flags, st);
            job.px = &px;
            job.clear_flags = false;
        }
        cert_job_enqueue(ctx, job, st, ctx->collect_timing ? ev : nullptr);
        if (ctx->collect_timing) ADAGIO_CUDA(cudaEventRecord(ev[3], st));
        CertDevResult *h =
            reinterpret_cast<CertDevResult *>(host_stage(ctx, sizeof(CertDevResult) + 64));
        ADAGIO_CUDA(cudaMemcpyAsync(h, job.dres, sizeof(CertDevResult), cudaMemcpyDeviceToHost, st));
        ADAGIO_CUDA(cudaStreamSynchronize(st));
        adagio_cert_stats &cs = ctx->last_stats;
        cs.prep_ms = cs.tile_ms = cs.recompute_ms = -1.0;
        if (ctx->collect_timing) {
            float ms[3] = {0.0f, 0.0f, 0.0f};
            for (int q = 0; q < 3; ++q) cudaEventElapsedTime(&ms[q], ev[q], ev[q + 1]);
            cs.prep_ms = ms[0];
            cs.tile_ms = ms[1];
            cs.recompute_ms = ms[2];
            for (auto &e : ev) cudaEventDestroy(e);
        }
        cs.queued = h->qlen;
        cs.grid = job.nparts;
        const int64_t T = pad_rows(n) / kTileRows;
        cs.tiles = T * (T + 1) / 2;
        const int rc = cert_job_collect(job, *h, out, stopped, part_out);
        if (rc == ADAGIO_E_QUEUE_OVERFLOW) {
            const unsigned long long need = h->qlen;
            if (attempt == 0 && !ctx->qbuf_fixed) {
                cert_ensure_queue(ctx, std::min<unsigned long long>(pairs, need + need / 8 + 1024));
                continue;
            }
            fail(ADAGIO_E_QUEUE_OVERFLOW, "recompute queue overflow (%llu pairs > capacity %llu)",
                 need, job.qcap);
        }
        ctx->ws.off = mark;
        return ADAGIO_OK;
    }
    return ADAGIO_E_QUEUE_OVERFLOW;
}

void tile_coords(adagio_ctx *ctx, int precision, int64_t n, long long t, int *I, int *J) {
    const int T = (int)(pad_rows(n) / kTileRows);
    if (precision == ADAGIO_PREC_FP32) {
        // row-major upper triangle (the SIMT kernel's order)
        int i = 0;
        long long off = 0;
        while (i < T && off + (T - i) <= t) off += T - i++;
        *I = i;
        *J = i + (int)(t - off);
    } else {
        tc_tile_coords(ctx, n, t, I, J);
    }
}

}  // namespace adagio
