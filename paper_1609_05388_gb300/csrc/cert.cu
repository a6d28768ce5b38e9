// Certificate orchestration (Eq. 2, Eq. 3): K0 prep of X and Y, K8 tile
// kernel (FP32 SIMT or tcgen05 split precision), K9 exact recompute of the
// flagged pairs, K10 finaliser, one device->host copy of the result.
#include "internal.cuh"
#include "cert.cuh"

#include <cmath>
#include <cstring>

namespace adagio {

// Initial capacity of the recompute queue: 1/1024 of the pairs (at least
// 2^20 entries); it grows to the observed need when a run overflows it.
static unsigned long long queue_capacity(unsigned long long pairs) {
    unsigned long long q = pairs / 1024;
    if (q < (1ull << 20)) q = 1ull << 20;
    if (q > pairs) q = pairs;
    return q;
}

static void ensure_queue(adagio_ctx *ctx, unsigned long long cap) {
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

static int tile_grid(adagio_ctx *ctx, int precision) {
    if (precision == ADAGIO_PREC_FP32) return ctx->num_sms;  // 1 CTA / SM (64 KB hist + regs)
    return cert_tc_grid(ctx);
}

static int recompute_grid(adagio_ctx *ctx) { return ctx->num_sms * 4; }

size_t certify_bytes(adagio_ctx *ctx, int64_t n, int d, int m, int precision) {
    const bool tc = precision != ADAGIO_PREC_FP32;
    const unsigned long long pairs = (unsigned long long)n * (n - 1) / 2;
    size_t b = prep_bytes(n, d, !tc, tc) + prep_bytes(n, m, !tc, tc);
    b += align_up(sizeof(CertPartial) * (tile_grid(ctx, precision) + recompute_grid(ctx)), 256);
    (void)pairs;
    b += 4096 + sizeof(CertDevResult);
    if (tc) b += align_up((size_t)((n + 127) / 128 * 128) * sizeof(float4), 256);
    return b;
}

int certify(adagio_ctx *ctx, const float *X, int64_t ldx, const float *Y, int64_t ldy, int64_t n,
            int d, int m, const CertOptions &opt, adagio_cert *out, cudaStream_t st,
            bool *stopped) {
    const bool tc = opt.precision != ADAGIO_PREC_FP32;
    const unsigned long long pairs = (unsigned long long)n * (unsigned long long)(n - 1) / 2;
    if (!ctx->qbuf_fixed) ensure_queue(ctx, queue_capacity(pairs));
    const size_t mark = ctx->ws.off;

    for (int attempt = 0; attempt < 2; ++attempt) {
        ctx->ws.off = mark;
        unsigned *flags = ws_array<unsigned>(ctx, 1);
        int *stop = ws_array<int>(ctx, 1);
        int *status = ws_array<int>(ctx, 1);
        unsigned long long *qcount = ws_array<unsigned long long>(ctx, 1);
        ADAGIO_CUDA(cudaMemsetAsync(flags, 0, sizeof(unsigned), st));
        ADAGIO_CUDA(cudaMemsetAsync(stop, 0, sizeof(int), st));
        ADAGIO_CUDA(cudaMemsetAsync(status, 0, sizeof(int), st));
        ADAGIO_CUDA(cudaMemsetAsync(qcount, 0, sizeof(unsigned long long), st));

        cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
        if (ctx->collect_timing) {
            for (auto &e : ev) ADAGIO_CUDA(cudaEventCreate(&e));
            ADAGIO_CUDA(cudaEventRecord(ev[0], st));
        }
        PrepMat px, py;
        prep_matrix(ctx, X, n, d, ldx, opt.precision, !tc, tc, px, flags, st);
        prep_matrix(ctx, Y, n, m, ldy, opt.precision, !tc, tc, py, flags, st);

        CertLaunch L;
        L.ctx = ctx;
        L.x = &px;
        L.y = &py;
        L.cc.lo = (float)opt.lo;
        L.cc.hi = (float)opt.hi;
        L.cc.w = (float)((opt.hi - opt.lo) / kBins);
        L.cc.inv_w = (float)(kBins / (opt.hi - opt.lo));
        L.cc.eps = (float)opt.eps;
        L.cc.c_r = 8.0f * 5.9604645e-08f;
        L.cc.lo_is_floor = opt.lo <= 0.0;
        L.grid = tile_grid(ctx, opt.precision);
        L.partials = ws_array<CertPartial>(ctx, L.grid);
        const int rgrid = recompute_grid(ctx);
        CertPartial *rparts = ws_array<CertPartial>(ctx, rgrid);
        const unsigned long long qcap = ctx->qbuf_cap;
        L.queue = ctx->qbuf;
        L.qcount = qcount;
        L.qcap = qcap;
        L.stop_flag = opt.stop_early ? stop : nullptr;
        L.status = status;
        L.dump = opt.dump;
        L.dump_tiles = opt.dump_tiles;
        CertDevResult *dres = ws_array<CertDevResult>(ctx, 1);
        if (tc) L.rs_xy = ws_array<float4>(ctx, (size_t)px.n_pad);

        if (ctx->collect_timing) ADAGIO_CUDA(cudaEventRecord(ev[1], st));
        if (tc) {
            if (!launch_cert_tc(L, opt.precision, st))
                fail(ADAGIO_E_UNSUPPORTED, "tensor-core certificate does not support d=%d m=%d", d, m);
        } else {
            launch_cert_simt(L, st);
        }
        if (ctx->collect_timing) ADAGIO_CUDA(cudaEventRecord(ev[2], st));
        launch_recompute(X, ldx, d, Y, ldy, m, L.queue, qcount, qcap, L.cc, rparts, rgrid, st);
        launch_finalize(L.partials, L.grid, rparts, rgrid, qcount, flags, status, stop, dres, st);
        if (ctx->collect_timing) ADAGIO_CUDA(cudaEventRecord(ev[3], st));

        CertDevResult *h = reinterpret_cast<CertDevResult *>(host_stage(ctx, sizeof(CertDevResult) + 64));
        unsigned long long *hq = reinterpret_cast<unsigned long long *>(h + 1);
        ADAGIO_CUDA(cudaMemcpyAsync(h, dres, sizeof(CertDevResult), cudaMemcpyDeviceToHost, st));
        ADAGIO_CUDA(cudaMemcpyAsync(hq, qcount, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
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
        cs.queued = *hq;
        cs.grid = L.grid;
        {
            const int64_t T = px.n_pad / kTileRows;
            cs.tiles = T * (T + 1) / 2;
        }

        if (h->flags & 1u) fail(ADAGIO_E_NONFINITE, "input holds NaN or Inf");
        if (h->status != 0)
            fail(ADAGIO_E_TIMEOUT, "certificate kernel gave up a bounded wait (status %d)", h->status);
        if (*hq > qcap) {
            if (attempt == 0 && !ctx->qbuf_fixed) {
                ensure_queue(ctx, std::min<unsigned long long>(pairs, *hq + *hq / 8 + 1024));
                continue;
            }
            fail(ADAGIO_E_QUEUE_OVERFLOW, "recompute queue overflow (%llu pairs > capacity %llu)",
                 (unsigned long long)*hq, qcap);
        }
        if (stopped) *stopped = h->stopped != 0;
        if (!h->stopped) {
            if (h->fast_pairs + h->queued != pairs || h->queued != *hq ||
                h->recomputed + h->degenerate != *hq)
                fail(ADAGIO_E_CUDA,
                     "internal: pair accounting mismatch (fast %llu + queued %llu != %llu, recomputed %llu, degenerate %llu)",
                     h->fast_pairs, h->queued, pairs, h->recomputed, h->degenerate);
        }
        std::memset(out, 0, sizeof(*out));
        out->pairs = pairs;
        out->degenerate = h->degenerate;
        out->violations = h->violations;
        out->overflow = h->overflow;
        out->recomputed = h->recomputed + h->degenerate;
        std::memcpy(out->hist, h->hist, sizeof(out->hist));
        const unsigned long long good = pairs - h->degenerate;
        if (h->max >= 0.0f) {
            out->max = h->max;
            out->argmax_i = h->argmax_i;
            out->argmax_j = h->argmax_j;
        } else {
            out->max = 0.0;
            out->argmax_i = out->argmax_j = -1;
        }
        out->mean = good ? h->sum / (double)good : 0.0;
        out->max_err_bound = std::max((double)h->max_bound, 1e-12);
        out->mean_err_bound = good ? h->bound_sum / (double)good : 0.0;
        out->hist_lo = opt.lo;
        out->hist_hi = opt.hi;
        out->eps = opt.eps;
        ctx->ws.off = mark;
        return ADAGIO_OK;
    }
    return ADAGIO_E_QUEUE_OVERFLOW;
}

void tile_coords(int precision, int T, long long t, int *I, int *J) {
    if (precision == ADAGIO_PREC_FP32) {
        // row-major upper triangle (the SIMT kernel's order)
        int i = 0;
        long long off = 0;
        while (i < T && off + (T - i) <= t) off += T - i++;
        *I = i;
        *J = i + (int)(t - off);
    } else {
        tc_tile_coords(T, t, I, J);
    }
}

}  // namespace adagio
