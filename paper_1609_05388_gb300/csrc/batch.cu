// Batched fit: many independent data sets of uneven n and d fitted in
// lock-step rounds.  Each instance goes through exactly the computation of
// the single fit (fit.cu): randomized PCA (pca.cu), the search of search.cuh,
// and per probe the JL rows, A = [P ; S (I - P^T P)] (Algorithm 1), Y = X A^T
// and the exhaustive certificate (Eq. 2, Eq. 3).  The host decisions of all
// instances -- PCA convergence tests and probe verdicts -- are taken together
// once per round, after one synchronisation:
//
//   round:  fork one stream per instance from an internal main stream;
//           enqueue each unfinished instance's next piece (subspace
//           iterations up to the next convergence test, or one probe);
//           join; optionally capture all of it as one CUDA graph; run; sync.
//
// Everything a round touches is reserved before the first round (workspace,
// recompute queues, pinned result slots, tile schedules, kernel attributes),
// so a round enqueues device work only and can be captured.
#include "internal.cuh"
#include "api_guard.cuh"
#include "cert.cuh"
#include "fit.cuh"
#include "jl.cuh"
#include "linalg.cuh"
#include "pca.cuh"
#include "search.cuh"
#include "tcgemm.cuh"

#include <algorithm>
#include <chrono>
#include <cstring>
#include <vector>

namespace adagio {
namespace {

constexpr int kMaxStreams = 64;
constexpr int kMaxCount = 4096;

enum class Wait { None, Init, Pca, Cert };

struct Inst {
    adagio_instance *pub = nullptr;
    cudaStream_t st = nullptr;
    int sidx = 0;
    bool search = false;
    int cap = 0, s_cap = 0, k_cap = 0, fixed_s = -1;
    PCA pca;
    float *S = nullptr, *A = nullptr, *Abest = nullptr, *T = nullptr, *Y = nullptr;
    EmbedPlanes ep;                  // X split once for every probe's embedding
    float *feats = nullptr;
    PrepMat px;
    unsigned *xflags = nullptr;
    unsigned *hx = nullptr;          // pinned: X's non-finite flag
    CertJob job;
    CertDevResult *hres = nullptr;   // pinned: the certificate's device result
    unsigned long long qcap = 0;
    Search se;
    Wait wait = Wait::None;
    bool predicting = false;         // PCA up to the predictor's 64 directions
    bool final_probe = false;        // the full certificate at the cap
    bool feats_pending = false;      // search over; PCA up to 64 directions for the features
    int r = 0;
    int retried_r = 0;
    bool done = false;
    int best_r = -1, best_s = 0;
    adagio_cert best_cert{};
    int probes = 0, full = 0;

    int split_s(int rr) const { return fixed_s >= 0 ? std::min(fixed_s, rr) : rr / 2; }
    unsigned long long pairs() const {
        return (unsigned long long)pub->n * (unsigned long long)(pub->n - 1) / 2;
    }
};

// Ends a capture that an exception interrupted, so the stream stays usable.
struct CaptureGuard {
    cudaStream_t st = nullptr;
    bool active = false;
    ~CaptureGuard() {
        if (active) {
            cudaGraph_t g = nullptr;
            cudaStreamEndCapture(st, &g);
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
        }
    }
};

void ensure_streams(adagio_ctx *ctx, int want) {
    while ((int)ctx->batch_streams.size() < want) {
        cudaStream_t s = nullptr;
        ADAGIO_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
        ctx->batch_streams.push_back(s);
    }
}

void *batch_host(adagio_ctx *ctx, size_t bytes) {
    if (bytes > ctx->batch_host_bytes) {
        if (ctx->batch_host) cudaFreeHost(ctx->batch_host);
        ctx->batch_host = nullptr;
        ctx->batch_host_bytes = 0;
        ADAGIO_CUDA(cudaMallocHost(&ctx->batch_host, bytes));
        ctx->batch_host_bytes = bytes;
    }
    return ctx->batch_host;
}

}  // namespace

int fit_batched(adagio_ctx *ctx, int count, adagio_instance *pub, const adagio_fit_opts &o,
                int flags, cudaStream_t user) {
    using clk = std::chrono::steady_clock;
    const auto t0 = clk::now();
    const bool tc = o.precision != ADAGIO_PREC_FP32;
    const bool graph = (flags & ADAGIO_BATCH_GRAPH) != 0;
    std::vector<Inst> in((size_t)count);

    // sizes, workspace and queue reservations --------------------------------
    size_t ws_fixed = 0, ws_round = 0;
    unsigned long long qtotal = 0;
    for (int i = 0; i < count; ++i) {
        Inst &I = in[i];
        adagio_instance &p = pub[i];
        I.pub = &p;
        I.search = p.eps > 0.0;
        I.fixed_s = o.s;
        const int d = p.d;
        if (I.search) {
            I.cap = std::min(p.m_cap, d);
            I.s_cap = o.s >= 0 ? std::min(o.s, I.cap) : I.cap / 2;
            I.k_cap = o.s >= 0 ? I.cap : I.cap - I.cap / 2;
            if (o.use_predictor || p.feats) I.s_cap = std::max(I.s_cap, std::min(64, d));
        } else {
            I.cap = p.m;
            I.s_cap = o.s >= 0 ? o.s : p.m / 2;
            I.k_cap = p.m - I.s_cap;
            if (p.feats) I.s_cap = std::max(I.s_cap, std::min(64, d));
        }
        ws_fixed += pca_bytes(ctx, p.n, d, I.s_cap, o.oversample, o.precision != ADAGIO_PREC_FP32);
        ws_fixed += align_up((size_t)std::max(I.k_cap, 1) * d * sizeof(float), 256);
        ws_fixed += 2 * align_up((size_t)std::max(I.cap, 1) * d * sizeof(float), 256);
        ws_fixed += align_up((size_t)std::max(I.k_cap, 1) * std::max(I.s_cap, 1) * sizeof(float), 256);
        ws_fixed += align_up((size_t)p.n * emb_ld(I.cap) * sizeof(float), 256);
        ws_fixed += cert_prep_x_bytes(p.n, d, o.precision) + cert_job_bytes(ctx, p.n, I.cap, o.precision);
        ws_fixed += align_up(embed_planes_bytes(ctx, p.n, d, I.cap), 256);
        ws_fixed += 3 * 256 + align_up(68 * sizeof(float), 256);
        ws_round += prep_bytes(p.n, std::max(I.cap, 1), !tc, tc);
        // a batch re-reserves its queues on every call: start at 1/64 of the
        // pairs (above the typical 1 % that split-precision tiles queue)
        I.qcap = std::min<unsigned long long>(I.pairs(), std::max<unsigned long long>(I.pairs() / 64, 1ull << 16));
        qtotal += I.qcap;
    }
    ws_reserve(ctx, ws_fixed + ws_round + align_up((size_t)count * 68 * sizeof(float), 256) +
                        align_up((size_t)count * sizeof(int), 256) + 65536);
    cert_ensure_queue(ctx, qtotal);
    auto carve_queues = [&]() {
        unsigned long long off = 0;
        for (Inst &I : in) {
            I.job.queue = ctx->qbuf + off;
            I.job.qcap = I.qcap;
            off += I.qcap;
        }
    };

    // pinned result slots, streams, events, kernel attributes ----------------
    const size_t hslot = align_up(sizeof(CertDevResult), 64) + align_up(pca_host_bytes(), 64) + 64;
    char *hb = reinterpret_cast<char *>(batch_host(ctx, hslot * count + 64 + (size_t)count * sizeof(int)));
    const int nstreams = std::min(count, kMaxStreams);
    ensure_streams(ctx, nstreams + 1);
    cudaStream_t main = ctx->batch_streams[0];
    std::vector<cudaEvent_t> ev((size_t)nstreams + 2, nullptr);
    struct EventsGuard {
        std::vector<cudaEvent_t> &e;
        ~EventsGuard() {
            for (cudaEvent_t x : e)
                if (x) cudaEventDestroy(x);
        }
    } evg{ev};
    for (auto &e : ev) ADAGIO_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    cert_init();
    linalg_init();
    tc_gemm_init();
    for (int i = 0; i < count; ++i) {
        Inst &I = in[i];
        I.sidx = 1 + i % nstreams;
        I.st = ctx->batch_streams[I.sidx];
        I.hres = reinterpret_cast<CertDevResult *>(hb + hslot * i);
        I.pca.hbuf = hb + hslot * i + align_up(sizeof(CertDevResult), 64);
        I.hx = reinterpret_cast<unsigned *>(hb + hslot * i + align_up(sizeof(CertDevResult), 64) +
                                            align_up(pca_host_bytes(), 64));
        if (tc) tc_prepare(ctx, I.pub->n);
    }
    int *hpred = reinterpret_cast<int *>(hb + hslot * count + 64);
    float *feats_all = ws_array<float>(ctx, (size_t)count * 68);
    int *dpred = ws_array<int>(ctx, count);

    CertOptions copt_base;
    copt_base.precision = o.precision;
    auto copt_for = [&](const Inst &I) {
        CertOptions c = copt_base;
        const double eps = I.search ? I.pub->eps : 0.1;
        c.eps = eps;
        if (o.hist_hi > o.hist_lo) {
            c.lo = o.hist_lo;
            c.hi = o.hist_hi;
        } else {
            c.lo = 0.0;
            c.hi = I.search ? 2.0 * eps : 1.0;
        }
        return c;
    };

    // one round: fork, enqueue, join, (capture), run, synchronise ------------
    adagio_batch_stats bs{0, 0, 0, 0.0};
    auto run_round = [&](auto &&enqueue) {
        CaptureGuard cg;
        if (graph) {
            // a graph launched on `main` is ordered after main's work only: the
            // work the last host decisions enqueued on the instance streams
            // (PCA steps, copies of the best map) is joined into main first
            for (int s = 1; s <= nstreams; ++s) {
                ADAGIO_CUDA(cudaEventRecord(ev[s], ctx->batch_streams[s]));
                ADAGIO_CUDA(cudaStreamWaitEvent(main, ev[s], 0));
            }
            ADAGIO_CUDA(cudaStreamBeginCapture(main, cudaStreamCaptureModeRelaxed));
            cg.st = main;
            cg.active = true;
        }
        ADAGIO_CUDA(cudaEventRecord(ev[0], main));
        for (int s = 1; s <= nstreams; ++s)
            ADAGIO_CUDA(cudaStreamWaitEvent(ctx->batch_streams[s], ev[0], 0));
        enqueue();
        for (int s = 1; s <= nstreams; ++s) {
            ADAGIO_CUDA(cudaEventRecord(ev[s], ctx->batch_streams[s]));
            ADAGIO_CUDA(cudaStreamWaitEvent(main, ev[s], 0));
        }
        if (graph) {
            cudaGraph_t g = nullptr;
            cg.active = false;
            ADAGIO_CUDA(cudaStreamEndCapture(main, &g));
            cudaGraphExec_t ge = nullptr;
            cudaError_t e = cudaGraphInstantiate(&ge, g, 0);
            if (e == cudaSuccess) e = cudaGraphLaunch(ge, main);
            if (e == cudaSuccess) e = cudaStreamSynchronize(main);
            if (ge) cudaGraphExecDestroy(ge);
            cudaGraphDestroy(g);
            ADAGIO_CUDA(e);
            ++bs.graphs;
        } else {
            ADAGIO_CUDA(cudaStreamSynchronize(main));
        }
        ++bs.rounds;
    };

    // the batch waits for the caller's earlier work on `user`
    ADAGIO_CUDA(cudaEventRecord(ev[nstreams + 1], user));
    ADAGIO_CUDA(cudaStreamWaitEvent(main, ev[nstreams + 1], 0));

    // init round: covariance and first preparations, all carving ------------
    run_round([&]() {
        for (Inst &I : in) {
            const adagio_instance &p = *I.pub;
            I.pca.init_enqueue(ctx, p.X, p.n, p.d, p.ldx, I.s_cap, o.seed, o.max_iter, o.tol,
                               o.oversample, o.precision != ADAGIO_PREC_FP32, I.st);
            I.S = ws_array<float>(ctx, (size_t)std::max(I.k_cap, 1) * p.d);
            I.A = ws_array<float>(ctx, (size_t)std::max(I.cap, 1) * p.d);
            I.Abest = ws_array<float>(ctx, (size_t)std::max(I.cap, 1) * p.d);
            I.T = ws_array<float>(ctx, (size_t)std::max(I.k_cap, 1) * std::max(I.s_cap, 1));
            I.Y = ws_array<float>(ctx, (size_t)p.n * emb_ld(I.cap));
            embed_planes_init(ctx, p.X, p.n, p.d, p.ldx, I.cap, I.ep, I.st);
            I.xflags = ws_array<unsigned>(ctx, 1);
            ADAGIO_CUDA(cudaMemsetAsync(I.xflags, 0, sizeof(unsigned), I.st));
            cert_prepare_x(ctx, p.X, p.ldx, p.n, p.d, o.precision, I.px, I.xflags, I.st);
            ADAGIO_CUDA(cudaMemcpyAsync(I.hx, I.xflags, sizeof(unsigned), cudaMemcpyDeviceToHost, I.st));
            I.job.X = p.X;
            I.job.ldx = p.ldx;
            I.job.n = p.n;
            I.job.d = p.d;
            I.job.opt = copt_for(I);
            cert_job_setup(ctx, I.job, nullptr, 0);
            I.job.px = &I.px;
            I.feats = feats_all + (size_t)(&I - in.data()) * 68;
        }
        ADAGIO_CUDA(cudaMemsetAsync(feats_all, 0, (size_t)count * 68 * sizeof(float), main));
    });
    carve_queues();
    for (Inst &I : in) {
        I.pca.init_check();
        if (*I.hx & 1u) fail(ADAGIO_E_NONFINITE, "input holds NaN or Inf");
        if (I.search && o.use_predictor) {
            I.predicting = true;
        } else if (I.search) {
            I.se.begin(I.cap, 0, false);
        }
    }
    const size_t round_base = ctx->ws.off;

    // the dimension to probe next (0: none, the instance waits or is done)
    auto next_r = [&](Inst &I) -> int {
        if (I.done || I.predicting) return 0;
        if (!I.search || I.final_probe) return I.cap;
        return I.se.next();
    };

    auto enqueue_probe = [&](Inst &I, int r) {
        const adagio_instance &p = *I.pub;
        const int s = I.split_s(r), k = r - s;
        if (k > 0) jl_matrix(o.seed, k, p.d, o.jl_dist, I.S, p.d, I.st);
        assemble(I.pca.P, s, p.d, I.S, k, p.d, p.d, I.A, p.d, I.T, I.st);
        embed_planes_run(ctx, I.ep, I.A, r, p.d, I.Y, emb_ld(r), I.st);
        I.job.Y = I.Y;
        I.job.ldy = emb_ld(r);
        I.job.m = r;
        I.job.opt = copt_for(I);
        I.job.opt.stop_early = I.search && !I.final_probe;
        cert_job_enqueue(ctx, I.job, I.st);
        ADAGIO_CUDA(cudaMemcpyAsync(I.hres, I.job.dres, sizeof(CertDevResult), cudaMemcpyDeviceToHost,
                                    I.st));
        I.r = r;
        I.wait = Wait::Cert;
    };

    // the predictor's features of a finished instance, then it is done
    auto emit_feats = [&](Inst &I) {
        const adagio_instance &p = *I.pub;
        if (p.feats)
            spectrum_features(I.pca.theta, I.pca.s_done, I.pca.C, p.d, p.n, I.search ? p.eps : 0.0,
                              p.feats, I.st);
        I.feats_pending = false;
        I.done = true;
    };

    auto finish = [&](Inst &I, int r, int s, const adagio_cert &c, const float *Asrc, int status) {
        adagio_instance &p = *I.pub;
        ADAGIO_CUDA(cudaMemcpyAsync(p.A, Asrc, sizeof(float) * (size_t)r * p.d, cudaMemcpyDeviceToDevice,
                                    I.st));
        p.m_out = r;
        p.s_out = s;
        p.cert = c;
        p.status = status;
        p.probes = I.probes;
        p.full_certs = I.full;
        if (p.feats && I.pca.needs(std::min(64, p.d))) I.feats_pending = true;
        else emit_feats(I);
    };

    for (;;) {
        bool any = false, any_pca = false;
        for (Inst &I : in) any |= !I.done;
        if (!any) break;
        // predictor: one network call once every predicting instance has its
        // 64 leading directions
        bool pred_ready = o.use_predictor;
        bool any_pred = false;
        for (Inst &I : in) {
            if (!I.predicting) continue;
            any_pred = true;
            if (I.pca.needs(std::min(64, I.pub->d))) pred_ready = false;
        }
        if (any_pred && pred_ready) {
            for (Inst &I : in)
                if (I.predicting)
                    spectrum_features(I.pca.theta, I.pca.s_done, I.pca.C, I.pub->d, I.pub->n,
                                      I.pub->eps, I.feats, I.st);
            for (int s = 1; s <= nstreams; ++s) {
                ADAGIO_CUDA(cudaEventRecord(ev[s], ctx->batch_streams[s]));
                ADAGIO_CUDA(cudaStreamWaitEvent(main, ev[s], 0));
            }
            predict_many(ctx, feats_all, count, dpred, hpred, main);
            ADAGIO_CUDA(cudaStreamSynchronize(main));
            for (int i = 0; i < count; ++i) {
                Inst &I = in[i];
                if (!I.predicting) continue;
                I.predicting = false;
                I.se.begin(I.cap, std::max(1, std::min(hpred[i], I.cap)), true);
            }
        }
        ctx->ws.off = round_base;
        run_round([&]() {
            for (Inst &I : in) {
                if (I.done) continue;
                if (I.feats_pending) {
                    I.pca.advance(std::min(64, I.pub->d), I.st);
                    I.wait = Wait::Pca;
                    any_pca = true;
                    continue;
                }
                if (I.predicting) {
                    const int s_need = std::min(64, I.pub->d);
                    if (I.pca.needs(s_need)) {
                        I.pca.advance(s_need, I.st);
                        I.wait = Wait::Pca;
                        any_pca = true;
                    }
                    continue;
                }
                const int r = next_r(I);
                const int s_need = I.split_s(r);
                if (I.pca.needs(s_need)) {
                    I.pca.advance(s_need, I.st);
                    I.wait = Wait::Pca;
                    any_pca = true;
                } else {
                    enqueue_probe(I, r);
                }
            }
        });
        if (any_pca) ++bs.pca_rounds;
        // host decisions of the round
        bool grow = false;
        for (Inst &I : in) {
            const Wait w = I.wait;
            I.wait = Wait::None;
            if (w == Wait::Pca) {
                I.pca.resolve(I.st);
                if (I.feats_pending && !I.pca.needs(std::min(64, I.pub->d))) emit_feats(I);
                continue;
            }
            if (w != Wait::Cert) continue;
            adagio_cert c;
            bool stopped = false;
            const int rc = cert_job_collect(I.job, *I.hres, &c, &stopped);
            if (rc == ADAGIO_E_QUEUE_OVERFLOW) {
                if (I.retried_r == I.r)
                    fail(ADAGIO_E_QUEUE_OVERFLOW, "recompute queue overflow (%llu pairs > capacity %llu)",
                         I.hres->qlen, I.qcap);
                I.retried_r = I.r;
                const unsigned long long need = I.hres->qlen;
                I.qcap = std::min<unsigned long long>(I.pairs(), need + need / 4 + 1024);
                grow = true;
                continue;  // the same probe runs again next round
            }
            I.retried_r = 0;
            const int r = I.r;
            if (!I.search) {
                finish(I, r, I.split_s(r), c, I.A, ADAGIO_OK);
                continue;
            }
            if (I.final_probe) {
                finish(I, r, I.split_s(r), c, I.A, ADAGIO_E_NOT_CERTIFIABLE);
                continue;
            }
            ++I.probes;
            const bool ok = !stopped && c.max <= I.job.opt.eps;
            if (ok) {
                ++I.full;
                if (I.best_r < 0 || r < I.best_r) {
                    I.best_r = r;
                    I.best_s = I.split_s(r);
                    I.best_cert = c;
                    ADAGIO_CUDA(cudaMemcpyAsync(I.Abest, I.A, sizeof(float) * (size_t)r * I.pub->d,
                                                cudaMemcpyDeviceToDevice, I.st));
                }
            }
            I.se.record(ok);
            if (I.se.next() == 0) {
                if (I.best_r > 0) finish(I, I.best_r, I.best_s, I.best_cert, I.Abest, ADAGIO_OK);
                else I.final_probe = true;  // not certifiable: full certificate at the cap
            }
        }
        if (grow) {
            unsigned long long total = 0;
            for (Inst &I : in) total += I.qcap;
            cert_ensure_queue(ctx, total);
            carve_queues();
        }
    }
    // the caller's stream waits for the batch
    for (int s = 1; s <= nstreams; ++s) {
        ADAGIO_CUDA(cudaEventRecord(ev[s], ctx->batch_streams[s]));
        ADAGIO_CUDA(cudaStreamWaitEvent(user, ev[s], 0));
    }
    check_device_status(ctx, user);  // synchronises
    bs.total_ms = std::chrono::duration<double, std::milli>(clk::now() - t0).count();
    ctx->last_batch = bs;
    return ADAGIO_OK;
}

}  // namespace adagio

using namespace adagio;

extern "C" int adagio_fit_batched(adagio_ctx *ctx, int count, adagio_instance *inst,
                                  const adagio_fit_opts *opts, int flags, void *stream) {
    API_BEGIN(ctx)
    ADAGIO_REQUIRE(inst && opts, "null pointer argument");
    ADAGIO_REQUIRE(count >= 1 && count <= kMaxCount, "count must lie in [1, %d]", kMaxCount);
    ADAGIO_REQUIRE((flags & ~ADAGIO_BATCH_GRAPH) == 0, "unknown flags 0x%x", flags);
    const adagio_fit_opts &o = *opts;
    ADAGIO_REQUIRE(o.precision == ADAGIO_PREC_FP32 || o.precision == ADAGIO_PREC_FP16X3 ||
                       o.precision == ADAGIO_PREC_BF16X3,
                   "unknown precision %d", o.precision);
    ADAGIO_REQUIRE(o.jl_dist == ADAGIO_JL_RADEMACHER || o.jl_dist == ADAGIO_JL_GAUSSIAN, "unknown jl_dist");
    ADAGIO_REQUIRE(o.oversample >= 1 && o.max_iter >= 1, "oversample and max_iter must be >= 1");
    if (o.use_predictor)
        ADAGIO_REQUIRE(has_predictor(ctx), "use_predictor needs a predictor (adagio_mlp_load)");
    for (int i = 0; i < count; ++i) {
        const adagio_instance &p = inst[i];
        ADAGIO_REQUIRE(p.X && p.A, "instance %d: null pointer", i);
        ADAGIO_REQUIRE(p.n >= 2 && p.n < (1ll << 31) - 256 && p.d >= 1 && p.ldx >= p.d,
                       "instance %d: bad sizes n=%lld d=%d ldx=%lld", i, (long long)p.n, p.d,
                       (long long)p.ldx);
        ADAGIO_REQUIRE(is_device_ptr(p.X, ctx->device) && is_device_ptr(p.A, ctx->device),
                       "instance %d: X and A must be device pointers", i);
        if (p.eps > 0.0) {
            ADAGIO_REQUIRE(p.eps < 1.0, "instance %d: eps must lie in (0, 1)", i);
            ADAGIO_REQUIRE(p.m_cap >= 1, "instance %d: m_cap must be >= 1", i);
        } else {
            ADAGIO_REQUIRE(!o.use_predictor, "instance %d: use_predictor needs eps > 0", i);
            ADAGIO_REQUIRE(p.m >= 1 && p.m <= p.m_cap && p.m <= p.d,
                           "instance %d: m must lie in [1, min(m_cap, d)]", i);
            ADAGIO_REQUIRE(o.s <= p.m, "instance %d: s must be <= m", i);
        }
    }
    return fit_batched(ctx, count, inst, o, flags, (cudaStream_t)stream);
    API_END(ctx)
}
