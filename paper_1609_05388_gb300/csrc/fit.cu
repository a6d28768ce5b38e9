// Fit of the ADAGIO map (Algorithm 1 with the Sec. 4.1 split) and the
// certified search for the smallest target dimension (the question Table 3
// answers: how many dimensions reach distortion eps).
//
// Search: the state machine of search.cuh (doubling, then bisection).  Each
// probe builds A_r = [P_s ; S_k (I - P_s^T P_s)] with s = floor(r/2),
// k = ceil(r/2) (P_s is a prefix of the incrementally computed principal
// rows; S_k is a prefix of the counter-generated JL rows, rescaled), embeds
// Y = X A_r^T and certifies it.  A failing probe stops at the first certain
// violation.  Passing probes are complete certificates.
#include "internal.cuh"
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

void assemble(const float *P, int s, int64_t ldp, const float *S, int k, int64_t lds, int d,
              float *A, int64_t lda, float *T, cudaStream_t st) {
    if (s > 0) copy_rows(P, ldp, A, lda, s, d, st);
    if (k == 0) return;
    float *AS = A + (int64_t)s * lda;
    copy_rows(S, lds, AS, lda, k, d, st);
    if (s == 0) return;
    // T = S P^T (k x s);  A_S = S - T P
    gemm<float, float, float, float>(k, s, d, 1.0f, MatView<float>{S, lds, 1},
                                     MatView<float>{P, 1, ldp}, 0.0f, T, s, st);
    gemm<float, float, float, float>(k, d, s, -1.0f, MatView<float>{T, s, 1},
                                     MatView<float>{P, ldp, 1}, 1.0f, AS, lda, st);
}

size_t embed_planes_bytes(adagio_ctx *ctx, int64_t n, int d, int m_cap) {
    const size_t planes = align_up((size_t)n * pad64(d) * sizeof(uint16_t), 256);
    return 2 * planes + align_up((size_t)n * sizeof(float), 256) +
           embed_tc_bytes(ctx, n, std::max(m_cap, 1), d) + 256;
}

void embed_planes_init(adagio_ctx *ctx, const float *X, int64_t n, int d, int64_t ldx, int m_cap,
                       EmbedPlanes &ep, cudaStream_t st) {
    ADAGIO_REQUIRE(n <= (1ll << 30), "n must be at most 2^30");
    const int Kd = pad64(d);
    uint16_t *xh = ws_array<uint16_t>(ctx, (size_t)n * Kd), *xl = ws_array<uint16_t>(ctx, (size_t)n * Kd);
    float *xs = ws_array<float>(ctx, (size_t)n);
    split_rows(X, n, d, ldx, xh, xl, xs, st);
    ep.Xp.hi = xh;
    ep.Xp.lo = xl;
    ep.Xp.rows = n;
    ep.Xp.Kp = Kd;
    ep.Xp.scale = xs;
    ep.Xp.scale_stride = 1;
    ep.n = n;
    ep.d = d;
    ep.scratch = ws_alloc(ctx, embed_tc_bytes(ctx, n, std::max(m_cap, 1), d));
}

void embed_planes_run(adagio_ctx *ctx, const EmbedPlanes &ep, const float *A, int m, int64_t lda,
                      float *Y, int64_t ldy, cudaStream_t st) {
    embed_tc(ctx, ep.Xp, ep.n, nullptr, A, m, ep.d, lda, Y, ldy, ep.scratch, st);
}

size_t fit_bytes(adagio_ctx *ctx, int64_t n, int d, int s_cap, int k_cap, int m_cap, int precision,
                 int oversample) {
    size_t b = pca_bytes(ctx, n, d, s_cap, oversample, precision != ADAGIO_PREC_FP32);
    b += align_up((size_t)std::max(k_cap, 1) * d * sizeof(float), 256);          // S
    b += 2 * align_up((size_t)std::max(m_cap, 1) * d * sizeof(float), 256);      // A probe, A best
    b += align_up((size_t)std::max(k_cap, 1) * std::max(s_cap, 1) * sizeof(float), 256);  // T
    b += align_up((size_t)n * emb_ld(m_cap) * sizeof(float), 256);               // Y
    b += certify_bytes(ctx, n, d, std::max(m_cap, 1), precision);
    b += embed_planes_bytes(ctx, n, d, m_cap);
    return b + 65536;
}

namespace {

struct Prober {
    adagio_ctx *ctx;
    const float *X;
    int64_t ldx, n;
    int d;
    const adagio_fit_opts *o;
    PCA *pca;
    float *S, *A, *Abest, *T, *Y;
    EmbedPlanes ep;            // X split once for every probe's embedding
    cudaEvent_t prep_ready = nullptr;  // ep and px are ready (side stream)
    CertOptions copt;
    const PrepMat *px = nullptr;  // X prepared once for every probe's certificate
    int fixed_s;  // >= 0: every probe uses this many principal rows
    struct Rec {
        int r;
        bool ok;
        double max;
    };
    std::vector<Rec> probes;
    int best_r = -1, best_s = 0;
    adagio_cert best_cert{};
    int last_r = -1, last_s = 0;
    adagio_cert last_cert{};

    int split_s(int r) const { return fixed_s >= 0 ? std::min(fixed_s, r) : r / 2; }

    // builds A_r into A (m = r rows, ld d)
    void build(int r, cudaStream_t st) {
        const int s = split_s(r), k = r - s;
        if (s > 0) pca->extend(s, st);
        if (k > 0) jl_matrix(o->seed, k, d, o->jl_dist, S, d, st);
        assemble(pca->P, s, d, S, k, d, d, A, d, T, st);
    }

    void embed(int r, cudaStream_t st) {
        if (prep_ready) {
            ADAGIO_CUDA(cudaStreamWaitEvent(st, prep_ready, 0));
            prep_ready = nullptr;
        }
        embed_planes_run(ctx, ep, A, r, d, Y, emb_ld(r), st);
    }

    bool probe(int r, bool stop_early, cudaStream_t st) {
        build(r, st);
        embed(r, st);
        adagio_cert c;
        CertOptions co = copt;
        co.stop_early = stop_early;
        bool stopped = false;
        certify(ctx, X, ldx, Y, emb_ld(r), n, d, r, co, &c, st, &stopped, px);
        const bool ok = !stopped && c.max <= copt.eps;
        probes.push_back({r, ok, c.max});
        last_r = r;
        last_s = split_s(r);
        last_cert = c;
        if (ok && (best_r < 0 || r < best_r)) {
            best_r = r;
            best_s = split_s(r);
            best_cert = c;
            ADAGIO_CUDA(cudaMemcpyAsync(Abest, A, sizeof(float) * (size_t)r * d,
                                        cudaMemcpyDeviceToDevice, st));
        }
        return ok;
    }
};

}  // namespace

int fit_device(adagio_ctx *ctx, const float *X, int64_t n, int d, int64_t ldx,
               const adagio_fit_opts *o, float *A_out, int m_cap, int *m_out, int *s_out,
               adagio_cert *cert, cudaStream_t st, FitTrace *trace) {
    const bool search = o->eps > 0.0;
    int cap, s_cap, k_cap;
    if (search) {
        cap = std::min(m_cap, d);
        if (o->s >= 0) {
            s_cap = std::min(o->s, cap);
            k_cap = cap;
        } else {
            s_cap = cap / 2;
            k_cap = cap - cap / 2;
        }
    } else {
        cap = o->m;
        s_cap = o->s >= 0 ? o->s : o->m / 2;
        k_cap = o->m - s_cap;
    }
    if (search && o->use_predictor) s_cap = std::max(s_cap, std::min(64, d));
    const size_t mark = ctx->ws.off;
    using clk = std::chrono::steady_clock;
    const auto t_start = clk::now();
    double pca_ms = 0.0;
    PCA pca;
    pca.init(ctx, X, n, d, ldx, s_cap, o->seed, o->max_iter, o->tol, o->oversample,
             o->precision != ADAGIO_PREC_FP32, st);
    pca_ms += std::chrono::duration<double, std::milli>(clk::now() - t_start).count();
    pca.elapsed_ms = &pca_ms;
    Prober pr{};
    pr.ctx = ctx;
    pr.X = X;
    pr.ldx = ldx;
    pr.n = n;
    pr.d = d;
    pr.o = o;
    pr.pca = &pca;
    pr.S = ws_array<float>(ctx, (size_t)std::max(k_cap, 1) * d);
    pr.A = ws_array<float>(ctx, (size_t)std::max(cap, 1) * d);
    pr.Abest = ws_array<float>(ctx, (size_t)std::max(cap, 1) * d);
    pr.T = ws_array<float>(ctx, (size_t)std::max(k_cap, 1) * std::max(s_cap, 1));
    pr.Y = ws_array<float>(ctx, (size_t)n * emb_ld(cap));
    const double eps = search ? o->eps : 0.1;
    pr.copt.eps = eps;
    pr.copt.precision = o->precision;
    if (o->hist_hi > o->hist_lo) {
        pr.copt.lo = o->hist_lo;
        pr.copt.hi = o->hist_hi;
    } else {
        pr.copt.lo = 0.0;
        pr.copt.hi = search ? 2.0 * eps : 1.0;
    }
    pr.fixed_s = o->s;
    // The embedding's split planes of X and the certificate's preparation of
    // X do not depend on the PCA: a side stream computes them while the
    // PCA's chain of small kernels leaves most of the GPU idle.  The first
    // embedding waits for them; every exit waits for the side stream, so no
    // later call reuses the workspace under it.
    PrepMat px;
    cudaStream_t side = side_stream(ctx);
    struct SideJoin {
        cudaStream_t s;
        ~SideJoin() { cudaStreamSynchronize(s); }
    } side_join{side};
    ADAGIO_CUDA(cudaEventRecord(ctx->side_ev[0], st));
    ADAGIO_CUDA(cudaStreamWaitEvent(side, ctx->side_ev[0], 0));
    embed_planes_init(ctx, X, n, d, ldx, cap, pr.ep, side);
    {
        unsigned *xflags = ws_array<unsigned>(ctx, 1);
        ADAGIO_CUDA(cudaMemsetAsync(xflags, 0, sizeof(unsigned), side));
        cert_prepare_x(ctx, X, ldx, n, d, o->precision, px, xflags, side);
        pr.px = &px;  // X is finite: the PCA's preparation checked it
    }
    ADAGIO_CUDA(cudaEventRecord(ctx->side_ev[1], side));
    pr.prep_ready = ctx->side_ev[1];

    int status = ADAGIO_OK;
    int r_final, s_final;
    if (!search) {
        pr.build(cap, st);
        if (cert) {
            pr.embed(cap, st);
            certify(ctx, X, ldx, pr.Y, emb_ld(cap), n, d, cap, pr.copt, cert, st, nullptr, &px);
        }
        ADAGIO_CUDA(cudaMemcpyAsync(A_out, pr.A, sizeof(float) * (size_t)cap * d,
                                    cudaMemcpyDeviceToDevice, st));
        r_final = cap;
        s_final = pr.split_s(cap);
    } else {
        int start = (trace && trace->start_r > 0) ? std::min(trace->start_r, cap) : 0;
        bool verify_only = trace && trace->verify_only;
        if (o->use_predictor) {
            // spectrum features from this fit's own PCA, then the network's guess
            pca.extend(std::min(64, d), st);
            float *feats = ws_array<float>(ctx, 68);
            spectrum_features(pca.theta, pca.s_done, pca.C, d, n, o->eps, feats, st);
            start = std::max(1, std::min(predict_one(ctx, feats, st), cap));
            verify_only = true;
            ctx->last_fit.predicted_m = start;
        }
        Search se;
        se.begin(cap, start, verify_only);
        for (int r; (r = se.next()) > 0;) se.record(pr.probe(r, true, st));
        if (pr.best_r > 0) {
            r_final = pr.best_r;
            s_final = pr.best_s;
            if (cert) *cert = pr.best_cert;
            ADAGIO_CUDA(cudaMemcpyAsync(A_out, pr.Abest, sizeof(float) * (size_t)r_final * d,
                                        cudaMemcpyDeviceToDevice, st));
        } else {
            // not certifiable at the cap: return the map at the cap and its full certificate
            pr.build(cap, st);
            pr.embed(cap, st);
            adagio_cert c;
            certify(ctx, X, ldx, pr.Y, emb_ld(cap), n, d, cap, pr.copt, &c, st, nullptr, &px);
            if (cert) *cert = c;
            ADAGIO_CUDA(cudaMemcpyAsync(A_out, pr.A, sizeof(float) * (size_t)cap * d,
                                        cudaMemcpyDeviceToDevice, st));
            r_final = cap;
            s_final = pr.split_s(cap);
            status = ADAGIO_E_NOT_CERTIFIABLE;
        }
    }
    if (m_out) *m_out = r_final;
    if (s_out) *s_out = s_final;
    if (!(search && o->use_predictor)) ctx->last_fit.predicted_m = 0;
    ctx->last_fit.probes = (int)pr.probes.size();
    ctx->last_fit.full_certs = 0;
    for (const auto &q : pr.probes) ctx->last_fit.full_certs += q.ok ? 1 : 0;
    ctx->last_fit.pca_iterations = pca.iterations;
    ctx->last_fit.s_computed = pca.s_done;
    ctx->last_fit.pca_ms = pca_ms;
    if (trace) {
        trace->probes.clear();
        for (const auto &p : pr.probes) trace->probes.push_back({p.r, p.ok ? 1 : 0, p.max});
        trace->pca_iterations = pca.iterations;
        trace->s_computed = pca.s_done;
    }
    check_device_status(ctx, st);  // synchronises
    ctx->last_fit.total_ms = std::chrono::duration<double, std::milli>(clk::now() - t_start).count();
    ctx->ws.off = mark;
    return status;
}

}  // namespace adagio
