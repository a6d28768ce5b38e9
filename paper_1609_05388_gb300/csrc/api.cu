// C ABI entry points (include/adagio.h): argument checks, host/device staging
// and translation of internal failures into status codes.
#include "internal.cuh"
#include "cert.cuh"
#include "fit.cuh"
#include "jl.cuh"
#include "linalg.cuh"
#include "pca.cuh"
#include "tcgemm.cuh"
#include "api_guard.cuh"

#include <algorithm>
#include <cmath>
#include <vector>
#include <cstring>
#include <exception>

using namespace adagio;

static size_t staging_bytes(adagio_ctx *ctx, const void *p, int64_t rows, int cols) {
    return is_device_ptr(p, ctx->device) ? 0 : align_up((size_t)rows * cols * sizeof(float), 256);
}

static void check_hist(double eps, double &lo, double &hi) {
    ADAGIO_REQUIRE(std::isfinite(eps) && eps > 0.0 && eps < 1.0, "eps must lie in (0, 1), got %g", eps);
    if (!(hi > lo)) {
        lo = 0.0;
        hi = 2.0 * eps;
    }
    ADAGIO_REQUIRE(std::isfinite(lo) && std::isfinite(hi) && lo >= 0.0, "bad histogram range [%g, %g)",
                   lo, hi);
}

static void check_precision(int precision) {
    ADAGIO_REQUIRE(precision == ADAGIO_PREC_FP32 || precision == ADAGIO_PREC_FP16X3 ||
                       precision == ADAGIO_PREC_BF16X3,
                   "unknown precision %d", precision);
}

extern "C" {

int adagio_tile_kernel_for(adagio_ctx *ctx, int64_t n) {
    API_BEGIN(ctx)
    ADAGIO_REQUIRE(n >= 2, "n must be at least 2");
    return tc_variant(ctx, n);
    API_END(ctx)
}

int adagio_distortion(adagio_ctx *ctx, const float *X, int64_t n, int d, int64_t ldx,
                      const float *Y, int m, int64_t ldy, double eps, double hist_lo,
                      double hist_hi, int precision, adagio_cert *out, void *stream) {
    API_BEGIN(ctx)
    ADAGIO_REQUIRE(X && Y && out, "null pointer argument");
    ADAGIO_REQUIRE(n >= 2 && n < (1ll << 31) - 256, "n = %lld out of range [2, 2^31)", (long long)n);
    ADAGIO_REQUIRE(d >= 1 && m >= 1, "d and m must be >= 1 (d=%d, m=%d)", d, m);
    ADAGIO_REQUIRE(ldx >= d && ldy >= m, "leading dimensions too small");
    check_precision(precision);
    check_hist(eps, hist_lo, hist_hi);
    cudaStream_t st = (cudaStream_t)stream;
    // rows staged 16-byte aligned: the recompute reads them with 16-byte loads
    size_t need = stage_aligned_bytes(ctx, X, n, d, ldx) + stage_aligned_bytes(ctx, Y, n, m, ldy) +
                  certify_bytes(ctx, n, d, m, precision) + 1024;
    ws_reserve(ctx, need);
    int64_t lx, ly;
    const float *dX = stage_aligned(ctx, X, n, d, ldx, &lx, st);
    const float *dY = stage_aligned(ctx, Y, n, m, ldy, &ly, st);
    CertOptions co;
    co.eps = eps;
    co.lo = hist_lo;
    co.hi = hist_hi;
    co.precision = precision;
    return certify(ctx, dX, lx, dY, ly, n, d, m, co, out, st);
    API_END(ctx)
}

int adagio_distortion_shard(adagio_ctx *ctx, const float *X, int64_t n, int d, int64_t ldx,
                            const float *Y, int m, int64_t ldy, double eps, double hist_lo,
                            double hist_hi, int precision, int shard, int nshards,
                            adagio_cert_part *out, void *stream) {
    API_BEGIN(ctx)
    ADAGIO_REQUIRE(X && Y && out, "null pointer argument");
    ADAGIO_REQUIRE(n >= 2 && n < (1ll << 31) - 256, "n = %lld out of range [2, 2^31)", (long long)n);
    ADAGIO_REQUIRE(d >= 1 && m >= 1, "d and m must be >= 1 (d=%d, m=%d)", d, m);
    ADAGIO_REQUIRE(ldx >= d && ldy >= m, "leading dimensions too small");
    const long long T = pad_rows(n) / kTileRows, ntp = T * (T + 1) / 2;
    ADAGIO_REQUIRE(nshards >= 1 && nshards <= ntp && shard >= 0 && shard < nshards,
                   "shard %d of %d: need 0 <= shard < nshards <= %lld (the tiles of n = %lld)", shard,
                   nshards, ntp, (long long)n);
    check_precision(precision);
    check_hist(eps, hist_lo, hist_hi);
    cudaStream_t st = (cudaStream_t)stream;
    size_t need = stage_aligned_bytes(ctx, X, n, d, ldx) + stage_aligned_bytes(ctx, Y, n, m, ldy) +
                  certify_bytes(ctx, n, d, m, precision) + align_up((size_t)ntp * 4, 256) + 1024;
    ws_reserve(ctx, need);
    int64_t lx, ly;
    const float *dX = stage_aligned(ctx, X, n, d, ldx, &lx, st);
    const float *dY = stage_aligned(ctx, Y, n, m, ldy, &ly, st);
    CertOptions co;
    co.eps = eps;
    co.lo = hist_lo;
    co.hi = hist_hi;
    co.precision = precision;
    co.shard = shard;
    co.nshards = nshards;
    return certify(ctx, dX, lx, dY, ly, n, d, m, co, nullptr, st, nullptr, nullptr, out);
    API_END(ctx)
}

int adagio_cert_merge(const adagio_cert_part *parts, int count, adagio_cert *out) {
    if (!parts || !out || count < 1) return ADAGIO_E_INVALID_ARG;
    std::vector<int> seen(count, 0);
    for (int q = 0; q < count; ++q) {
        const adagio_cert_part &p = parts[q];
        if (p.nshards != count || p.shard < 0 || p.shard >= count || seen[p.shard]++) return ADAGIO_E_INVALID_ARG;
        if (p.eps != parts[0].eps || p.hist_lo != parts[0].hist_lo || p.hist_hi != parts[0].hist_hi)
            return ADAGIO_E_INVALID_ARG;
    }
    // parts in shard order, so the sums do not depend on the order given
    std::vector<adagio_cert_part> ordered(count);
    for (int q = 0; q < count; ++q) ordered[parts[q].shard] = parts[q];
    cert_from_parts(ordered.data(), count, out);
    return ADAGIO_OK;
}

int adagio_debug_tile_bounds(adagio_ctx *ctx, const float *X, int64_t n, int d, int64_t ldx,
                             const float *Y, int m, int64_t ldy, int precision, int64_t tiles,
                             int64_t stride, float *out, int *tile_ij, void *stream) {
    API_BEGIN(ctx)
    ADAGIO_REQUIRE(X && Y && out && tile_ij, "null pointer argument");
    ADAGIO_REQUIRE(n >= 2 && n < (1ll << 31) - 256 && d >= 1 && m >= 1 && ldx >= d && ldy >= m,
                   "bad sizes");
    check_precision(precision);
    const int T = (int)(pad_rows(n) / 128);  // the tile grid the kernels visit
    const long long ntp = (long long)T * (T + 1) / 2;
    ADAGIO_REQUIRE(stride >= 1 && tiles >= 1 && (tiles - 1) * stride < ntp,
                   "need stride >= 1 and tiles >= 1 with (tiles - 1) * stride < %lld", ntp);
    cudaStream_t st = (cudaStream_t)stream;
    const bool out_dev = is_device_ptr(out, ctx->device);
    const size_t dump_bytes = (size_t)tiles * 128 * 128 * 4 * sizeof(float);
    size_t need = staging_bytes(ctx, X, n, d) + staging_bytes(ctx, Y, n, m) +
                  certify_bytes(ctx, n, d, m, precision) + (out_dev ? 0 : align_up(dump_bytes, 256));
    ws_reserve(ctx, need);
    int64_t lx, ly;
    const float *dX = stage_input(ctx, X, n, d, ldx, &lx, st);
    const float *dY = stage_input(ctx, Y, n, m, ldy, &ly, st);
    float *dump = out_dev ? out : reinterpret_cast<float *>(ws_alloc(ctx, dump_bytes));
    CertOptions co;
    co.eps = 0.5;
    co.lo = 0.0;
    co.hi = 1.0;
    co.precision = precision;
    co.dump = dump;
    co.dump_tiles = tiles;
    co.dump_stride = stride;
    adagio_cert c;
    const int rc = certify(ctx, dX, lx, dY, ly, n, d, m, co, &c, st);
    if (!out_dev) {
        ADAGIO_CUDA(cudaMemcpyAsync(out, dump, dump_bytes, cudaMemcpyDeviceToHost, st));
        ADAGIO_CUDA(cudaStreamSynchronize(st));
    }
    for (long long t = 0; t < tiles; ++t)
        tile_coords(ctx, precision, n, t * stride, &tile_ij[2 * t], &tile_ij[2 * t + 1]);
    return rc;
    API_END(ctx)
}

int adagio_embed(adagio_ctx *ctx, const float *A, int m, int d, int64_t lda, const float *X,
                 int64_t n, int64_t ldx, float *Y, int64_t ldy, void *stream) {
    API_BEGIN(ctx)
    ADAGIO_REQUIRE(A && X && Y, "null pointer argument");
    ADAGIO_REQUIRE(n >= 1 && d >= 1 && m >= 1, "sizes must be positive");
    ADAGIO_REQUIRE(lda >= d && ldx >= d && ldy >= m, "leading dimensions too small");
    cudaStream_t st = (cudaStream_t)stream;
    ADAGIO_REQUIRE(n <= (1ll << 30), "n must be at most 2^30");
    const bool y_dev = is_device_ptr(Y, ctx->device);
    // tensor cores: per-row FP16 split planes of X and A, three products
    size_t need = staging_bytes(ctx, A, m, d) + staging_bytes(ctx, X, n, d) +
                  (y_dev ? 0 : align_up((size_t)n * m * sizeof(float), 256)) +
                  embed_planes_bytes(ctx, n, d, m) + 4096;
    ws_reserve(ctx, need);
    int64_t la, lx;
    const float *dA = stage_input(ctx, A, m, d, lda, &la, st);
    const float *dX = stage_input(ctx, X, n, d, ldx, &lx, st);
    float *dY = y_dev ? Y : ws_array<float>(ctx, (size_t)n * m);
    const int64_t ly = y_dev ? ldy : m;
    EmbedPlanes ep;
    embed_planes_init(ctx, dX, n, d, lx, m, ep, st);
    embed_planes_run(ctx, ep, dA, m, la, dY, ly, st);
    if (!y_dev) {
        ADAGIO_CUDA(cudaMemcpy2DAsync(Y, (size_t)ldy * sizeof(float), dY, (size_t)m * sizeof(float),
                                      (size_t)m * sizeof(float), (size_t)n, cudaMemcpyDeviceToHost, st));
        check_device_status(ctx, st);
    }
    return ADAGIO_OK;
    API_END(ctx)
}

int adagio_jl_matrix(adagio_ctx *ctx, uint64_t seed, int k, int d, int jl_dist, float *S,
                     int64_t lds, void *stream) {
    API_BEGIN(ctx)
    ADAGIO_REQUIRE(S, "null pointer argument");
    ADAGIO_REQUIRE(k >= 1 && d >= 1 && lds >= d, "bad sizes k=%d d=%d lds=%lld", k, d, (long long)lds);
    ADAGIO_REQUIRE(jl_dist == ADAGIO_JL_RADEMACHER || jl_dist == ADAGIO_JL_GAUSSIAN, "unknown jl_dist %d",
                   jl_dist);
    cudaStream_t st = (cudaStream_t)stream;
    const bool dev = is_device_ptr(S, ctx->device);
    ws_reserve(ctx, dev ? 4096 : align_up((size_t)k * d * sizeof(float), 256) + 4096);
    float *dS = dev ? S : ws_array<float>(ctx, (size_t)k * d);
    jl_matrix(seed, k, d, jl_dist, dS, dev ? lds : d, st);
    if (!dev) {
        ADAGIO_CUDA(cudaMemcpy2DAsync(S, (size_t)lds * sizeof(float), dS, (size_t)d * sizeof(float),
                                      (size_t)d * sizeof(float), (size_t)k, cudaMemcpyDeviceToHost, st));
        ADAGIO_CUDA(cudaStreamSynchronize(st));
    }
    return ADAGIO_OK;
    API_END(ctx)
}

int adagio_pca(adagio_ctx *ctx, const float *X, int64_t n, int d, int64_t ldx, int s,
               const adagio_fit_opts *opts, float *P, int64_t ldp, double *theta, void *stream) {
    API_BEGIN(ctx)
    ADAGIO_REQUIRE(X && P, "null pointer argument");
    ADAGIO_REQUIRE(n >= 2 && d >= 1 && ldx >= d, "bad sizes");
    ADAGIO_REQUIRE(s >= 1 && s <= d && ldp >= d, "s must lie in [1, d] (s=%d, d=%d)", s, d);
    adagio_fit_opts o;
    if (opts) o = *opts; else adagio_default_fit_opts(&o);
    cudaStream_t st = (cudaStream_t)stream;
    ws_reserve(ctx, staging_bytes(ctx, X, n, d) + pca_bytes(ctx, n, d, s, o.oversample, o.precision != ADAGIO_PREC_FP32) + 4096);
    int64_t lx;
    const float *dX = stage_input(ctx, X, n, d, ldx, &lx, st);
    PCA pca;
    pca.init(ctx, dX, n, d, lx, s, o.seed, o.max_iter, o.tol, o.oversample,
             o.precision != ADAGIO_PREC_FP32, st);
    pca.extend(s, st);
    if (is_device_ptr(P, ctx->device)) {
        copy_rows(pca.P, d, P, ldp, s, d, st);
    } else {
        ADAGIO_CUDA(cudaMemcpy2DAsync(P, (size_t)ldp * sizeof(float), pca.P, (size_t)d * sizeof(float),
                                      (size_t)d * sizeof(float), (size_t)s, cudaMemcpyDeviceToHost, st));
    }
    if (theta)
        ADAGIO_CUDA(cudaMemcpyAsync(theta, pca.theta, sizeof(double) * s, cudaMemcpyDefault, st));
    ADAGIO_CUDA(cudaStreamSynchronize(st));
    return ADAGIO_OK;
    API_END(ctx)
}

int adagio_assemble(adagio_ctx *ctx, const float *P, int s, int64_t ldp, const float *S, int k,
                    int64_t lds, int d, float *A, int64_t lda, void *stream) {
    API_BEGIN(ctx)
    ADAGIO_REQUIRE(A && (s == 0 || P) && (k == 0 || S), "null pointer argument");
    ADAGIO_REQUIRE(s >= 0 && k >= 0 && s + k >= 1 && d >= 1, "bad sizes s=%d k=%d d=%d", s, k, d);
    ADAGIO_REQUIRE((s == 0 || ldp >= d) && (k == 0 || lds >= d) && lda >= d, "leading dimensions too small");
    cudaStream_t st = (cudaStream_t)stream;
    const bool a_dev = is_device_ptr(A, ctx->device);
    size_t need = (s ? staging_bytes(ctx, P, s, d) : 0) + (k ? staging_bytes(ctx, S, k, d) : 0) +
                  align_up((size_t)std::max(k * s, 1) * sizeof(float), 256) +
                  (a_dev ? 0 : align_up((size_t)(s + k) * d * sizeof(float), 256)) + 4096;
    ws_reserve(ctx, need);
    int64_t lp = d, ls = d;
    const float *dP = s ? stage_input(ctx, P, s, d, ldp, &lp, st) : nullptr;
    const float *dS = k ? stage_input(ctx, S, k, d, lds, &ls, st) : nullptr;
    float *T = ws_array<float>(ctx, (size_t)std::max(k * s, 1));
    float *dA = a_dev ? A : ws_array<float>(ctx, (size_t)(s + k) * d);
    const int64_t la = a_dev ? lda : d;
    assemble(dP, s, lp, dS, k, ls, d, dA, la, T, st);
    if (!a_dev) {
        ADAGIO_CUDA(cudaMemcpy2DAsync(A, (size_t)lda * sizeof(float), dA, (size_t)d * sizeof(float),
                                      (size_t)d * sizeof(float), (size_t)(s + k), cudaMemcpyDeviceToHost, st));
        ADAGIO_CUDA(cudaStreamSynchronize(st));
    }
    return ADAGIO_OK;
    API_END(ctx)
}

}  // extern "C"

namespace adagio {

int fit_entry(adagio_ctx *ctx, const float *X, int64_t n, int d, int64_t ldx,
              const adagio_fit_opts *opts, float *A, int m_cap, int *m_out, int *s_out,
              adagio_cert *cert, void *stream, FitTrace *trace) {
    API_BEGIN(ctx)
    ADAGIO_REQUIRE(X && opts && A, "null pointer argument");
    ADAGIO_REQUIRE(n >= 2 && n < (1ll << 31) - 256 && d >= 1 && ldx >= d, "bad sizes n=%lld d=%d",
                   (long long)n, d);
    const adagio_fit_opts &o = *opts;
    check_precision(o.precision);
    ADAGIO_REQUIRE(o.jl_dist == ADAGIO_JL_RADEMACHER || o.jl_dist == ADAGIO_JL_GAUSSIAN, "unknown jl_dist");
    ADAGIO_REQUIRE(o.oversample >= 1 && o.max_iter >= 1, "oversample and max_iter must be >= 1");
    int s_cap, k_cap, cap;
    if (o.eps > 0.0) {
        ADAGIO_REQUIRE(o.eps < 1.0, "eps must lie in (0, 1)");
        ADAGIO_REQUIRE(m_cap >= 1, "m_cap must be >= 1");
        cap = std::min(m_cap, d);
        s_cap = o.s >= 0 ? std::min(o.s, cap) : cap / 2;
        k_cap = o.s >= 0 ? cap : cap - cap / 2;
    } else {
        ADAGIO_REQUIRE(o.m >= 1 && o.m <= m_cap, "m must lie in [1, m_cap] (m=%d, m_cap=%d)", o.m, m_cap);
        ADAGIO_REQUIRE(o.s <= o.m && o.s <= d, "s must be <= m and <= d");
        cap = o.m;
        s_cap = o.s >= 0 ? o.s : o.m / 2;
        k_cap = o.m - s_cap;
        ADAGIO_REQUIRE(s_cap <= d, "s must be <= d");
    }
    if (o.use_predictor) {
        ADAGIO_REQUIRE(o.eps > 0.0, "use_predictor needs eps > 0");
        ADAGIO_REQUIRE(has_predictor(ctx), "use_predictor needs a predictor (adagio_mlp_load)");
        s_cap = std::max(s_cap, std::min(64, d));
    }
    cudaStream_t st = (cudaStream_t)stream;
    const bool a_dev = is_device_ptr(A, ctx->device);
    size_t need = staging_bytes(ctx, X, n, d) +
                  fit_bytes(ctx, n, d, s_cap, k_cap, cap, o.precision, o.oversample) +
                  (a_dev ? 0 : align_up((size_t)cap * d * sizeof(float), 256)) + 4096;
    ws_reserve(ctx, need);
    int64_t lx;
    const float *dX = stage_input(ctx, X, n, d, ldx, &lx, st);
    float *dA = a_dev ? A : ws_array<float>(ctx, (size_t)cap * d);
    int m = 0, s = 0;
    const int rc = fit_device(ctx, dX, n, d, lx, &o, dA, m_cap, &m, &s, cert, st, trace);
    if (!a_dev) {
        ADAGIO_CUDA(cudaMemcpyAsync(A, dA, sizeof(float) * (size_t)m * d, cudaMemcpyDeviceToHost, st));
        ADAGIO_CUDA(cudaStreamSynchronize(st));
    }
    if (m_out) *m_out = m;
    if (s_out) *s_out = s;
    if (rc == ADAGIO_E_NOT_CERTIFIABLE)
        ctx->last_error = "eps not reached at m_cap; the map at m_cap and its certificate are returned";
    return rc;
    API_END(ctx)
}

}  // namespace adagio

extern "C" {

int adagio_fit(adagio_ctx *ctx, const float *X, int64_t n, int d, int64_t ldx,
               const adagio_fit_opts *opts, float *A, int m_cap, int *m_out, int *s_out,
               adagio_cert *cert, void *stream) {
    return fit_entry(ctx, X, n, d, ldx, opts, A, m_cap, m_out, s_out, cert, stream, nullptr);
}

}  // extern "C"
