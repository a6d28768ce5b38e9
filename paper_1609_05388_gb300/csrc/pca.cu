// Randomized PCA (Sec. 2 "PCA"; the randomized variant of Sec. 4.5, after
// Martinsson et al.): top principal directions of the centred data, computed
// by block subspace iteration on the covariance C = Xc^T Xc.
//
//   C        : split-K FP32 Gram of the centred rows, partials summed in FP64
//   start    : +-1 block V (b x d, rows are vectors) from the counter RNG
//   iterate  : W = V C; H = V W^T (FP64); H = U diag(theta) U^T (Jacobi);
//              V <- U^T V, W <- U^T W (Rayleigh-Ritz); stop when every kept
//              Ritz residual ||W_i - theta_i V_i|| <= tol * theta_1 (taken
//              outside span(V), which is what an exact Rayleigh-Ritz leaves);
//              otherwise V <- orth(W) (shifted CholeskyQR3 in FP32 with an
//              FP64 Gram in the first pass; only the first, shifted pass when
//              the next iteration is not a Rayleigh-Ritz step: the iteration
//              needs a well-conditioned basis of the subspace there, and the
//              Rayleigh-Ritz step an orthonormal one)
//   blocks   : directions are found in blocks of at most kJacobiMax - p;
//              later blocks iterate in the orthogonal complement of the
//              earlier ones (deflation), so the rows of P stay sorted by
//              eigenvalue and any prefix P[:s] is the top-s subspace.
#include "internal.cuh"
#include "linalg.cuh"
#include "jl.cuh"
#include "pca.cuh"
#include "prep.cuh"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>

namespace adagio {

static int64_t pca_part_floats(int d, int s_cap) {
    return (int64_t)8 * std::min(kJacobiMax, d) * std::max(d, std::max(s_cap, 1));
}

size_t pca_bytes(adagio_ctx *ctx, int64_t n, int d, int s_cap, int oversample, bool tensor) {
    const int b = std::min(kJacobiMax, d);
    size_t bytes = prep_bytes(n, d, !tensor, false);
    bytes += align_up((size_t)d * d * sizeof(float), 256);                          // C
    if (tensor) {
        const int Kn = pad64(n), Kd = pad64(d);
        bytes += 2 * align_up((size_t)d * Kn * sizeof(uint16_t), 256) + 256;       // X^T planes
        bytes += align_up((size_t)tc_gemm_workspace(ctx, d, d, Kn, true) * sizeof(float), 256);
        bytes += 2 * align_up((size_t)d * Kd * sizeof(uint16_t), 256);             // C planes
        bytes += align_up((size_t)d * sizeof(float), 256);
        bytes += 2 * align_up((size_t)b * Kd * sizeof(uint16_t), 256);             // V planes
        bytes += align_up((size_t)b * sizeof(float), 256);
        bytes += align_up((size_t)tc_gemm_workspace(ctx, b, d, Kd, false) * sizeof(float), 256);
    } else {
        bytes += align_up((size_t)splitk_chunks(n) * d * d * sizeof(float), 256);   // partials
    }
    bytes += 3 * align_up((size_t)b * d * sizeof(float), 256);                      // V, W, T
    bytes += align_up((size_t)b * 32 * sizeof(float), 256);                         // Dinv
    bytes += align_up((size_t)std::max(s_cap, 1) * d * sizeof(float), 256);         // P
    bytes += align_up((size_t)std::max(s_cap, 1) * b * sizeof(float), 256);         // proj coeffs
    bytes += 2 * align_up((size_t)b * b * sizeof(double), 256);                     // G, H
    bytes += align_up((size_t)b * b * sizeof(float), 256);                          // U
    bytes += align_up((size_t)(b + std::max(s_cap, 1)) * sizeof(double), 256);     // theta
    bytes += align_up((size_t)b * sizeof(float), 256);                              // residuals
    bytes += align_up((size_t)ceil_div(d, kF64Chunk) * b * b * sizeof(double), 256); // split-K
    bytes += 2 * align_up((size_t)b * b * sizeof(float), 256);                     // G32, R32
    bytes += align_up(pca_part_floats(d, s_cap) * sizeof(float), 256);             // FP32 split-K
    (void)oversample;
    return bytes + 8192;
}

size_t pca_host_bytes() { return (size_t)kJacobiMax * 12 + 128; }

void *PCA::stage(size_t bytes) { return hbuf ? hbuf : host_stage(ctx, bytes); }

void PCA::init_enqueue(adagio_ctx *ctx_, const float *X, int64_t n_, int d_, int64_t ldx,
                       int s_cap_, uint64_t seed_, int max_iter_, double tol_, int oversample_,
                       bool tensor_, cudaStream_t st) {
    ctx = ctx_;
    tensor = tensor_;
    n = n_;
    d = d_;
    s_cap = std::max(0, std::min(s_cap_, d_));
    seed = seed_;
    max_iter = std::max(1, max_iter_);
    tol = tol_ > 0 ? tol_ : 1e-6;
    p = std::max(1, std::min(oversample_, kJacobiMax / 2));
    s_done = 0;
    iterations = 0;
    theta1 = 0.0;
    blk = Block{};
    flags = ws_array<unsigned>(ctx, 1);
    ADAGIO_CUDA(cudaMemsetAsync(flags, 0, sizeof(unsigned), st));
    // centring (K0) and the covariance C = Xc^T Xc: tensor cores from the
    // transposed split planes of Xc, or FP32 SIMT from a centred copy
    PrepMat pm;
    prep_matrix(ctx, X, n, d, ldx, ADAGIO_PREC_FP32, !tensor, false, pm, flags, st);
    C = ws_array<float>(ctx, (size_t)d * d);
    const int bmax = std::min(kJacobiMax, d);
    if (tensor) {
        const int Kn = pad64(n), Kd = pad64(d);
        SplitPlanes XT;
        uint16_t *xh = ws_array<uint16_t>(ctx, (size_t)d * Kn), *xl = ws_array<uint16_t>(ctx, (size_t)d * Kn);
        float *xs = ws_array<float>(ctx, 1);
        split_transpose_centred(X, n, d, ldx, pm.mu, pm.amax, xh, xl, xs, st);
        XT.hi = xh;
        XT.lo = xl;
        XT.rows = d;
        XT.Kp = Kn;
        XT.scale = xs;
        float *cpart = ws_array<float>(ctx, (size_t)std::max<int64_t>(1, tc_gemm_workspace(ctx, d, d, Kn, true)));
        tc_gemm(ctx, XT, XT, d, d, nullptr, C, d, true, cpart, ctx->dev_status, st);
        // planes of C (rows) and room for those of each block V
        uint16_t *ch = ws_array<uint16_t>(ctx, (size_t)d * Kd), *cl = ws_array<uint16_t>(ctx, (size_t)d * Kd);
        float *cs = ws_array<float>(ctx, d);
        split_rows(C, d, d, d, ch, cl, cs, st);
        Cp.hi = ch;
        Cp.lo = cl;
        Cp.rows = d;
        Cp.Kp = Kd;
        Cp.scale = cs;
        Cp.scale_stride = 1;
        Vp.hi = ws_array<uint16_t>(ctx, (size_t)bmax * Kd);
        Vp.lo = ws_array<uint16_t>(ctx, (size_t)bmax * Kd);
        Vp.scale = ws_array<float>(ctx, bmax);
        Vp.Kp = Kd;
        Vp.scale_stride = 1;
        gpart = ws_array<float>(ctx, (size_t)std::max<int64_t>(1, tc_gemm_workspace(ctx, bmax, d, Kd, false)));
    } else {
        float *partials = ws_array<float>(ctx, (size_t)splitk_chunks(n) * d * d);
        gemm_tn_splitk(d, d, n, pm.c32, pm.Kp32, pm.c32, pm.Kp32, C, d, partials, st);
    }
    V = ws_array<float>(ctx, (size_t)bmax * d);
    W = ws_array<float>(ctx, (size_t)bmax * d);
    T = ws_array<float>(ctx, (size_t)bmax * d);
    Dinv = ws_array<float>(ctx, (size_t)bmax * 32);
    P = ws_array<float>(ctx, (size_t)std::max(s_cap, 1) * d);
    coef = ws_array<float>(ctx, (size_t)std::max(s_cap, 1) * bmax);
    G = ws_array<double>(ctx, (size_t)bmax * bmax);
    H = ws_array<double>(ctx, (size_t)bmax * bmax);
    U = ws_array<float>(ctx, (size_t)bmax * bmax);
    theta_blk = ws_array<double>(ctx, bmax);
    theta = ws_array<double>(ctx, std::max(s_cap, 1));
    res = ws_array<float>(ctx, bmax);
    f64part = ws_array<double>(ctx, (size_t)ceil_div(d, kF64Chunk) * bmax * bmax);
    G32 = ws_array<float>(ctx, (size_t)bmax * bmax);
    R32 = ws_array<float>(ctx, (size_t)bmax * bmax);
    part_floats = pca_part_floats(d, s_cap);
    part = ws_array<float>(ctx, (size_t)part_floats);
    unsigned *hflag = reinterpret_cast<unsigned *>(stage(pca_host_bytes()));
    ADAGIO_CUDA(cudaMemcpyAsync(hflag, flags, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    copy_status(st);
}

// the tensor-core GEMMs' status word, copied beside the convergence data
static constexpr size_t kStatusOff = (size_t)kJacobiMax * 12 + 64;

void PCA::copy_status(cudaStream_t st) {
    if (!tensor) return;
    char *hs = reinterpret_cast<char *>(stage(pca_host_bytes()));
    ADAGIO_CUDA(cudaMemcpyAsync(hs + kStatusOff, ctx->dev_status, sizeof(int), cudaMemcpyDeviceToHost, st));
}

void PCA::check_status() {
    if (!tensor) return;
    const int h = *reinterpret_cast<const int *>(reinterpret_cast<const char *>(stage(pca_host_bytes())) +
                                                 kStatusOff);
    if (h != 0) {
        ADAGIO_CUDA(cudaMemset(ctx->dev_status, 0, sizeof(int)));
        fail(ADAGIO_E_TIMEOUT, "tensor-core GEMM of the PCA gave up a bounded wait (status %d)", h);
    }
}

void PCA::init_check() {
    const unsigned hflag = *reinterpret_cast<unsigned *>(stage(pca_host_bytes()));
    if (hflag & 1u) fail(ADAGIO_E_NONFINITE, "input holds NaN or Inf");
    check_status();
}

void PCA::init(adagio_ctx *ctx_, const float *X, int64_t n_, int d_, int64_t ldx, int s_cap_,
               uint64_t seed_, int max_iter_, double tol_, int oversample_, bool tensor_,
               cudaStream_t st) {
    init_enqueue(ctx_, X, n_, d_, ldx, s_cap_, seed_, max_iter_, tol_, oversample_, tensor_, st);
    ADAGIO_CUDA(cudaStreamSynchronize(st));
    init_check();
}

// out (b x d) = M C for the rows of M (C symmetric)
void PCA::times_C(const float *M, int b, float *out, cudaStream_t st) {
    if (tensor) {
        Vp.rows = b;
        split_rows(M, b, d, d, const_cast<uint16_t *>(Vp.hi), const_cast<uint16_t *>(Vp.lo),
                   const_cast<float *>(Vp.scale), st);
        tc_gemm(ctx, Vp, Cp, b, d, nullptr, out, d, false, gpart, ctx->dev_status, st);
    } else {
        gemm_f32(b, d, d, 1.0f, MatView<float>{const_cast<float *>(M), d, 1}, MatView<float>{C, d, 1},
                 0.0f, out, d, part, part_floats, st);
    }
}

// rows of M (r x d) <- M - (M P^T) P over the s_done finished directions
void PCA::deflate(float *M, int r, cudaStream_t st) {
    if (s_done == 0 || r == 0) return;
    gemm_f32(r, s_done, d, 1.0f, MatView<float>{M, d, 1}, MatView<float>{P, 1, d}, 0.0f, coef,
             s_done, part, part_floats, st);
    gemm_f32(r, d, s_done, -1.0f, MatView<float>{coef, s_done, 1}, MatView<float>{P, d, 1}, 1.0f,
             M, d, part, part_floats, st);
}

// Orthonormalises the rows of M (b x d): shifted CholeskyQR3 (Fukaya et al.,
// SIAM J. Sci. Comput. 2020) in FP32.  Each pass forms the Gram M M^T, factors
// it as R^T R with the blocked one-CTA Cholesky and replaces M by R^{-T} M
// (block forward substitution).  The first pass takes its Gram in FP64 and
// (by default) a shift of 1e-5 of the largest diagonal entry, so it succeeds
// for any conditioning an FP32 matrix can carry and leaves a basis with
// condition number below ~300; passes with FP32 Grams (shift 1e-7, then
// none) then restore orthonormality.
void PCA::orth(float *M, int b, cudaStream_t st, int passes, float shift0) {
    for (int pass = 0; pass < passes; ++pass) {
        if (pass == 0) {
            gemm_f64_splitk(b, b, d, MatView<float>{M, d, 1}, MatView<float>{M, 1, d}, G, f64part,
                            kF64Chunk, st);
            cholesky_blocked<double>(G, b, shift0, R32, Dinv, st);
        } else {
            gemm_f32(b, b, d, 1.0f, MatView<float>{M, d, 1}, MatView<float>{M, 1, d}, 0.0f, G32, b,
                     part, part_floats, st);
            cholesky_blocked<float>(G32, b, pass == 1 ? 1e-7f : 0.0f, R32, Dinv, st);
        }
        trsm_blocked(R32, Dinv, b, M, d, d, st);
    }
}

// Rayleigh-Ritz (and the convergence test) after kRRFirst iterations, then at
// the iteration where the last test predicts convergence (at most kRRMax
// iterations later), and on the last; CholeskyQR keeps V orthonormal in
// between.  The prediction: the Ritz residual of direction i shrinks by about
// theta_b / theta_i per iteration (the block's smallest Ritz value standing
// in for the first eigenvalue outside the block).
constexpr int kRRMax = 8;
// The first Rayleigh-Ritz step of a block comes after a few iterations: on
// the random start block its convergence test cannot pass, and its dense
// Jacobi solve is the most expensive one.
constexpr int kRRFirst = 3;

// whether iteration `it` of the current block ends with a Rayleigh-Ritz step
bool PCA::rr_follows(int it) const {
    return it >= blk.next_rr || it == max_iter - 1 || blk.b == blk.remaining;
}

void PCA::begin_block(int s_needed, cudaStream_t st) {
    (void)s_needed;
    blk.remaining = d - s_done;
    blk.s_blk = std::min({s_cap - s_done, kJacobiMax - p, blk.remaining});
    blk.b = std::min(blk.s_blk + p, blk.remaining);
    blk.it = 0;
    blk.next_rr = std::min(kRRFirst, max_iter - 1);
    blk.rr = 0;
    blk.last = false;
    blk.active = true;
    rademacher_block(seed + (uint64_t)s_done * 0x9E3779B9ull, blk.b, d, V, d, st);
    deflate(V, blk.b, st);
    // the +-1 rows are nearly orthogonal (|cos| ~ 1/sqrt(d)) and their common
    // scale does not matter to the iteration: only a Rayleigh-Ritz step right
    // away needs an orthonormal start
    if (rr_follows(0)) orth(V, blk.b, st, 3);
}

void PCA::advance(int s_needed, cudaStream_t st) {
    if (!blk.active) begin_block(s_needed, st);
    const int b = blk.b, s_blk = blk.s_blk;
    for (;;) {
        ++iterations;
        // W = V C (C symmetric)
        times_C(V, b, W, st);
        deflate(W, b, st);
        const int it = blk.it;
        blk.last = it == max_iter - 1 || b == blk.remaining;
        if (it >= blk.next_rr || blk.last) {
            // Rayleigh-Ritz: H = V W^T, H = U diag(theta) U^T
            gemm_f64_splitk(b, b, d, MatView<float>{V, d, 1}, MatView<float>{W, 1, d}, H, f64part,
                            kF64Chunk, st);
            // the first Rayleigh-Ritz step of a block sees a dense H; later ones
            // start near-diagonal, where Jacobi converges quadratically for
            // separated Ritz values.  Rotations inside a cluster of nearly equal
            // values are left unfinished: they mix directions that are
            // interchangeable, and the convergence test measures the subspace.
            // the off-diagonal rows of H are in-subspace residuals of the
            // Ritz rows: once their norm is below 0.1 tol theta_1 (squared:
            // 0.01 tol^2 of the diagonal mass, which is at least theta_1^2)
            // they are negligible next to what the residual test accepts
            jacobi_eig(H, b, theta_blk, U, blk.rr == 0 ? 6 : 3, (float)(0.01 * tol * tol), st);
            ++blk.rr;
            // V <- U^T V, W <- U^T W
            gemm_f32(b, d, b, 1.0f, MatView<float>{U, 1, b}, MatView<float>{V, d, 1}, 0.0f, T, d,
                     part, part_floats, st);
            std::swap(V, T);
            gemm_f32(b, d, b, 1.0f, MatView<float>{U, 1, b}, MatView<float>{W, d, 1}, 0.0f, T, d,
                     part, part_floats, st);
            std::swap(W, T);
            // T (the old W) is free: scratch of the residuals
            ritz_residuals_projected(W, V, d, d, b, theta_blk, s_blk, T, coef, part, part_floats, res,
                                     st);
            char *hs = reinterpret_cast<char *>(stage(pca_host_bytes()));
            ADAGIO_CUDA(cudaMemcpyAsync(hs, theta_blk, sizeof(double) * b, cudaMemcpyDeviceToHost, st));
            ADAGIO_CUDA(cudaMemcpyAsync(hs + (size_t)kJacobiMax * 8, res, sizeof(float) * s_blk,
                                        cudaMemcpyDeviceToHost, st));
            copy_status(st);
            return;
        }
        // next iterate: V <- orth(W), orthonormal if a Rayleigh-Ritz step follows
        std::swap(V, W);
        orth(V, b, st, rr_follows(blk.it + 1) ? 3 : 1);
        ++blk.it;
    }
}

void PCA::resolve(cudaStream_t st) {
    check_status();
    const char *hs = reinterpret_cast<const char *>(stage(pca_host_bytes()));
    const double *hth = reinterpret_cast<const double *>(hs);
    const float *hres = reinterpret_cast<const float *>(hs + (size_t)kJacobiMax * 8);
    if (s_done == 0) theta1 = std::max(hth[0], 0.0);
    float worst = 0.0f;
    for (int i = 0; i < blk.s_blk; ++i) worst = std::max(worst, hres[i]);
    if (!(worst > tol * theta1) || blk.last) {
        accept_block(st);
        return;
    }
    int k_pred = 1;
    const double theta_b = hth[blk.b - 1];
    for (int i = 0; i < blk.s_blk; ++i) {
        const double r = hres[i], target = tol * theta1;
        if (!(r > target)) continue;
        const double rho = hth[i] > 0.0 ? theta_b / hth[i] : 1.0;
        int k = kRRMax;
        if (rho > 0.0 && rho < 0.999) k = (int)std::ceil(std::log(target / r) / std::log(rho));
        k_pred = std::max(k_pred, std::min(std::max(k, 1), kRRMax));
    }
    blk.next_rr = blk.it + k_pred;
    std::swap(V, W);
    orth(V, blk.b, st, rr_follows(blk.it + 1) ? 3 : 1);
    ++blk.it;
}

// accept the first s_blk Ritz vectors; re-orthonormalise against the earlier
// blocks and among themselves
void PCA::accept_block(cudaStream_t st) {
    const int s_blk = blk.s_blk;
    float *dst = P + (size_t)s_done * d;
    copy_rows(V, d, dst, d, s_blk, d, st);
    // the Ritz vectors are orthonormal to ~1e-6 (an orthonormal basis turned
    // by the Jacobi rotations); a later block's deflation moves them by less,
    // and one unshifted pass with an FP64 Gram restores FP32 orthonormality
    if (s_done > 0) {
        deflate(dst, s_blk, st);
        orth(dst, s_blk, st, 1, 0.0f);
    }
    canonical_signs(dst, s_blk, d, d, st);
    ADAGIO_CUDA(cudaMemcpyAsync(theta + s_done, theta_blk, sizeof(double) * s_blk,
                                cudaMemcpyDeviceToDevice, st));
    s_done += s_blk;
    blk.active = false;
}

void PCA::extend(int s_needed, cudaStream_t st) {
    const auto t0 = std::chrono::steady_clock::now();
    struct Timer {
        double *acc;
        std::chrono::steady_clock::time_point t0;
        ~Timer() {
            if (acc) *acc += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        }
    } timer{elapsed_ms, t0};
    while (needs(s_needed)) {
        advance(s_needed, st);
        ADAGIO_CUDA(cudaStreamSynchronize(st));
        resolve(st);
    }
}

}  // namespace adagio
