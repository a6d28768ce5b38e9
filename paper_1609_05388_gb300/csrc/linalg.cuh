// Dense linear-algebra building blocks of the fit (randomized PCA, Algorithm
// 1's assembly, the embedding).  All matrices live in device memory.
#pragma once

#include "internal.cuh"

namespace adagio {

// Strided matrix view: element (i, k) at p[i * rs + k * cs].
template <typename T>
struct MatView {
    const T *p;
    int64_t rs, cs;
};

// C[M x N] = alpha * A[M x K] * B[K x N] + beta * C, accumulating in TACC.
// Strides are arbitrary; C is row-major with leading dimension ldc.
template <typename TA, typename TB, typename TC, typename TACC>
void gemm(int M, int N, int K, TACC alpha, MatView<TA> A, MatView<TB> B, TACC beta, TC *C,
          int64_t ldc, cudaStream_t st);

// C[M x N] (FP32) = A^T B for tall A (K x M) and B (K x N) row-major with K
// rows (the covariance Xc^T Xc), split over K into FP32 partials that are
// summed in FP64.  `partials` must hold chunks(K) * M * N floats.
void gemm_tn_splitk(int M, int N, int64_t K, const float *A, int64_t lda, const float *B,
                    int64_t ldb, float *C, int64_t ldc, float *partials, cudaStream_t st);
int64_t splitk_chunks(int64_t K);

// C[M x N] (FP64, row-major, ld N) = A B with FP64 accumulation, split over K
// in chunks of kchunk so that small outputs still use many SMs; partials holds
// ceil(K / kchunk) * M * N doubles.
void gemm_f64_splitk(int M, int N, int K, MatView<float> A, MatView<float> B, double *C,
                     double *partials, int kchunk, cudaStream_t st);
constexpr int kF64Chunk = 32;

// raises the shared-memory limits of the block kernels (Cholesky, TRSM,
// Jacobi) to their largest block once, so later launches set no attribute
void linalg_init();

// Cholesky factorisation in place of an SPD b x b FP64 matrix (upper factor R,
// G = R^T R), one CTA.  Pivots below `floor_rel * max diagonal` are raised
// to it (shifted CholeskyQR guard).
void cholesky_upper(double *G, int b, double floor_rel, cudaStream_t st);

// V (b x d rows, FP32, leading dimension ldv) <- R^{-T} V, i.e. row i of the
// result is (v_i - sum_{k<i} R_ki r_k) / R_ii; FP32 arithmetic.
void trsm_rows(const double *R, int b, float *V, int64_t ldv, int d, cudaStream_t st);

// FP32 Cholesky (one CTA) of the SPD b x b Gram G (FP64 or FP32, row-major)
// with a diagonal shift of shift_rel * max(diag G): R (FP32 b x b upper,
// row-major).  Pivots are floored at 1e-7 of the largest diagonal entry.
template <typename TG>
void cholesky32(const TG *G, int b, float shift_rel, float *R, cudaStream_t st);

// Blocked FP32 Cholesky (one CTA) of the SPD b x b Gram G (FP64 or FP32,
// row-major) with a diagonal shift of shift_rel * max(diag G): R (b x b
// upper, row-major) and the inverses of its 32 x 32 diagonal blocks, Dinv
// (b x 32: row r holds row r - 32 floor(r / 32) of its block's inverse).
// Pivots are floored at 1e-7 of the largest diagonal entry.
template <typename TG>
void cholesky_blocked(const TG *G, int b, float shift_rel, float *R, float *Dinv, cudaStream_t st);

// M (b x d rows, leading dimension ldm) <- R^{-T} M with R and Dinv from
// cholesky_blocked (block forward substitution, one CTA per 16 columns).
void trsm_blocked(const float *R, const float *Dinv, int b, float *M, int64_t ldm, int d,
                  cudaStream_t st);

// V (b x d rows, FP32, leading dimension ldv) <- R^{-T} V with R from
// cholesky32: one warp per column of V.
void trsm_warp(const float *R, int b, float *V, int64_t ldv, int d, cudaStream_t st);

// FP32 GEMM like gemm<float...>, split over K when the output has too few
// tiles to fill the GPU: partial products go to `partials` (up to
// partial_floats floats) and are summed in a fixed order, so the result is
// deterministic.  partials == nullptr: no split.
void gemm_f32(int M, int N, int K, float alpha, MatView<float> A, MatView<float> B, float beta,
              float *C, int64_t ldc, float *partials, int64_t partial_floats, cudaStream_t st);

// Symmetric eigen-decomposition of a b x b matrix (b <= kJacobiMax) by
// parallel cyclic Jacobi in one CTA: H (FP64 in) -> theta (descending, FP64
// out) and U (b x b FP32 row-major, column c = eigenvector of theta[c]).
// Sweeps stop once the squared off-diagonal Frobenius norm is at most
// off_rel2 (at least 1e-12) of the diagonal's, at the FP32 floor, or after
// max_sweeps.
constexpr int kJacobiMax = 160;
void jacobi_eig(const double *H, int b, double *theta, float *U, int max_sweeps, float off_rel2,
                cudaStream_t st);

// Per-row residual norms ||W_i - theta_i V_i|| for i < s (FP32 out).
void ritz_residuals(const float *W, const float *V, int64_t ld, int d, const double *theta, int s,
                    float *res, cudaStream_t st);

// Ritz residual norms taken outside the subspace: for i < s,
// res_i = ||(I - V^T V)(W_i - theta_i V_i)|| with V (b x d) orthonormal rows.
// For exact Rayleigh-Ritz pairs this equals ||W_i - theta_i V_i|| (the
// residual is orthogonal to the subspace); it does not count the part that an
// inexact rotation leaves inside the subspace.  Rm: s x d scratch; coef:
// s x b scratch; partials: split-K scratch of gemm_f32.
void ritz_residuals_projected(const float *W, const float *V, int64_t ld, int d, int b,
                              const double *theta, int s, float *Rm, float *coef, float *partials,
                              int64_t partial_floats, float *res, cudaStream_t st);

// Flip the sign of each row of P (s x d) so its largest-magnitude entry
// (lowest index on ties) is positive.
void canonical_signs(float *P, int s, int d, int64_t ldp, cudaStream_t st);

// Copies of strided matrices.
void copy_rows(const float *src, int64_t lds, float *dst, int64_t ldd, int rows, int cols,
               cudaStream_t st);

}  // namespace adagio
