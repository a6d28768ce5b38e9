// Split-precision GEMM on tcgen05 tensor cores (the covariance and subspace
// products of the randomized PCA, Sec. 2 / Sec. 4.5, and the projection
// Y = X A^T of Algorithm 1).
#pragma once

#include "internal.cuh"

namespace adagio {

// A matrix held as two 16-bit planes hi + lo (FP16, or BF16) of s * values,
// rows x Kp, row-major, Kp a multiple of 64 (zero beyond the real columns).
// The scale s is a power of two per row (scale[r * scale_stride]; stride 0:
// one scale for the whole matrix).
struct SplitPlanes {
    const uint16_t *hi = nullptr, *lo = nullptr;
    int64_t rows = 0;
    int Kp = 0;
    const float *scale = nullptr;
    int scale_stride = 0;
    bool bf16 = false;
};

inline int pad64(int64_t k) { return (int)((k + 63) / 64 * 64); }

// Planes of a row-major FP32 matrix (rows x cols, leading dimension ld) with a
// power-of-two FP16 scale per row; hi, lo hold rows x pad64(cols) halves and
// scale `rows` floats (caller-allocated device memory).
void split_rows(const float *src, int64_t rows, int cols, int64_t ld, uint16_t *hi, uint16_t *lo,
                float *scale, cudaStream_t st);

// Planes of the transpose of (X - mu): cols x pad64(n) halves (row c holds
// column c of X over all n rows), one power-of-two FP16 scale for the matrix
// from amax = max |x - mu| (device, as float bits), written to *scale.
void split_transpose_centred(const float *X, int64_t n, int cols, int64_t ldx, const float *mu,
                             const unsigned *amax_bits, uint16_t *hi, uint16_t *lo, float *scale,
                             cudaStream_t st);

// Workspace floats tc_gemm needs for any M' x N' with M' <= M, N' <= N and
// K = Kp (split-K partials; sym: M' = N').
int64_t tc_gemm_workspace(adagio_ctx *ctx, int M, int N, int Kp, bool sym);

// C (M x N, FP32, leading dimension ldc) = A B^T (+ bias[c] per column), from
// the planes of A (M x K) and B (N x K), three products per 64-wide K chunk
// (hi.lo + lo.hi + hi.hi), each chunk accumulated in a fresh TMEM slot and
// summed in FP32 registers, split-K partials summed in FP64.  sym: A and B are
// the same matrix, only the upper tiles are formed and C is mirrored.
// `part` holds tc_gemm_workspace floats; `status` (device) gets a nonzero
// code when a bounded wait gave up.
void tc_gemm(adagio_ctx *ctx, const SplitPlanes &A, const SplitPlanes &B, int M, int N,
             const float *bias, float *C, int64_t ldc, bool sym, float *part, int *status,
             cudaStream_t st);

void tc_gemm_init();

// The projection of Algorithm 1 on tensor cores: Y (n x m, leading dimension
// ldy) = X A^T for the map A (m x d, FP32, leading dimension lda), from the
// split planes Xp of X (Kp = pad64(d)) that hold s (x - mu) (mu given) or
// s x (mu null); with mu the product adds back A mu per column.  `scratch`
// holds embed_tc_bytes device bytes.  FP16 planes only.
size_t embed_tc_bytes(adagio_ctx *ctx, int64_t n, int m, int d);
void embed_tc(adagio_ctx *ctx, const SplitPlanes &Xp, int64_t n, const float *mu, const float *A, int m,
              int d, int64_t lda, float *Y, int64_t ldy, void *scratch, cudaStream_t st);

}  // namespace adagio
