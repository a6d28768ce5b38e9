// Dense linear algebra of the fit: a strided SIMT GEMM (FP32 or FP64
// accumulation), split-K covariance, one-CTA Cholesky and parallel cyclic
// Jacobi, row-wise triangular solve, Ritz residuals and sign canonicalisation.
#include "linalg.cuh"

namespace adagio {

namespace {

constexpr int GT = 64, GK = 16, GNT = 256;

template <typename TA, typename TB, typename TC, typename TACC>
__global__ void __launch_bounds__(GNT) gemm_kernel(int M, int N, int K, int kchunk, TACC alpha,
                                                   MatView<TA> A, MatView<TB> B, TACC beta, TC *C,
                                                   int64_t ldc, int64_t zstride) {
    __shared__ TACC As[GK][GT + 1];
    __shared__ TACC Bs[GK][GT + 1];
    const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
    const int row0 = blockIdx.y * GT, col0 = blockIdx.x * GT;
    const int kbeg = blockIdx.z * kchunk;
    const int kend = min(K, kbeg + kchunk);
    C += (int64_t)blockIdx.z * zstride;
    TACC acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0;
    const bool a_kmajor = (A.cs == 1);
    const bool b_nmajor = (B.cs == 1);
    for (int k0 = kbeg; k0 < kend; k0 += GK) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int e = tid + GNT * q;
            int r, k;
            if (a_kmajor) { r = e >> 4; k = e & 15; } else { k = e >> 6; r = e & 63; }
            const int gr = row0 + r, gk = k0 + k;
            As[k][r] = (gr < M && gk < kend) ? (TACC)A.p[(int64_t)gr * A.rs + (int64_t)gk * A.cs] : (TACC)0;
            int c, kb;
            if (b_nmajor) { kb = e >> 6; c = e & 63; } else { c = e >> 4; kb = e & 15; }
            const int gc = col0 + c, gkb = k0 + kb;
            Bs[kb][c] = (gc < N && gkb < kend) ? (TACC)B.p[(int64_t)gkb * B.rs + (int64_t)gc * B.cs] : (TACC)0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GK; ++kk) {
            TACC a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * b[j];
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int r = row0 + ty + 16 * i;
        if (r >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int c = col0 + tx + 16 * j;
            if (c >= N) continue;
            TACC v = alpha * acc[i][j];
            if (beta != (TACC)0) v += beta * (TACC)C[(int64_t)r * ldc + c];
            C[(int64_t)r * ldc + c] = (TC)v;
        }
    }
}

__global__ void splitk_reduce_kernel(const float *__restrict__ part, int64_t chunks, int M, int N,
                                     float *__restrict__ C, int64_t ldc) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)M * N) return;
    double acc = 0.0;
    for (int64_t z = 0; z < chunks; ++z) acc += (double)part[z * (int64_t)M * N + e];
    C[(e / N) * ldc + (e % N)] = (float)acc;
}

constexpr int kSplitRows = 2048;

// C_z = A B over the K chunk z, FP32 operands, each product exact (FMA
// TwoProduct) and summed as an unevaluated double-float (TwoSum; Dekker 1971,
// Knuth TAOCP vol. 2, 4.2.2): FP64-grade sums on the FP32 pipes, which run far
// faster than FP64 on this GPU.  Same tiling as gemm_kernel; FP64 output.
__device__ __forceinline__ void df_fma(float a, float b, float &hi, float &lo) {
    const float p = __fmul_rn(a, b);
    const float pe = __fmaf_rn(a, b, -p);  // a b = p + pe exactly
    const float s = __fadd_rn(hi, p);
    const float bp = __fsub_rn(s, hi);
    const float ap = __fsub_rn(s, bp);
    const float e = __fadd_rn(__fsub_rn(hi, ap), __fsub_rn(p, bp));
    hi = s;
    lo = __fadd_rn(lo, __fadd_rn(e, pe));
}

__global__ void __launch_bounds__(GNT) gemm_df_kernel(int M, int N, int K, int kchunk, MatView<float> A,
                                                      MatView<float> B, double *C, int64_t ldc,
                                                      int64_t zstride) {
    __shared__ float As[GK][GT + 1];
    __shared__ float Bs[GK][GT + 1];
    const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
    const int row0 = blockIdx.y * GT, col0 = blockIdx.x * GT;
    const int kbeg = blockIdx.z * kchunk;
    const int kend = min(K, kbeg + kchunk);
    C += (int64_t)blockIdx.z * zstride;
    float hi[4][4], lo[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) hi[i][j] = lo[i][j] = 0.0f;
    const bool a_kmajor = (A.cs == 1);
    const bool b_nmajor = (B.cs == 1);
    for (int k0 = kbeg; k0 < kend; k0 += GK) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int e = tid + GNT * q;
            int r, k;
            if (a_kmajor) { r = e >> 4; k = e & 15; } else { k = e >> 6; r = e & 63; }
            const int gr = row0 + r, gk = k0 + k;
            As[k][r] = (gr < M && gk < kend) ? A.p[(int64_t)gr * A.rs + (int64_t)gk * A.cs] : 0.0f;
            int c, kb;
            if (b_nmajor) { kb = e >> 6; c = e & 63; } else { c = e >> 4; kb = e & 15; }
            const int gc = col0 + c, gkb = k0 + kb;
            Bs[kb][c] = (gc < N && gkb < kend) ? B.p[(int64_t)gkb * B.rs + (int64_t)gc * B.cs] : 0.0f;
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < GK; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) df_fma(a[i], b[j], hi[i][j], lo[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int r = row0 + ty + 16 * i;
        if (r >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int c = col0 + tx + 16 * j;
            if (c >= N) continue;
            C[(int64_t)r * ldc + c] = (double)hi[i][j] + (double)lo[i][j];
        }
    }
}

__global__ void splitk_reduce_f64_kernel(const double *__restrict__ part, int chunks, int64_t mn,
                                         double *__restrict__ C) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= mn) return;
    double acc = 0.0;
    for (int z = 0; z < chunks; ++z) acc += part[(int64_t)z * mn + e];
    C[e] = acc;
}

__global__ void cholesky_kernel(double *G, int b, double floor_rel) {
    extern __shared__ double S[];  // [b][b+1]
    const int ld = b + 1;
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int e = tid; e < b * b; e += nt) S[(e / b) * ld + (e % b)] = G[e];
    __syncthreads();
    __shared__ double s_floor, s_piv;
    if (tid == 0) {
        double mx = 0.0;
        for (int i = 0; i < b; ++i) mx = fmax(mx, S[i * ld + i]);
        s_floor = fmax(mx * floor_rel, 1e-300);
    }
    __syncthreads();
    for (int k = 0; k < b; ++k) {
        if (tid == 0) {
            double p = S[k * ld + k];
            if (!(p > s_floor)) p = s_floor;
            s_piv = sqrt(p);
            S[k * ld + k] = s_piv;
        }
        __syncthreads();
        const double inv = 1.0 / s_piv;
        for (int j = k + 1 + tid; j < b; j += nt) S[k * ld + j] *= inv;
        __syncthreads();
        // trailing update of the upper triangle, 32 x 32 thread grid
        const int tx = tid & 31, ty = tid >> 5, nty = nt >> 5;
        for (int i = k + 1 + ty; i < b; i += nty) {
            const double rki = S[k * ld + i];
            for (int j = i + tx; j < b; j += 32) S[i * ld + j] -= rki * S[k * ld + j];
        }
        __syncthreads();
    }
    for (int e = tid; e < b * b; e += nt) {
        const int i = e / b, j = e % b;
        G[e] = (j >= i) ? S[i * ld + j] : 0.0;
    }
}

// FP32 Cholesky of a b x b SPD Gram (FP64 or FP32 input, row-major), one
// CTA: G + shift * max(diag) I = R^T R with R upper triangular (FP32,
// row-major, lower part zero).  Pivots are floored at 1e-7 of the largest
// diagonal entry (the factor stays finite for a rank-deficient Gram).
// Right-looking with the trailing matrix resident in registers: the upper
// triangle is cut into 4 x 4 blocks, each thread owns up to two of them; at
// step k the owners of row k publish it to a double-buffered shared row, one
// barrier later every thread applies the rank-1 update to its blocks.
constexpr int kCholThreads = 512;
constexpr int kCholBlk = 2;  // 4 x 4 blocks per thread (ceil(40 * 41 / 2 / 512))
template <typename TG>
__global__ void __launch_bounds__(kCholThreads) cholesky32_kernel(const TG *__restrict__ G, int b,
                                                                  float shift_rel,
                                                                  float *__restrict__ R) {
    __shared__ float rowbuf[2][kJacobiMax + 4];
    __shared__ float s_red[kCholThreads / 32];
    __shared__ float s_shift, s_floor;
    const int tid = threadIdx.x;
    float mx = 0.0f;
    for (int i = tid; i < b; i += kCholThreads) mx = fmaxf(mx, (float)G[(int64_t)i * b + i]);
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((tid & 31) == 0) s_red[tid >> 5] = mx;
    for (int e = tid; e < b * b; e += kCholThreads)
        if (e % b < e / b) R[e] = 0.0f;
    __syncthreads();
    if (tid == 0) {
        float m = 0.0f;
        for (int w = 0; w < kCholThreads / 32; ++w) m = fmaxf(m, s_red[w]);
        s_shift = shift_rel * m;
        s_floor = fmaxf(1e-7f * m, 1e-30f);
    }
    __syncthreads();
    const int nb = (b + 3) / 4;
    const int nblocks = nb * (nb + 1) / 2;
    int bi[kCholBlk], bj[kCholBlk];
    float S[kCholBlk][4][4];
#pragma unroll
    for (int q = 0; q < kCholBlk; ++q) {
        int lin = tid + q * kCholThreads;
        bi[q] = -1;
        bj[q] = -1;
        if (lin < nblocks) {
            int ib = 0;
            while (lin >= nb - ib) {
                lin -= nb - ib;
                ++ib;
            }
            bi[q] = ib;
            bj[q] = ib + lin;
        }
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int i = bi[q] * 4 + r, j = bj[q] * 4 + c;
                float v = 0.0f;
                if (bi[q] >= 0 && i < b && j < b && j >= i) v = (float)G[(int64_t)i * b + j] + (i == j ? s_shift : 0.0f);
                S[q][r][c] = v;
            }
        // publish row 0
        if (bi[q] == 0)
#pragma unroll
            for (int c = 0; c < 4; ++c) rowbuf[0][bj[q] * 4 + c] = S[q][0][c];
    }
    for (int k = 0; k < b; ++k) {
        __syncthreads();
        const float *row = rowbuf[k & 1];
        float piv = row[k];
        if (!(piv > s_floor)) piv = s_floor;
        const float inv = rsqrtf(piv);
        const float inv2 = inv * inv;
        for (int j = k + tid; j < b; j += kCholThreads)
            R[(int64_t)k * b + j] = j == k ? piv * inv : row[j] * inv;
        const int kn = k + 1;
#pragma unroll
        for (int q = 0; q < kCholBlk; ++q) {
            if (bi[q] < 0 || bi[q] * 4 + 3 <= k) continue;
            float a[4], w[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int i = bi[q] * 4 + r;
                a[r] = (i > k && i < b) ? row[i] * inv2 : 0.0f;
            }
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int j = bj[q] * 4 + c;
                w[c] = (j > k && j < b) ? row[j] : 0.0f;
            }
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) S[q][r][c] = fmaf(-a[r], w[c], S[q][r][c]);
            // row k + 1 lives in this block row: publish it for the next step
            if (kn < b && (kn >> 2) == bi[q]) {
                const int rr = kn & 3;
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const float v = rr == 0 ? S[q][0][c] : rr == 1 ? S[q][1][c] : rr == 2 ? S[q][2][c] : S[q][3][c];
                    rowbuf[kn & 1][bj[q] * 4 + c] = v;
                }
            }
        }
    }
}

// Blocked Cholesky G + shift I = R^T R (R upper, FP32) of an SPD b x b Gram,
// in one CTA, with 32 x 32 blocks.  For each diagonal block: one warp factors
// it (row k scaled by its pivot, then the rank-1 update of the rows below,
// warp-synchronous) and inverts it by back substitution (lane j = column j);
// the CTA then forms the panel to its right as D^T A_12 with that inverse D,
// and updates the trailing submatrix with 4 x 4 register tiles (SYRK).  The
// diagonal-block inverses are returned with R, so that the triangular solve
// R^{-T} M (trsm_blocked) is a short sequence of small products.  Pivots below
// 1e-7 of the largest diagonal entry are raised to it (the shifted CholeskyQR
// guard).
constexpr int kCiThreads = 512;
constexpr int kCiBlk = 32;
constexpr int kCiLd = kJacobiMax + 1;
constexpr size_t kCiSmem = (size_t)(kJacobiMax * kCiLd + 2 * kCiBlk * kCiLd) * sizeof(float);

template <typename TG>
__global__ void __launch_bounds__(kCiThreads) chol_blocked_kernel(const TG *__restrict__ G, int b,
                                                                  float shift_rel,
                                                                  float *__restrict__ R,
                                                                  float *__restrict__ Dinv) {
    extern __shared__ float ci_sm[];
    float *A = ci_sm;                        // [b][kCiLd]: R in the upper triangle
    float *D = A + kJacobiMax * kCiLd;       // [32][kCiLd]: inverse of the current diagonal block
    float *Z = D + kCiBlk * kCiLd;           // [32][kCiLd]: the panel D^T A_12
    __shared__ float s_red[kCiThreads / 32];
    __shared__ float s_shift, s_floor;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    float mx = 0.0f;
    for (int i = tid; i < b; i += kCiThreads) mx = fmaxf(mx, (float)G[(int64_t)i * b + i]);
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) s_red[warp] = mx;
    __syncthreads();
    if (tid == 0) {
        float m = 0.0f;
        for (int w = 0; w < kCiThreads / 32; ++w) m = fmaxf(m, s_red[w]);
        s_shift = shift_rel * m;
        s_floor = fmaxf(1e-7f * m, 1e-30f);
    }
    __syncthreads();
    const float shift = s_shift, floor_v = s_floor;
    for (int e = tid; e < b * b; e += kCiThreads) {
        const int i = e / b, j = e % b;
        A[i * kCiLd + j] = j >= i ? (float)G[(int64_t)i * b + j] + (i == j ? shift : 0.0f) : 0.0f;
    }
    __syncthreads();
    const int nb = (b + kCiBlk - 1) / kCiBlk;
    for (int kb = 0; kb < nb; ++kb) {
        const int k0 = kb * kCiBlk, bs = min(kCiBlk, b - k0), k1 = k0 + bs;
        if (warp == 0) {
            // the diagonal block in registers: lane j holds column j,
            // a[i] = A[k0 + i][k0 + j] for i <= j (an identity pad beyond bs)
            float a[kCiBlk], x[kCiBlk];
#pragma unroll
            for (int i = 0; i < kCiBlk; ++i) {
                const bool in = i < bs && lane < bs;
                a[i] = in ? (i <= lane ? A[(k0 + i) * kCiLd + k0 + lane] : 0.0f) : (i == lane ? 1.0f : 0.0f);
            }
            // factor: row k scaled by its pivot, then the rank-1 update below
#pragma unroll
            for (int k = 0; k < kCiBlk; ++k) {
                float piv = __shfl_sync(0xffffffffu, a[k], k);
                if (k < bs && !(piv > floor_v)) piv = floor_v;
                const float rkk = sqrtf(piv);
                const float inv = 1.0f / rkk;
                a[k] = lane == k ? rkk : (lane > k ? a[k] * inv : a[k]);
                // constant trip counts (resolved after unrolling) keep a[] in registers
#pragma unroll
                for (int i = 0; i < kCiBlk; ++i) {
                    if (i <= k) continue;
                    const float rki = __shfl_sync(0xffffffffu, a[k], i);
                    if (lane >= i) a[i] = fmaf(-rki, a[k], a[i]);
                }
            }
            // invert: x[i] = (R_kk^{-1})[i][lane], back substitution
#pragma unroll
            for (int i = kCiBlk - 1; i >= 0; --i) {
                const float rii = __shfl_sync(0xffffffffu, a[i], i);
                float acc = i == lane ? 1.0f : 0.0f;
#pragma unroll
                for (int m = 0; m < kCiBlk; ++m) {
                    if (m <= i) continue;
                    const float rim = __shfl_sync(0xffffffffu, a[i], m);
                    if (m <= lane) acc = fmaf(-rim, x[m], acc);
                }
                x[i] = i <= lane ? acc / rii : 0.0f;
            }
#pragma unroll
            for (int i = 0; i < kCiBlk; ++i) {
                if (lane < bs && i <= lane) A[(k0 + i) * kCiLd + k0 + lane] = a[i];
                D[i * kCiLd + lane] = (lane < bs && i < bs) ? x[i] : 0.0f;
            }
        }
        __syncthreads();
        if (k1 < b) {
            // panel: R_12 = D^T A_12 (A_12 = rows k0..k1, columns k1..b)
            const int rem = b - k1;
            for (int e = tid; e < bs * rem; e += kCiThreads) {
                const int i = e / rem, c = k1 + e % rem;
                float acc = 0.0f;
                for (int m = 0; m <= i; ++m) acc = fmaf(D[m * kCiLd + i], A[(k0 + m) * kCiLd + c], acc);
                Z[i * kCiLd + c] = acc;
            }
            __syncthreads();
            for (int e = tid; e < bs * rem; e += kCiThreads) {
                const int i = e / rem, c = k1 + e % rem;
                A[(k0 + i) * kCiLd + c] = Z[i * kCiLd + c];
            }
            __syncthreads();
            // trailing update A_22 -= R_12^T R_12 on 4 x 4 tiles of the upper triangle
            const int nt4 = (rem + 3) / 4;
            for (int e = tid; e < nt4 * nt4; e += kCiThreads) {
                const int ti = e / nt4, tj = e % nt4;
                if (tj < ti) continue;
                float acc[4][4];
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int c = 0; c < 4; ++c) acc[r][c] = 0.0f;
                const int i0 = k1 + 4 * ti, j0 = k1 + 4 * tj;
                for (int m = k0; m < k1; ++m) {
                    float u[4], w[4];
#pragma unroll
                    for (int r = 0; r < 4; ++r) u[r] = (i0 + r < b) ? A[m * kCiLd + i0 + r] : 0.0f;
#pragma unroll
                    for (int c = 0; c < 4; ++c) w[c] = (j0 + c < b) ? A[m * kCiLd + j0 + c] : 0.0f;
#pragma unroll
                    for (int r = 0; r < 4; ++r)
#pragma unroll
                        for (int c = 0; c < 4; ++c) acc[r][c] = fmaf(u[r], w[c], acc[r][c]);
                }
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const int i = i0 + r, j = j0 + c;
                        if (i < b && j < b && j >= i) A[i * kCiLd + j] -= acc[r][c];
                    }
            }
        }
        // the inverse of this diagonal block, rows k0..k1 of Dinv (b x 32)
        for (int e = tid; e < bs * kCiBlk; e += kCiThreads) {
            const int i = e / kCiBlk, c = e % kCiBlk;
            Dinv[(int64_t)(k0 + i) * kCiBlk + c] = c < bs ? D[i * kCiLd + c] : 0.0f;
        }
        __syncthreads();
    }
    for (int e = tid; e < b * b; e += kCiThreads) {
        const int i = e / b, j = e % b;
        R[e] = j >= i ? A[i * kCiLd + j] : 0.0f;
    }
}

// M (b x d rows) <- R^{-T} M by 32-row blocks with the diagonal-block
// inverses D_i of chol_blocked_kernel:
//   Y_i = D_i^T (M_i - sum_{k < i} R_ki^T Y_k)
// one CTA per 16 columns of M, everything in shared memory.
constexpr int kTbCols = 16;
constexpr int kTbThreads = 512;
constexpr size_t kTbSmem = (size_t)(kJacobiMax * kCiLd + kJacobiMax * kCiBlk + 2 * kJacobiMax * kTbCols) * sizeof(float);

__global__ void __launch_bounds__(kTbThreads) trsm_blocked_kernel(const float *__restrict__ R,
                                                                  const float *__restrict__ Dinv,
                                                                  int b, float *M, int64_t ldm, int d) {
    extern __shared__ float tb_sm[];
    float *Rs = tb_sm;                                // [b][kCiLd]
    float *Ds = Rs + kJacobiMax * kCiLd;              // [b][32]
    float *Ys = Ds + kJacobiMax * kCiBlk;             // [b][16]: solved rows
    float *Ts = Ys + kJacobiMax * kTbCols;            // [b][16]: right-hand sides
    const int tid = threadIdx.x;
    const int c0 = blockIdx.x * kTbCols;
    for (int e = tid; e < b * b; e += kTbThreads) {
        const int i = e / b, j = e % b;
        Rs[i * kCiLd + j] = R[e];
    }
    for (int e = tid; e < b * kCiBlk; e += kTbThreads) Ds[e] = Dinv[e];
    for (int e = tid; e < b * kTbCols; e += kTbThreads) {
        const int i = e / kTbCols, c = c0 + e % kTbCols;
        Ts[e] = c < d ? M[(int64_t)i * ldm + c] : 0.0f;
    }
    __syncthreads();
    const int nb = (b + kCiBlk - 1) / kCiBlk;
    for (int kb = 0; kb < nb; ++kb) {
        const int k0 = kb * kCiBlk, bs = min(kCiBlk, b - k0);
        // right-hand side of block kb minus the solved blocks
        for (int e = tid; e < bs * kTbCols; e += kTbThreads) {
            const int r = k0 + e / kTbCols, c = e % kTbCols;
            float acc = Ts[r * kTbCols + c];
            for (int m = 0; m < k0; ++m) acc = fmaf(-Rs[m * kCiLd + r], Ys[m * kTbCols + c], acc);
            Ts[r * kTbCols + c] = acc;
        }
        __syncthreads();
        // Y_kb = D^T T_kb (D upper: rows m <= r)
        for (int e = tid; e < bs * kTbCols; e += kTbThreads) {
            const int rl = e / kTbCols, c = e % kTbCols;
            float acc = 0.0f;
            for (int m = 0; m <= rl; ++m) acc = fmaf(Ds[(k0 + m) * kCiBlk + rl], Ts[(k0 + m) * kTbCols + c], acc);
            Ys[(k0 + rl) * kTbCols + c] = acc;
        }
        __syncthreads();
    }
    for (int e = tid; e < b * kTbCols; e += kTbThreads) {
        const int i = e / kTbCols, c = c0 + e % kTbCols;
        if (c < d) M[(int64_t)i * ldm + c] = Ys[e];
    }
}

// V (b x d rows) <- R^{-T} V, two columns per warp: each half-warp solves
// one column, lane l keeping the solved entries l, l + 16, ... in registers;
// each step is a lane-local partial dot product and a 16-lane reduction.  R
// (FP32 upper) is staged transposed in shared memory with a padded stride,
// so both the staging and the lanes of a step touch distinct banks.
constexpr int kTrsmWarps = 8;
constexpr int kTrsmRegs = (kJacobiMax + 15) / 16;
__global__ void __launch_bounds__(32 * kTrsmWarps) trsm_warp_kernel(const float *__restrict__ R, int b,
                                                                   float *V, int64_t ldv, int d) {
    extern __shared__ float Rsm[];  // Rsm[i * (b + 1) + k] = R[k][i]
    const int ldr = b + 1;
    for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
        const int k = e / b, i = e % b;
        Rsm[i * ldr + k] = R[e];
    }
    __syncthreads();
    const int lane = threadIdx.x & 15;
    const int j = (blockIdx.x * kTrsmWarps + (threadIdx.x >> 5)) * 2 + ((threadIdx.x >> 4) & 1);
    const bool ok = j < d;
    float v[kTrsmRegs], x[kTrsmRegs];
#pragma unroll
    for (int m = 0; m < kTrsmRegs; ++m) {
        const int k = lane + 16 * m;
        v[m] = (ok && k < b) ? V[(int64_t)k * ldv + j] : 0.0f;
        x[m] = 0.0f;
    }
#pragma unroll
    for (int m = 0; m < kTrsmRegs; ++m) {
        if (16 * m >= b) break;
        for (int ii = 0; ii < 16; ++ii) {
            const int i = 16 * m + ii;
            if (i >= b) break;
            // partial of sum_{k < i} R[k][i] x_k over this lane's k
            float part = 0.0f;
#pragma unroll
            for (int q = 0; q <= m; ++q) {
                const int k = lane + 16 * q;
                if (k < i) part = fmaf(Rsm[i * ldr + k], x[q], part);
            }
            for (int o = 8; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o, 16);
            const float vi = __shfl_sync(0xffffffffu, v[m], ii, 16);
            const float xi = __fdividef(vi - part, Rsm[i * ldr + i]);
            if (lane == ii) x[m] = xi;
        }
    }
    if (ok) {
#pragma unroll
        for (int m = 0; m < kTrsmRegs; ++m) {
            const int k = lane + 16 * m;
            if (k < b) V[(int64_t)k * ldv + j] = x[m];
        }
    }
}

// C = alpha * sum_z P_z + beta * C (split-K partials, fixed summation order)
__global__ void splitk_reduce_ab_kernel(const float *__restrict__ part, int chunks, int M, int N,
                                        float alpha, float beta, float *__restrict__ C, int64_t ldc) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)M * N) return;
    float acc = 0.0f;
    for (int z = 0; z < chunks; ++z) acc += part[(int64_t)z * M * N + e];
    float *c = C + (e / N) * ldc + (e % N);
    *c = beta != 0.0f ? fmaf(alpha, acc, beta * *c) : alpha * acc;
}

// Row-wise triangular solve: one thread per column of V, R's upper triangle
// staged in shared memory as FP32, four independent partial sums per row.
// FP32 arithmetic: the first CholeskyQR pass only needs a well-conditioned
// result (the second pass restores orthonormality to FP32 precision).
constexpr int kTrsmCols = 64;
__global__ void trsm_rows_kernel(const double *__restrict__ R, int b, float *V, int64_t ldv, int d) {
    extern __shared__ float sm_trsm[];
    float *Rs = sm_trsm;                 // [b][b] (row-major, upper triangle used)
    float *col = sm_trsm + b * b;        // [b][kTrsmCols]
    for (int e = threadIdx.x; e < b * b; e += blockDim.x) Rs[e] = (float)R[e];
    __syncthreads();
    const int j = blockIdx.x * kTrsmCols + threadIdx.x;
    const bool ok = j < d;
    for (int i = 0; i < b; ++i) {
        float a0 = ok ? V[(int64_t)i * ldv + j] : 0.0f, a1 = 0.0f, a2 = 0.0f, a3 = 0.0f;
        int k = 0;
        for (; k + 4 <= i; k += 4) {
            a0 = fmaf(-Rs[(k + 0) * b + i], col[(k + 0) * kTrsmCols + threadIdx.x], a0);
            a1 = fmaf(-Rs[(k + 1) * b + i], col[(k + 1) * kTrsmCols + threadIdx.x], a1);
            a2 = fmaf(-Rs[(k + 2) * b + i], col[(k + 2) * kTrsmCols + threadIdx.x], a2);
            a3 = fmaf(-Rs[(k + 3) * b + i], col[(k + 3) * kTrsmCols + threadIdx.x], a3);
        }
        for (; k < i; ++k) a0 = fmaf(-Rs[k * b + i], col[k * kTrsmCols + threadIdx.x], a0);
        const float v = ((a0 + a1) + (a2 + a3)) / Rs[i * b + i];
        col[i * kTrsmCols + threadIdx.x] = v;
        if (ok) V[(int64_t)i * ldv + j] = v;
    }
}

constexpr int kJacobiThreads = 1024;
constexpr int kJacobiColIt = (kJacobiMax / 2 + 31) / 32;  // column-pair rotations per lane

// Parallel cyclic Jacobi (round-robin pairing, b / 2 disjoint rotations per
// round) on H (FP32 in shared memory).  A round's rotations form a
// block-diagonal orthogonal matrix, so the two-sided update is applied block
// by block: for rotation pairs (a, b) the 2 x 2 block H_ab becomes
// A_a H_ab A_b^T, every element read and written once per round.  The
// eigenvectors accumulate as rows of U^T (row operations, float4 wide).
__global__ void __launch_bounds__(kJacobiThreads) jacobi_kernel(const double *__restrict__ Hin, int b,
                                                                double *__restrict__ theta,
                                                                float *__restrict__ Uout,
                                                                int max_sweeps, float off_rel2) {
    extern __shared__ float sm[];
    const int B = (b + 1) & ~1;   // even size (index b is a zero dummy when b is odd)
    const int half = B / 2;
    const int ld = B + 1;
    const int ldu = (B + 3) & ~3;
    float *H = sm;                 // [B][ld]
    float *Ut = sm + ((B * ld + 3) & ~3);  // [B][ldu], 16-byte aligned rows
    __shared__ float cs[kJacobiMax / 2 + 1], sn[kJacobiMax / 2 + 1];
    __shared__ int pp[kJacobiMax / 2 + 1], qq[kJacobiMax / 2 + 1];
    __shared__ float red[kJacobiThreads / 32][2];
    __shared__ int s_done;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int lx = tid & 31, wy = tid >> 5, nwy = nt >> 5;
    for (int i = wy; i < B; i += nwy)
        for (int j = lx; j < B; j += 32) {
            H[i * ld + j] = (i < b && j < b) ? (float)(0.5 * (Hin[i * b + j] + Hin[j * b + i])) : 0.0f;
            Ut[i * ldu + j] = (i == j) ? 1.0f : 0.0f;
        }
    float prev_off = 3.0e38f;
    __syncthreads();
    for (int sweep = 0; sweep < max_sweeps; ++sweep) {
        for (int r = 0; r < B - 1; ++r) {
            if (tid < half) {
                // round-robin pairing: index B - 1 stays, the others rotate
                int p, q;
                if (tid == 0) {
                    p = r;
                    q = B - 1;
                } else {
                    p = r + tid;
                    if (p >= B - 1) p -= B - 1;
                    q = r - tid;
                    if (q < 0) q += B - 1;
                }
                if (p > q) { int t = p; p = q; q = t; }
                float c = 1.0f, s = 0.0f;
                const float apq = H[p * ld + q];
                const float app = H[p * ld + p], aqq = H[q * ld + q];
                // a rotation whose angle is below FP32 resolution of the
                // diagonal changes nothing: identity
                if (q < b && fabsf(apq) > 1e-8f * fmaxf(fabsf(app), fabsf(aqq)) && apq != 0.0f) {
                    const float tau = (aqq - app) / (2.0f * apq);
                    const float t = (tau >= 0.0f ? 1.0f : -1.0f) / (fabsf(tau) + sqrtf(1.0f + tau * tau));
                    c = rsqrtf(1.0f + t * t);
                    s = t * c;
                }
                pp[tid] = p; qq[tid] = q; cs[tid] = c; sn[tid] = s;
            }
            __syncthreads();
            // this lane's column-pair rotations, read once per round
            int pb[kJacobiColIt], qb[kJacobiColIt];
            float cb[kJacobiColIt], sb[kJacobiColIt];
#pragma unroll
            for (int u = 0; u < kJacobiColIt; ++u) {
                const int rb = lx + 32 * u;
                const bool in = rb < half;
                pb[u] = in ? pp[rb] : 0;
                qb[u] = in ? qq[rb] : 0;
                cb[u] = in ? cs[rb] : 1.0f;
                sb[u] = in ? sn[rb] : 0.0f;
            }
            // H <- J^T H J, one 2 x 2 block (rotation a = row pair, b = column pair) per step
            for (int ra = wy; ra < half; ra += nwy) {
                const int pa = pp[ra], qa = qq[ra];
                const float ca = cs[ra], sa = sn[ra];
                const bool ida = sa == 0.0f;
#pragma unroll
                for (int u = 0; u < kJacobiColIt; ++u) {
                    const int rb = lx + 32 * u;
                    if (rb >= half || (ida && sb[u] == 0.0f)) continue;
                    float *r0 = H + pa * ld, *r1 = H + qa * ld;
                    const float h00 = r0[pb[u]], h01 = r0[qb[u]];
                    const float h10 = r1[pb[u]], h11 = r1[qb[u]];
                    const float t00 = ca * h00 - sa * h10, t01 = ca * h01 - sa * h11;
                    const float t10 = sa * h00 + ca * h10, t11 = sa * h01 + ca * h11;
                    r0[pb[u]] = cb[u] * t00 - sb[u] * t01;
                    r0[qb[u]] = sb[u] * t00 + cb[u] * t01;
                    r1[pb[u]] = cb[u] * t10 - sb[u] * t11;
                    r1[qb[u]] = sb[u] * t10 + cb[u] * t11;
                }
                // U^T rows pa, qa (the same rotation as H's rows)
                if (!ida) {
                    float4 *up = reinterpret_cast<float4 *>(Ut + pa * ldu);
                    float4 *uq = reinterpret_cast<float4 *>(Ut + qa * ldu);
                    for (int v = lx; v < ldu / 4; v += 32) {
                        const float4 x = up[v], y = uq[v];
                        up[v] = make_float4(ca * x.x - sa * y.x, ca * x.y - sa * y.y, ca * x.z - sa * y.z,
                                            ca * x.w - sa * y.w);
                        uq[v] = make_float4(sa * x.x + ca * y.x, sa * x.y + ca * y.y, sa * x.z + ca * y.z,
                                            sa * x.w + ca * y.w);
                    }
                }
            }
            __syncthreads();
        }
        // convergence: off-diagonal vs diagonal mass
        float off = 0.0f, dia = 0.0f;
        for (int i = wy; i < b; i += nwy)
            for (int j = lx; j < b; j += 32) {
                const float v = H[i * ld + j];
                if (i == j) dia += v * v; else off += v * v;
            }
        for (int o = 16; o > 0; o >>= 1) {
            off += __shfl_xor_sync(0xffffffffu, off, o);
            dia += __shfl_xor_sync(0xffffffffu, dia, o);
        }
        if ((tid & 31) == 0) { red[tid >> 5][0] = off; red[tid >> 5][1] = dia; }
        __syncthreads();
        if (tid == 0) {
            float o2 = 0.0f, d2 = 0.0f;
            for (int w = 0; w < nt / 32; ++w) { o2 += red[w][0]; d2 += red[w][1]; }
            // converged: squared off-diagonal norm <= off_rel2 of the
            // diagonal's; or at the FP32 rounding floor: after the first
            // sweeps (the quadratic phase) a sweep no longer halves the
            // off-diagonal mass
            s_done = (o2 <= off_rel2 * d2) || (sweep >= 2 && o2 > 0.25f * prev_off);
            prev_off = o2;
        }
        __syncthreads();
        if (s_done) break;
    }
    // sort descending (ties by index) and write out: U column `rank` = U^T row c
    for (int c = wy; c < b; c += nwy) {
        const float tc = H[c * ld + c];
        int rank = 0;
        for (int o = lx; o < b; o += 32) {
            const float to = H[o * ld + o];
            rank += (to > tc) || (to == tc && o < c);
        }
        for (int o = 16; o > 0; o >>= 1) rank += __shfl_xor_sync(0xffffffffu, rank, o);
        if (lx == 0) theta[rank] = (double)tc;
        for (int i = lx; i < b; i += 32) Uout[i * b + rank] = Ut[c * ldu + i];
    }
}

__global__ void ritz_residual_kernel(const float *__restrict__ W, const float *__restrict__ V, int64_t ld,
                                     int d, const double *__restrict__ theta, int s, float *__restrict__ res) {
    const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= s) return;
    const float th = (float)theta[row];
    float acc = 0.0f;
    for (int j = lane; j < d; j += 32) {
        const float r = W[(int64_t)row * ld + j] - th * V[(int64_t)row * ld + j];
        acc += r * r;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) res[row] = sqrtf(acc);
}

__global__ void residual_rows_kernel(const float *__restrict__ W, const float *__restrict__ V, int64_t ld,
                                     int d, const double *__restrict__ theta, int s,
                                     float *__restrict__ Rm) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)s * d) return;
    const int i = (int)(e / d), j = (int)(e % d);
    Rm[e] = W[(int64_t)i * ld + j] - (float)theta[i] * V[(int64_t)i * ld + j];
}

__global__ void row_norms_kernel(const float *__restrict__ Rm, int d, int s, float *__restrict__ res) {
    const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= s) return;
    float acc = 0.0f;
    for (int j = lane; j < d; j += 32) {
        const float r = Rm[(int64_t)row * d + j];
        acc = fmaf(r, r, acc);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) res[row] = sqrtf(acc);
}

__global__ void canonical_signs_kernel(float *P, int d, int64_t ldp) {
    float *row = P + (int64_t)blockIdx.x * ldp;
    __shared__ float bv[256];
    __shared__ int bi[256];
    float best = -1.0f;
    int idx = 0x7fffffff;
    for (int j = threadIdx.x; j < d; j += blockDim.x) {
        const float a = fabsf(row[j]);
        if (a > best || (a == best && j < idx)) { best = a; idx = j; }
    }
    bv[threadIdx.x] = best;
    bi[threadIdx.x] = idx;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            const float a = bv[threadIdx.x + o];
            const int ia = bi[threadIdx.x + o];
            if (a > bv[threadIdx.x] || (a == bv[threadIdx.x] && ia < bi[threadIdx.x])) {
                bv[threadIdx.x] = a;
                bi[threadIdx.x] = ia;
            }
        }
        __syncthreads();
    }
    const bool flip = row[bi[0]] < 0.0f;
    __syncthreads();
    if (flip)
        for (int j = threadIdx.x; j < d; j += blockDim.x) row[j] = -row[j];
}

__global__ void copy_rows_kernel(const float *__restrict__ src, int64_t lds, float *__restrict__ dst,
                                 int64_t ldd, int rows, int cols) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)rows * cols) return;
    const int64_t r = e / cols, c = e % cols;
    dst[r * ldd + c] = src[r * lds + c];
}

}  // namespace

template <typename TA, typename TB, typename TC, typename TACC>
void gemm(int M, int N, int K, TACC alpha, MatView<TA> A, MatView<TB> B, TACC beta, TC *C,
          int64_t ldc, cudaStream_t st) {
    if (M <= 0 || N <= 0) return;
    dim3 grid((unsigned)ceil_div(N, GT), (unsigned)ceil_div(M, GT), 1);
    gemm_kernel<TA, TB, TC, TACC><<<grid, GNT, 0, st>>>(M, N, K, K > 0 ? K : 1, alpha, A, B, beta,
                                                        C, ldc, 0);
    ADAGIO_CHECK_LAUNCH();
}

template void gemm<float, float, float, float>(int, int, int, float, MatView<float>, MatView<float>,
                                               float, float *, int64_t, cudaStream_t);
template void gemm<float, float, double, double>(int, int, int, double, MatView<float>, MatView<float>,
                                                 double, double *, int64_t, cudaStream_t);
template void gemm<double, double, double, double>(int, int, int, double, MatView<double>,
                                                   MatView<double>, double, double *, int64_t,
                                                   cudaStream_t);
template void gemm<float, __nv_bfloat16, float, float>(int, int, int, float, MatView<float>,
                                                       MatView<__nv_bfloat16>, float, float *,
                                                       int64_t, cudaStream_t);
template void gemm<float, float, double, float>(int, int, int, float, MatView<float>, MatView<float>,
                                                float, double *, int64_t, cudaStream_t);

int64_t splitk_chunks(int64_t K) { return ceil_div(K, kSplitRows); }

void gemm_f64_splitk(int M, int N, int K, MatView<float> A, MatView<float> B, double *C,
                     double *partials, int kchunk, cudaStream_t st) {
    if (M <= 0 || N <= 0) return;
    const int chunks = (int)ceil_div(K, kchunk);
    dim3 grid((unsigned)ceil_div(N, GT), (unsigned)ceil_div(M, GT), (unsigned)chunks);
    gemm_df_kernel<<<grid, GNT, 0, st>>>(M, N, K, kchunk, A, B, partials, N, (int64_t)M * N);
    ADAGIO_CHECK_LAUNCH();
    const int64_t mn = (int64_t)M * N;
    splitk_reduce_f64_kernel<<<(unsigned)ceil_div(mn, 256), 256, 0, st>>>(partials, chunks, mn, C);
    ADAGIO_CHECK_LAUNCH();
}

void gemm_tn_splitk(int M, int N, int64_t K, const float *A, int64_t lda, const float *B,
                    int64_t ldb, float *C, int64_t ldc, float *partials, cudaStream_t st) {
    const int64_t chunks = splitk_chunks(K);
    dim3 grid((unsigned)ceil_div(N, GT), (unsigned)ceil_div(M, GT), (unsigned)chunks);
    MatView<float> a{A, 1, lda};
    MatView<float> b{B, ldb, 1};
    gemm_kernel<float, float, float, float><<<grid, GNT, 0, st>>>(
        M, N, (int)K, kSplitRows, 1.0f, a, b, 0.0f, partials, N, (int64_t)M * N);
    ADAGIO_CHECK_LAUNCH();
    const int64_t total = (int64_t)M * N;
    splitk_reduce_kernel<<<(unsigned)ceil_div(total, 256), 256, 0, st>>>(partials, chunks, M, N, C, ldc);
    ADAGIO_CHECK_LAUNCH();
}

static size_t jacobi_smem(int b) {
    const size_t B = (size_t)((b + 1) & ~1);
    return (B * (B + 1) + B * ((B + 3) & ~(size_t)3)) * sizeof(float) + 16;
}

void linalg_init() {
    const size_t b = kJacobiMax;
    set_max_dyn_smem((const void *)cholesky_kernel, (int)(b * (b + 1) * sizeof(double)));
    set_max_dyn_smem((const void *)trsm_rows_kernel, (int)((b * b + b * kTrsmCols) * sizeof(float)));
    set_max_dyn_smem((const void *)jacobi_kernel, (int)(jacobi_smem(kJacobiMax)));
    set_max_dyn_smem((const void *)trsm_warp_kernel, (int)(b * (b + 1) * sizeof(float)));
    set_max_dyn_smem((const void *)chol_blocked_kernel<float>, (int)kCiSmem);
    set_max_dyn_smem((const void *)chol_blocked_kernel<double>, (int)kCiSmem);
    set_max_dyn_smem((const void *)trsm_blocked_kernel, (int)kTbSmem);
}

template <typename TG>
void cholesky32(const TG *G, int b, float shift_rel, float *R, cudaStream_t st) {
    if (b > kJacobiMax) fail(ADAGIO_E_INVALID_ARG, "internal: Cholesky block %d > %d", b, kJacobiMax);
    cholesky32_kernel<TG><<<1, kCholThreads, 0, st>>>(G, b, shift_rel, R);
    ADAGIO_CHECK_LAUNCH();
}
template void cholesky32<double>(const double *, int, float, float *, cudaStream_t);
template void cholesky32<float>(const float *, int, float, float *, cudaStream_t);

template <typename TG>
void cholesky_blocked(const TG *G, int b, float shift_rel, float *R, float *Dinv, cudaStream_t st) {
    if (b > kJacobiMax) fail(ADAGIO_E_INVALID_ARG, "internal: Cholesky block %d > %d", b, kJacobiMax);
    set_max_dyn_smem((const void *)chol_blocked_kernel<TG>, (int)kCiSmem);
    chol_blocked_kernel<TG><<<1, kCiThreads, kCiSmem, st>>>(G, b, shift_rel, R, Dinv);
    ADAGIO_CHECK_LAUNCH();
}
template void cholesky_blocked<double>(const double *, int, float, float *, float *, cudaStream_t);
template void cholesky_blocked<float>(const float *, int, float, float *, float *, cudaStream_t);

void trsm_blocked(const float *R, const float *Dinv, int b, float *M, int64_t ldm, int d,
                  cudaStream_t st) {
    if (b > kJacobiMax) fail(ADAGIO_E_INVALID_ARG, "internal: TRSM block %d > %d", b, kJacobiMax);
    set_max_dyn_smem((const void *)trsm_blocked_kernel, (int)kTbSmem);
    trsm_blocked_kernel<<<(unsigned)ceil_div(d, kTbCols), kTbThreads, kTbSmem, st>>>(R, Dinv, b, M,
                                                                                  ldm, d);
    ADAGIO_CHECK_LAUNCH();
}

void trsm_warp(const float *R, int b, float *V, int64_t ldv, int d, cudaStream_t st) {
    if (b > kJacobiMax) fail(ADAGIO_E_INVALID_ARG, "internal: TRSM block %d > %d", b, kJacobiMax);
    const size_t smem = (size_t)b * (b + 1) * sizeof(float);
    set_max_dyn_smem((const void *)trsm_warp_kernel, (int)smem);
    trsm_warp_kernel<<<(unsigned)ceil_div(d, 2 * kTrsmWarps), 32 * kTrsmWarps, smem, st>>>(R, b, V, ldv, d);
    ADAGIO_CHECK_LAUNCH();
}

static int device_sms() {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        ADAGIO_CUDA(cudaGetDevice(&dev));
        ADAGIO_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    }
    return sms;
}

void gemm_f32(int M, int N, int K, float alpha, MatView<float> A, MatView<float> B, float beta,
              float *C, int64_t ldc, float *partials, int64_t partial_floats, cudaStream_t st) {
    if (M <= 0 || N <= 0) return;
    const int64_t tiles = ceil_div(M, GT) * ceil_div(N, GT);
    int64_t chunks = std::min<int64_t>(ceil_div(2 * (int64_t)device_sms(), tiles), ceil_div(K, 64));
    if (partials) chunks = std::min<int64_t>(chunks, partial_floats / ((int64_t)M * N));
    if (chunks <= 1 || !partials) {
        gemm<float, float, float, float>(M, N, K, alpha, A, B, beta, C, ldc, st);
        return;
    }
    const int kchunk = (int)(ceil_div(ceil_div(K, chunks), GK) * GK);
    chunks = ceil_div(K, kchunk);
    dim3 grid((unsigned)ceil_div(N, GT), (unsigned)ceil_div(M, GT), (unsigned)chunks);
    gemm_kernel<float, float, float, float><<<grid, GNT, 0, st>>>(M, N, K, kchunk, 1.0f, A, B, 0.0f,
                                                                   partials, N, (int64_t)M * N);
    ADAGIO_CHECK_LAUNCH();
    const int64_t mn = (int64_t)M * N;
    splitk_reduce_ab_kernel<<<(unsigned)ceil_div(mn, 256), 256, 0, st>>>(partials, (int)chunks, M, N,
                                                                       alpha, beta, C, ldc);
    ADAGIO_CHECK_LAUNCH();
}

void cholesky_upper(double *G, int b, double floor_rel, cudaStream_t st) {
    const size_t smem = (size_t)b * (b + 1) * sizeof(double);
    set_max_dyn_smem((const void *)cholesky_kernel, (int)smem);
    cholesky_kernel<<<1, 1024, smem, st>>>(G, b, floor_rel);
    ADAGIO_CHECK_LAUNCH();
}

void trsm_rows(const double *R, int b, float *V, int64_t ldv, int d, cudaStream_t st) {
    const size_t smem = ((size_t)b * b + (size_t)b * kTrsmCols) * sizeof(float);
    set_max_dyn_smem((const void *)trsm_rows_kernel, (int)smem);
    trsm_rows_kernel<<<(unsigned)ceil_div(d, kTrsmCols), kTrsmCols, smem, st>>>(R, b, V, ldv, d);
    ADAGIO_CHECK_LAUNCH();
}

void jacobi_eig(const double *H, int b, double *theta, float *U, int max_sweeps, float off_rel2,
                cudaStream_t st) {
    if (b > kJacobiMax) fail(ADAGIO_E_INVALID_ARG, "internal: Jacobi block %d > %d", b, kJacobiMax);
    const size_t smem = jacobi_smem(b);
    set_max_dyn_smem((const void *)jacobi_kernel, (int)smem);
    jacobi_kernel<<<1, kJacobiThreads, smem, st>>>(H, b, theta, U, max_sweeps, std::max(off_rel2, 1e-12f));
    ADAGIO_CHECK_LAUNCH();
}

void ritz_residuals(const float *W, const float *V, int64_t ld, int d, const double *theta, int s,
                    float *res, cudaStream_t st) {
    if (s <= 0) return;
    ritz_residual_kernel<<<(unsigned)ceil_div(s, 8), 256, 0, st>>>(W, V, ld, d, theta, s, res);
    ADAGIO_CHECK_LAUNCH();
}

void ritz_residuals_projected(const float *W, const float *V, int64_t ld, int d, int b,
                              const double *theta, int s, float *Rm, float *coef, float *partials,
                              int64_t partial_floats, float *res, cudaStream_t st) {
    if (s <= 0) return;
    residual_rows_kernel<<<(unsigned)ceil_div((int64_t)s * d, 256), 256, 0, st>>>(W, V, ld, d, theta,
                                                                                   s, Rm);
    ADAGIO_CHECK_LAUNCH();
    // Rm <- Rm - (Rm V^T) V: the part of each residual outside span(V)
    gemm_f32(s, b, d, 1.0f, MatView<float>{Rm, d, 1}, MatView<float>{V, 1, ld}, 0.0f, coef, b,
             partials, partial_floats, st);
    gemm_f32(s, d, b, -1.0f, MatView<float>{coef, b, 1}, MatView<float>{V, ld, 1}, 1.0f, Rm, d,
             partials, partial_floats, st);
    row_norms_kernel<<<(unsigned)ceil_div(s, 8), 256, 0, st>>>(Rm, d, s, res);
    ADAGIO_CHECK_LAUNCH();
}

void canonical_signs(float *P, int s, int d, int64_t ldp, cudaStream_t st) {
    if (s <= 0) return;
    canonical_signs_kernel<<<s, 256, 0, st>>>(P, d, ldp);
    ADAGIO_CHECK_LAUNCH();
}

void copy_rows(const float *src, int64_t lds, float *dst, int64_t ldd, int rows, int cols,
               cudaStream_t st) {
    const int64_t total = (int64_t)rows * cols;
    if (total <= 0) return;
    copy_rows_kernel<<<(unsigned)ceil_div(total, 256), 256, 0, st>>>(src, lds, dst, ldd, rows, cols);
    ADAGIO_CHECK_LAUNCH();
}

}  // namespace adagio
