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

constexpr int kJacobiThreads = 512;

__global__ void __launch_bounds__(kJacobiThreads) jacobi_kernel(const double *__restrict__ Hin, int b,
                                                                double *__restrict__ theta,
                                                                float *__restrict__ Uout,
                                                                int max_sweeps) {
    extern __shared__ float sm[];
    const int ld = b + 1;
    float *H = sm;                 // [b][ld]
    float *U = sm + b * ld;        // [b][ld]
    __shared__ float cs[kJacobiMax / 2 + 1], sn[kJacobiMax / 2 + 1];
    __shared__ int pp[kJacobiMax / 2 + 1], qq[kJacobiMax / 2 + 1];
    __shared__ float red[kJacobiThreads / 32][2];
    __shared__ int s_done;
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int e = tid; e < b * b; e += nt) {
        const int i = e / b, j = e % b;
        H[i * ld + j] = (float)(0.5 * (Hin[i * b + j] + Hin[j * b + i]));
        U[i * ld + j] = (i == j) ? 1.0f : 0.0f;
    }
    const int B = (b + 1) & ~1;   // even number of players (index b is a dummy when b is odd)
    const int half = B / 2;
    __syncthreads();
    for (int sweep = 0; sweep < max_sweeps; ++sweep) {
        for (int r = 0; r < B - 1; ++r) {
            if (tid < half) {
                int p, q;
                if (tid == 0) { p = r; q = B - 1; }
                else { p = (r + tid) % (B - 1); q = (r - tid + (B - 1)) % (B - 1); }
                if (p > q) { int t = p; p = q; q = t; }
                float c = 1.0f, s = 0.0f;
                if (q < b) {
                    const float apq = H[p * ld + q];
                    if (apq != 0.0f) {
                        const float app = H[p * ld + p], aqq = H[q * ld + q];
                        const float tau = (aqq - app) / (2.0f * apq);
                        const float t = (tau >= 0.0f ? 1.0f : -1.0f) / (fabsf(tau) + sqrtf(1.0f + tau * tau));
                        c = rsqrtf(1.0f + t * t);
                        s = t * c;
                    }
                }
                pp[tid] = p; qq[tid] = q; cs[tid] = c; sn[tid] = s;
            }
            __syncthreads();
            // rows: H <- J^T H
            for (int e = tid; e < half * b; e += nt) {
                const int k = e / b, j = e % b;
                const int p = pp[k], q = qq[k];
                if (q >= b) continue;
                const float c = cs[k], s = sn[k];
                const float hp = H[p * ld + j], hq = H[q * ld + j];
                H[p * ld + j] = c * hp - s * hq;
                H[q * ld + j] = s * hp + c * hq;
            }
            __syncthreads();
            // columns: H <- H J, U <- U J
            for (int e = tid; e < half * b; e += nt) {
                const int k = e % half, i = e / half;
                const int p = pp[k], q = qq[k];
                if (q >= b) continue;
                const float c = cs[k], s = sn[k];
                const float hp = H[i * ld + p], hq = H[i * ld + q];
                H[i * ld + p] = c * hp - s * hq;
                H[i * ld + q] = s * hp + c * hq;
                const float up = U[i * ld + p], uq = U[i * ld + q];
                U[i * ld + p] = c * up - s * uq;
                U[i * ld + q] = s * up + c * uq;
            }
            __syncthreads();
        }
        // convergence: off-diagonal vs diagonal mass
        float off = 0.0f, dia = 0.0f;
        for (int e = tid; e < b * b; e += nt) {
            const int i = e / b, j = e % b;
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
            s_done = o2 <= 1e-12f * d2;   // off-diagonal norm <= 1e-6 of the diagonal's
        }
        __syncthreads();
        if (s_done) break;
    }
    // sort descending (ties by index) and write out
    for (int c = tid; c < b; c += nt) {
        const float tc = H[c * ld + c];
        int rank = 0;
        for (int o = 0; o < b; ++o) {
            const float to = H[o * ld + o];
            rank += (to > tc) || (to == tc && o < c);
        }
        theta[rank] = (double)tc;
        for (int i = 0; i < b; ++i) Uout[i * b + rank] = U[i * ld + c];
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
    gemm_kernel<float, float, double, double><<<grid, GNT, 0, st>>>(
        M, N, K, kchunk, 1.0, A, B, 0.0, partials, N, (int64_t)M * N);
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

void embed_gemm(const float *X, int64_t ldx, int64_t n, int d, const float *A, int64_t lda, int m,
                float *Y, int64_t ldy, cudaStream_t st) {
    // row blocks of at most 2^20 rows keep every index in int range
    for (int64_t r0 = 0; r0 < n; r0 += (1 << 20)) {
        const int rows = (int)std::min<int64_t>(n - r0, 1 << 20);
        gemm<float, float, float, float>(rows, m, d, 1.0f, MatView<float>{X + r0 * ldx, ldx, 1},
                                         MatView<float>{A, 1, lda}, 0.0f, Y + r0 * ldy, ldy, st);
    }
}

void linalg_init() {
    const size_t b = kJacobiMax;
    set_max_dyn_smem((const void *)cholesky_kernel, (int)(b * (b + 1) * sizeof(double)));
    set_max_dyn_smem((const void *)trsm_rows_kernel, (int)((b * b + b * kTrsmCols) * sizeof(float)));
    set_max_dyn_smem((const void *)jacobi_kernel, (int)(2 * b * (b + 1) * sizeof(float)));
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

void jacobi_eig(const double *H, int b, double *theta, float *U, int max_sweeps, cudaStream_t st) {
    if (b > kJacobiMax) fail(ADAGIO_E_INVALID_ARG, "internal: Jacobi block %d > %d", b, kJacobiMax);
    const size_t smem = (size_t)2 * b * (b + 1) * sizeof(float);
    set_max_dyn_smem((const void *)jacobi_kernel, (int)smem);
    jacobi_kernel<<<1, kJacobiThreads, smem, st>>>(H, b, theta, U, max_sweeps);
    ADAGIO_CHECK_LAUNCH();
}

void ritz_residuals(const float *W, const float *V, int64_t ld, int d, const double *theta, int s,
                    float *res, cudaStream_t st) {
    if (s <= 0) return;
    ritz_residual_kernel<<<(unsigned)ceil_div(s, 8), 256, 0, st>>>(W, V, ld, d, theta, s, res);
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
