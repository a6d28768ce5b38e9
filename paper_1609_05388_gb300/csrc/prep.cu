// K0: centring and packing of a point matrix for the all-pairs tiles.
//
// PCA works on zero-centred data (Sec. 2); the certificate also centres both
// X and Y before forming Gram tiles, because Eq. 2 depends only on
// differences and centring shrinks ||x||^2 + ||y||^2 - 2 x.y cancellation.
//
// Outputs (all rows padded to a multiple of the tile height with zeros):
//   mu    column means (FP64 accumulation, stored FP32)
//   c32   FP32 centred copy, leading dimension Kp32 (SIMT tiles)
//   hi/lo 2-term split planes of s * (x - mu), 16-bit, leading dimension Kp16,
//         s a power of two chosen so that max |s (x - mu)| <= 2^14 (FP16 range)
//   rs    per-row statistics for the pair error bound
//   flags bit 0 set when any input element is NaN or Inf
#include "internal.cuh"
#include "cert_common.cuh"
#include "prep.cuh"

namespace adagio {

namespace {

// Error-free sum of two floats (TwoSum, Knuth TAOCP vol. 2, 4.2.2): s + e = a + b.
__device__ __forceinline__ void two_sum_f(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bp = __fsub_rn(s, a);
    const float ap = __fsub_rn(s, bp);
    e = __fadd_rn(__fsub_rn(a, ap), __fsub_rn(b, bp));
}

// Column sums of a chunk of rows.  Each thread keeps an unevaluated
// double-float sum (hi + lo, TwoSum per element): about 2^-44 relative per
// step, FP64-grade without the slow FP64 pipe; the 8 partial sums of a column
// are then added in FP64.
__global__ void colsum_partial_kernel(const float *__restrict__ X, int64_t n, int K, int64_t ld,
                                      int64_t rows_per_chunk, double *__restrict__ part) {
    const int c = blockIdx.x * 32 + threadIdx.x;
    const int64_t r0 = (int64_t)blockIdx.y * rows_per_chunk;
    const int64_t r1 = min(n, r0 + rows_per_chunk);
    float hi = 0.0f, lo = 0.0f;
    if (c < K)
        for (int64_t r = r0 + threadIdx.y; r < r1; r += blockDim.y) {
            float s, e;
            two_sum_f(hi, __ldg(X + r * ld + c), s, e);
            hi = s;
            lo = __fadd_rn(lo, e);
        }
    __shared__ double sh[8][33];
    sh[threadIdx.y][threadIdx.x] = (double)hi + (double)lo;
    __syncthreads();
    if (threadIdx.y == 0 && c < K) {
        double t = 0.0;
        for (int y = 0; y < 8; ++y) t += sh[y][threadIdx.x];
        part[(int64_t)blockIdx.y * K + c] = t;
    }
}

__global__ void colmean_kernel(const double *__restrict__ part, int chunks, int K, int64_t n,
                               float *__restrict__ mu) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= K) return;
    double t = 0.0;
    for (int q = 0; q < chunks; ++q) t += part[(int64_t)q * K + c];
    mu[c] = (float)(t / (double)n);
}

// One warp per row: centre, FP32 copy, norms, |max|, finiteness.  The squared
// 2-norm is a double-float sum of exact squares (FMA TwoProduct, TwoSum), so
// it is correct to about one FP32 rounding without the slow FP64 pipe.  The
// 4-norm feeds only a bound coefficient: an FP32 sum of fourth powers, taken
// 2^-10 high, while the row's largest |x| lies in [1e-8, 1e8] (no overflow, and
// what underflows is below 1e-6 of the sum); outside that range the upper
// bound ||x||_4 <= sqrt(||x||_inf ||x||_2).
__global__ void rowprep_kernel(const float *__restrict__ X, int64_t n, int64_t n_pad, int K,
                               int64_t ld, const float *__restrict__ mu, float *__restrict__ c32,
                               int Kp32, RowStat *__restrict__ rs, float s4, float s1,
                               unsigned *__restrict__ amax_bits, unsigned *__restrict__ flags) {
    const int lane = threadIdx.x & 31;
    const int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (r >= n_pad) return;
    float h2 = 0.0f, l2 = 0.0f, n4 = 0.0f;
    float amax = 0.0f;
    bool bad = false;
    if (r < n) {
        for (int k = lane; k < K; k += 32) {
            const float x = __ldg(X + r * ld + k);
            bad |= !isfinite(x);
            const float xc = __fsub_rn(x, __ldg(mu + k));
            amax = fmaxf(amax, fabsf(xc));
            const float p = __fmul_rn(xc, xc);
            const float pe = __fmaf_rn(xc, xc, -p);  // xc^2 = p + pe exactly
            float s, e;
            two_sum_f(h2, p, s, e);
            h2 = s;
            l2 = __fadd_rn(l2, __fadd_rn(e, pe));
            n4 = __fmaf_rn(p, p, n4);
            if (c32) c32[r * Kp32 + k] = xc;
        }
    }
    if (c32) {
        int k0 = (r < n) ? K : 0;
        for (int k = k0 + lane; k < Kp32; k += 32) c32[r * Kp32 + k] = 0.0f;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const float oh = __shfl_xor_sync(0xffffffffu, h2, o), ol = __shfl_xor_sync(0xffffffffu, l2, o);
        float s, e;
        two_sum_f(h2, oh, s, e);
        h2 = s;
        l2 = __fadd_rn(__fadd_rn(l2, ol), e);
        n4 += __shfl_xor_sync(0xffffffffu, n4, o);
        amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    }
    unsigned anybad = __ballot_sync(0xffffffffu, bad);
    if (lane == 0) {
        RowStat st;
        const float n2 = __fadd_rn(h2, l2);
        st.n2 = n2;
        const bool in_range = amax >= 1e-8f && amax <= 1e8f;
        st.q4 = s4 * (in_range ? sqrtf(sqrtf(n4 * (1.0f + 9.765625e-4f))) : sqrtf(amax * sqrtf(n2)));
        st.q1 = s1 * sqrtf(n2);
        st.pad = 0.0f;
        rs[r] = st;
        if (amax > 0.0f) atomicMax(amax_bits, __float_as_uint(amax));
        if (anybad) atomicOr(flags, 1u);
    }
}

// 2-term split of s*(x - mu) into 16-bit planes; 8 consecutive elements per
// thread so that every store is a 16-byte vector.
template <bool FP16>
__global__ void split_kernel(const float *__restrict__ X, int64_t n, int64_t n_pad, int K,
                             int64_t ld, const float *__restrict__ mu,
                             const unsigned *__restrict__ amax_bits, uint16_t *__restrict__ hi,
                             uint16_t *__restrict__ lo, int Kp16, float *__restrict__ scale_out) {
    const int64_t groups_per_row = Kp16 / 8;
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n_pad * groups_per_row) return;
    const int64_t r = g / groups_per_row;
    const int k0 = (int)(g % groups_per_row) * 8;
    float amax = __uint_as_float(*amax_bits);
    float s = 1.0f;
    if (FP16 && amax > 0.0f) {
        int e = (int)floorf(log2f(16384.0f / amax));
        e = max(-100, min(e, 100));
        s = ldexpf(1.0f, e);
        // guard the rounding of log2f: keep max |s x| <= 2^14
        while (amax * s > 16384.0f) s *= 0.5f;
    }
    if (g == 0) *scale_out = s;
    uint16_t h[8], l[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        int k = k0 + q;
        float v = 0.0f;
        if (r < n && k < K) v = __fmul_rn(__fsub_rn(X[r * ld + k], mu[k]), s);
        if (FP16) {
            __half hh = __float2half_rn(v);
            __half ll = __float2half_rn(__fsub_rn(v, __half2float(hh)));
            h[q] = __half_as_ushort(hh);
            l[q] = __half_as_ushort(ll);
        } else {
            __nv_bfloat16 hh = __float2bfloat16_rn(v);
            __nv_bfloat16 ll = __float2bfloat16_rn(__fsub_rn(v, __bfloat162float(hh)));
            h[q] = __bfloat16_as_ushort(hh);
            l[q] = __bfloat16_as_ushort(ll);
        }
    }
    uint4 vh, vl;
    vh.x = h[0] | ((unsigned)h[1] << 16); vh.y = h[2] | ((unsigned)h[3] << 16);
    vh.z = h[4] | ((unsigned)h[5] << 16); vh.w = h[6] | ((unsigned)h[7] << 16);
    vl.x = l[0] | ((unsigned)l[1] << 16); vl.y = l[2] | ((unsigned)l[3] << 16);
    vl.z = l[4] | ((unsigned)l[5] << 16); vl.w = l[6] | ((unsigned)l[7] << 16);
    *reinterpret_cast<uint4 *>(hi + r * Kp16 + k0) = vh;
    *reinterpret_cast<uint4 *>(lo + r * Kp16 + k0) = vl;
}

}  // namespace

BoundModel bound_model(int precision, int K) {
    // Coefficients of the pair error bound (cert_common.cuh).
    //  * products (c4): the split arithmetic drops lo*lo and the residual
    //    beyond hi + lo; the relative error of one term has an RMS of 3.2e-6
    //    (BF16) or 5.4e-8 (FP16, power-of-two scaled) and averages over the K
    //    terms, hence the 4-norm form; eight (BF16) to sixteen (FP16) RMS.
    //  * accumulation (cacc, times ||a||_2 ||b||_2):
    //      FP32 SIMT: FMA chains of 32 terms, each added into the running
    //      sum (cert_simt.cu), a worst-case bound of
    //      (32 + ceil(K / 32) + 1) u |a| |b| (round-to-nearest IEEE steps);
    //      tensor cores: the FP32 accumulator truncates (up to one unit in the
    //      last place per MMA, observed about half on average); each 64-wide
    //      K chunk ends with 4 full-size MMAs (<= 4 * 2^-23 of the chunk's
    //      absolute Gram, which sums to <= ||a|| ||b|| over the chunks) and the
    //      chunks are added in FP32 with round to nearest (<= 2^-24 of the
    //      running sum per chunk).
    //  * FP16x3 is a worst-case bound under one hardware assumption: the
    //    FP16 products are exact, the dropped split terms (lo.lo and the
    //    residual beyond hi + lo, at most 3 * 2^-22 |a_k b_k| per term) sum to
    //    at most 12u |a| |b| (Cauchy-Schwarz), each of the 4 full-size MMAs of
    //    a chunk loses less than 2 units in the last place of its result
    //    (16u of the chunk's sum of |a_k b_k|), and the chunk sums are added
    //    with round to nearest (u per chunk), in all at most
    //    (41 + chunks - 13) u |a| |b|, within cacc (n2_a + n2_b) >= 2 cacc |a| |b|.
    //  * BF16x3 rests on a statistical term (the RMS error of the products),
    //    multiplied by a safety factor of 4.5 chosen so that over a strided
    //    1 % of the tiles of the 60 000 x 784 and 200 000 x 2048 launches the
    //    largest |error| / bound is at most 1/4: a calibrated bound keeps a
    //    fourfold margin.  tests/test_gpu_bounds.py measures all three.
    BoundModel bm;
    const float u = 5.9604645e-08f;  // 2^-24
    if (precision == ADAGIO_PREC_FP32) {
        bm.c4 = 0.0f;
        bm.cacc = (33.0f + ceilf(fmaxf((float)K, 1.0f) / 32.0f)) * u;
    } else {
        const float safety = precision == ADAGIO_PREC_FP16X3 ? 1.0f : 4.5f;
        bm.c4 = safety * (precision == ADAGIO_PREC_FP16X3 ? 9.0e-7f : 2.6e-5f);
        const float chunks = fmaxf((float)K / 64.0f, 1.0f);
        bm.cacc = safety * (8.0f * u + chunks * u);
    }
    return bm;
}

void prep_matrix(adagio_ctx *ctx, const float *X, int64_t n, int K, int64_t ld, int precision,
                 bool want_c32, bool want_split, PrepMat &pm, unsigned *flags, cudaStream_t st) {
    pm.n = n;
    pm.K = K;
    pm.n_pad = pad_rows(n);
    pm.Kp32 = (int)align_up((size_t)K, 8);
    pm.Kp16 = (int)align_up((size_t)K, 64);
    pm.mu = ws_array<float>(ctx, K);
    pm.rs = ws_array<RowStat>(ctx, pm.n_pad);
    pm.c32 = want_c32 ? ws_array<float>(ctx, (size_t)pm.n_pad * pm.Kp32) : nullptr;
    pm.hi = want_split ? ws_array<uint16_t>(ctx, (size_t)pm.n_pad * pm.Kp16) : nullptr;
    pm.lo = want_split ? ws_array<uint16_t>(ctx, (size_t)pm.n_pad * pm.Kp16) : nullptr;
    pm.scale = ws_array<float>(ctx, 1);
    unsigned *amax = ws_array<unsigned>(ctx, 1);
    pm.amax = amax;
    ADAGIO_CUDA(cudaMemsetAsync(amax, 0, sizeof(unsigned), st));

    const int64_t rows_per_chunk = 2048;
    const int chunks = (int)ceil_div(n, rows_per_chunk);
    double *part = ws_array<double>(ctx, (size_t)chunks * K);
    colsum_partial_kernel<<<dim3((unsigned)ceil_div(K, 32), chunks), dim3(32, 8), 0, st>>>(
        X, n, K, ld, rows_per_chunk, part);
    ADAGIO_CHECK_LAUNCH();
    colmean_kernel<<<(unsigned)ceil_div(K, 256), 256, 0, st>>>(part, chunks, K, n, pm.mu);
    ADAGIO_CHECK_LAUNCH();

    BoundModel bm = bound_model(precision, want_split ? pm.Kp16 : pm.Kp32);
    pm.bm = bm;
    const float s4 = sqrtf(2.0f * bm.c4), s1 = sqrtf(2.0f * bm.cacc);
    rowprep_kernel<<<(unsigned)ceil_div(pm.n_pad, 8), 256, 0, st>>>(
        X, n, pm.n_pad, K, ld, pm.mu, pm.c32, pm.Kp32, pm.rs, s4, s1, amax, flags);
    ADAGIO_CHECK_LAUNCH();
    if (want_split) {
        const int64_t groups = pm.n_pad * (pm.Kp16 / 8);
        const unsigned blocks = (unsigned)ceil_div(groups, 256);
        if (precision == ADAGIO_PREC_BF16X3)
            split_kernel<false><<<blocks, 256, 0, st>>>(X, n, pm.n_pad, K, ld, pm.mu, amax, pm.hi,
                                                        pm.lo, pm.Kp16, pm.scale);
        else
            split_kernel<true><<<blocks, 256, 0, st>>>(X, n, pm.n_pad, K, ld, pm.mu, amax, pm.hi,
                                                       pm.lo, pm.Kp16, pm.scale);
        ADAGIO_CHECK_LAUNCH();
    }
}

}  // namespace adagio
