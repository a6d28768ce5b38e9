// k nearest neighbours in an embedded space: the applications of the paper's
// Sec. 4.6 (a 10-nearest-neighbour vote on embedded descriptors) and Sec. 4.7
// (a k = 30 nearest-neighbour graph of the embedded points) search the output
// of the map, so a certified embedding is followed by this search.
//
// The answer is exact: for every query q, the k base points b with the
// smallest Euclidean distance ||q - b|| of the FP32 inputs, nearest first,
// ties (equal distances) broken by the smaller base index, query i's own index
// left out when `exclude_self` (the graph of one point set).
//
// Steps, per block of query rows (1024 to 8192 of them, as many as a 2 GiB
// Gram block holds):
//   1. Gram block G = Q_blk B^T on tcgen05 tensor cores (the split-precision
//      GEMM of tcgemm.cu: per-row power-of-two FP16 hi + lo planes, three
//      products per term, FP32 accumulation), rows x nb floats;
//   2. one warp per query row scans its Gram row (each lane loading kUnroll
//      columns ahead of filtering them), forms the approximate squared
//      distances d~ = |q|^2 + |b|^2 - 2 q.b and keeps the 64 smallest (d~, j)
//      in a sorted list (kCand = k_max + 16 candidates);
//   3. the candidates' distances are recomputed exactly from coordinate
//      differences in FP64 and ranked by (distance, index); the first k are
//      the answer when no base point outside the list can beat the k-th:
//      every such point has d~ >= tau (the smallest d~ the list dropped), and
//      |d~ - d| <= c (|q|^2 + |b|^2) with c = 128 u (u = 2^-24; the GEMM's
//      accumulation and split error is about 20 u, the formation of d~ 3 u),
//      so the answer is final when d_k < tau - c (|q|^2 + max |b|^2);
//   4. the rare rows where that test fails are searched again over every base
//      point with exact FP64 distances.
#include "internal.cuh"
#include "tcgemm.cuh"

#include <algorithm>
#include <cmath>
#include <vector>

namespace adagio {

namespace {

constexpr int kMaxK = 48;                 // largest k served
constexpr int kCand = 64;                 // candidates kept per query (two per lane)
constexpr int kBlockQMin = 1024;          // query rows per Gram block: at least
constexpr int kBlockQMax = 8192;          // and at most (one warp per row in the scan)
constexpr size_t kGramBudget = size_t(2) << 30;  // bytes of one FP32 Gram block, at most
constexpr int kUnroll = 8;                // columns a lane loads before filtering them
constexpr int kSelWarps = 8;              // warps (query rows) per selection CTA
constexpr float kDistErr = 128.0f * 5.9604645e-08f;  // c: 128 u

// Squared 2-norm of every row, summed in FP64 (exact products, one rounding
// per addition), rounded to FP32; the largest is returned through *max_bits
// (the bits of a non-negative float order like the float).
__global__ void knn_norms_kernel(const float *__restrict__ Y, int64_t rows, int m, int64_t ld,
                                 float *__restrict__ n2, unsigned *__restrict__ max_bits) {
    const int lane = threadIdx.x & 31;
    const int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (r >= rows) return;
    double acc = 0.0;
    for (int c = lane; c < m; c += 32) {
        const double v = Y[r * ld + c];
        acc = fma(v, v, acc);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) {
        const float f = (float)acc;
        n2[r] = f;
        if (max_bits) atomicMax(max_bits, __float_as_uint(f));
    }
}

// (d, j) comes before (e, l): smaller distance, then smaller index
__device__ __forceinline__ bool key_before(float d, int j, float e, int l) {
    return d < e || (d == e && j < l);
}
__device__ __forceinline__ bool key_before(double d, int j, double e, int l) {
    return d < e || (d == e && j < l);
}

// Inserts (d, j) into a warp's sorted list (ld[0 .. cnt), lj[0 .. cnt)) of at
// most kCand entries, in shared memory; lane l holds slots l and l + 32.  The
// entry the insertion pushes out of a full list is returned through
// (out_d, out_j) (out_d = +inf when none).  Every lane calls it with the same
// (d, j).
template <typename T>
__device__ __forceinline__ void list_insert(T *ld, int *lj, int &cnt, T d, int j, T &out_d) {
    const int lane = threadIdx.x & 31;
    const T v0 = lane < cnt ? ld[lane] : T(0);
    const int j0 = lane < cnt ? lj[lane] : 0;
    const T v1 = lane + 32 < cnt ? ld[lane + 32] : T(0);
    const int j1 = lane + 32 < cnt ? lj[lane + 32] : 0;
    const unsigned b0 = __ballot_sync(0xffffffffu, lane < cnt && key_before(v0, j0, d, j));
    const unsigned b1 = __ballot_sync(0xffffffffu, lane + 32 < cnt && key_before(v1, j1, d, j));
    const int pos = __popc(b0) + __popc(b1);  // entries before (d, j): a prefix
    out_d = T(INFINITY);
    if (cnt == kCand) out_d = __shfl_sync(0xffffffffu, v1, 31);
    __syncwarp();
    if (pos < kCand) {
        // every entry at or after pos moves one slot on (the last one drops out)
        if (lane < cnt && lane >= pos && lane + 1 < kCand) {
            ld[lane + 1] = v0;
            lj[lane + 1] = j0;
        }
        if (lane + 32 < cnt && lane + 32 >= pos && lane + 33 < kCand) {
            ld[lane + 33] = v1;
            lj[lane + 33] = j1;
        }
        __syncwarp();
        if (lane == 0) {
            ld[pos] = d;
            lj[pos] = j;
        }
        if (cnt < kCand) ++cnt;
    } else {
        out_d = d;  // (d, j) itself is not kept
    }
    __syncwarp();
}

struct SelArgs {
    const float *G;          // Gram block: rows q0 .. q0 + rows - 1, ld nb
    const float *Q, *B;      // FP32 inputs
    int64_t ldq, ldb;
    const float *n2q, *n2b;  // squared norms (all queries / all base points)
    const unsigned *n2b_max;
    int64_t q0, rows, nb;
    int m, k, exclude_self;
    int64_t *idx;            // nq x k
    double *d2;              // nq x k
    int64_t *redo;           // rows whose answer is not final (appended)
    unsigned long long *nredo;
};

// The k nearest base points of FP64 exact squared distances among a warp's
// candidate list (cj[0 .. cnt)); writes them out in (distance, index) order
// and returns the k-th distance (or +inf when fewer than k).
__device__ __forceinline__ double rank_and_write(const SelArgs &p, int64_t i, const int *cj,
                                                 double *ed, int cnt) {
    const int lane = threadIdx.x & 31;
    const float *q = p.Q + i * p.ldq;
    for (int c = 0; c < cnt; ++c) {
        const float *b = p.B + (int64_t)cj[c] * p.ldb;
        double acc = 0.0;
        for (int t = lane; t < p.m; t += 32) {
            const double u = (double)q[t] - (double)b[t];
            acc = fma(u, u, acc);
        }
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) ed[c] = acc;
    }
    __syncwarp();
    double dk = INFINITY;
    for (int h = 0; h < 2; ++h) {
        const int c = lane + 32 * h;
        if (c < cnt) {
            int rank = 0;
            for (int o = 0; o < cnt; ++o) rank += key_before(ed[o], cj[o], ed[c], cj[c]) ? 1 : 0;
            if (rank < p.k) {
                p.idx[i * p.k + rank] = cj[c];
                p.d2[i * p.k + rank] = ed[c];
            }
            if (rank == p.k - 1) dk = ed[c];
        }
    }
    for (int o = 16; o > 0; o >>= 1) dk = fmin(dk, __shfl_xor_sync(0xffffffffu, dk, o));
    return dk;
}

__global__ void __launch_bounds__(32 * kSelWarps)
    knn_select_kernel(SelArgs p) {
    __shared__ float s_d[kSelWarps][kCand];
    __shared__ int s_j[kSelWarps][kCand];
    __shared__ double s_e[kSelWarps][kCand];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t r = (int64_t)blockIdx.x * kSelWarps + w;
    if (r >= p.rows) return;
    const int64_t i = p.q0 + r;
    const float *g = p.G + r * p.nb;
    const float nq = p.n2q[i];
    float *ld = s_d[w];
    int *lj = s_j[w];
    int cnt = 0;
    float tau = INFINITY;  // smallest approximate distance not kept (this lane's share)
    // the list's last key: a point must come before it to enter a full list
    float td = INFINITY;
    int tj = 0x7fffffff;
    for (int64_t base = 0; base < p.nb; base += 32 * kUnroll) {
        float d[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const int64_t j = base + 32 * u + lane;
            const bool valid = j < p.nb && !(p.exclude_self && j == i);
            d[u] = valid ? fmaf(-2.0f, __ldg(g + j), __fadd_rn(nq, __ldg(p.n2b + j))) : INFINITY;
        }
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const int jj = (int)(base + 32 * u + lane);
            const bool valid = d[u] < INFINITY;
            const bool want = valid && key_before(d[u], jj, td, tj);
            if (valid && !want) tau = fminf(tau, d[u]);
            unsigned mask = __ballot_sync(0xffffffffu, want);
            if (!mask) continue;
            while (mask) {
                const int l = __ffs(mask) - 1;
                mask &= mask - 1;
                const float dl = __shfl_sync(0xffffffffu, d[u], l);
                const int jl = __shfl_sync(0xffffffffu, jj, l);
                if (cnt == kCand && !key_before(dl, jl, td, tj)) {
                    if (lane == 0) tau = fminf(tau, dl);
                    continue;
                }
                float out;
                list_insert(ld, lj, cnt, dl, jl, out);
                if (lane == 0) tau = fminf(tau, out);
                if (cnt == kCand) {
                    td = ld[kCand - 1];
                    tj = lj[kCand - 1];
                }
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) tau = fminf(tau, __shfl_xor_sync(0xffffffffu, tau, o));
    const double dk = rank_and_write(p, i, lj, s_e[w], cnt);
    if (lane == 0) {
        // points outside the list have exact distance >= tau - c (|q|^2 + max |b|^2)
        const double lower = (double)tau - (double)kDistErr * ((double)nq + (double)__uint_as_float(*p.n2b_max));
        const bool final_ = cnt < p.k ? false : (tau == INFINITY || dk < lower);
        if (!final_) {
            const unsigned long long slot = atomicAdd(p.nredo, 1ull);
            p.redo[slot] = i;
        }
    }
}

// Rows whose list could not be shown final: every base point's exact FP64
// squared distance into `dist` (one row at a time), then the k smallest by
// (distance, index) with the same list routine.
__global__ void knn_exact_dist_kernel(const float *__restrict__ Q, int64_t ldq, const float *__restrict__ B,
                                      int64_t ldb, int64_t i, int64_t nb, int m, double *__restrict__ dist) {
    const int lane = threadIdx.x & 31;
    const int64_t j = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (j >= nb) return;
    const float *q = Q + i * ldq, *b = B + j * ldb;
    double acc = 0.0;
    for (int t = lane; t < m; t += 32) {
        const double u = (double)q[t] - (double)b[t];
        acc = fma(u, u, acc);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) dist[j] = acc;
}

__global__ void knn_exact_select_kernel(const double *__restrict__ dist, int64_t i, int64_t nb, int k,
                                        int exclude_self, int64_t *idx, double *d2) {
    __shared__ double s_d[kCand];
    __shared__ int s_j[kCand];
    const int lane = threadIdx.x & 31;
    int cnt = 0;
    for (int64_t base = 0; base < nb; base += 32) {
        const int64_t j = base + lane;
        const bool valid = j < nb && !(exclude_self && j == i);
        const double d = valid ? dist[j] : INFINITY;
        const double td = cnt == kCand ? s_d[kCand - 1] : INFINITY;
        const int tj = cnt == kCand ? s_j[kCand - 1] : 0x7fffffff;
        unsigned mask = __ballot_sync(0xffffffffu, valid && (cnt < kCand || key_before(d, (int)j, td, tj)));
        while (mask) {
            const int l = __ffs(mask) - 1;
            mask &= mask - 1;
            const double dl = __shfl_sync(0xffffffffu, d, l);
            const int jl = (int)__shfl_sync(0xffffffffu, (unsigned)j, l);
            double out;
            list_insert(s_d, s_j, cnt, dl, jl, out);
        }
    }
    for (int c = lane; c < k && c < cnt; c += 32) {
        idx[i * k + c] = s_j[c];
        d2[i * k + c] = s_d[c];
    }
}

}  // namespace

}  // namespace adagio

using namespace adagio;

extern "C" int adagio_knn(adagio_ctx *ctx, const float *Q, int64_t nq, int64_t ldq, const float *B,
                          int64_t nb, int64_t ldb, int m, int k, int exclude_self, int64_t *idx,
                          double *d2, void *stream) {
    if (!ctx) return ADAGIO_E_INVALID_ARG;
    ctx->last_error.clear();
    try {
        DeviceGuard guard(ctx->device);
        ws_reset(ctx);
        ADAGIO_REQUIRE(Q && B && idx && d2, "null pointer argument");
        ADAGIO_REQUIRE(nq >= 1 && nb >= 1 && nq < (1ll << 31) && nb < (1ll << 31), "nq, nb out of range");
        ADAGIO_REQUIRE(m >= 1 && ldq >= m && ldb >= m, "bad dimension or leading dimensions");
        ADAGIO_REQUIRE(k >= 1 && k <= kMaxK, "k must lie in [1, %d], got %d", kMaxK, k);
        ADAGIO_REQUIRE(k <= nb - (exclude_self ? 1 : 0), "k = %d exceeds the %lld base points available", k,
                       (long long)(nb - (exclude_self ? 1 : 0)));
        cudaStream_t st = (cudaStream_t)stream;
        const bool same = Q == B && ldq == ldb && nq == nb;
        const int Kp = pad64(m);
        const bool out_dev = is_device_ptr(idx, ctx->device) && is_device_ptr(d2, ctx->device);
        // as many query rows per block as 2 GiB of Gram values hold (whole
        // multiples of 1024, up to 8192): more rows keep more scan warps in flight
        const int64_t fit_rows = (int64_t)(kGramBudget / ((size_t)nb * 4)) / kBlockQMin * kBlockQMin;
        const int64_t block_q = std::max<int64_t>(kBlockQMin, std::min<int64_t>(kBlockQMax, fit_rows));
        const int64_t qrows_max = std::min<int64_t>(nq, block_q);
        const size_t part_floats =
            (size_t)std::max<int64_t>(1, tc_gemm_workspace(ctx, (int)qrows_max, (int)nb, Kp, false));
        size_t need = align_up((size_t)nb * ldb * 4, 256) + (same ? 0 : align_up((size_t)nq * ldq * 4, 256));
        need += 2 * align_up((size_t)nb * Kp * 2, 256) + align_up((size_t)nb * 4, 256) * 2;
        if (!same) need += 2 * align_up((size_t)nq * Kp * 2, 256) + align_up((size_t)nq * 4, 256) * 2;
        need += align_up((size_t)qrows_max * nb * 4, 256) + align_up(part_floats * 4, 256);
        need += align_up((size_t)nq * 8, 256) + align_up((size_t)nb * 8, 256) + 4096;
        if (!out_dev) need += align_up((size_t)nq * k * 8, 256) * 2;
        ws_reserve(ctx, need);

        int64_t lb, lq;
        const float *dB = stage_input(ctx, B, nb, m, ldb, &lb, st);
        const float *dQ = same ? dB : stage_input(ctx, Q, nq, m, ldq, &lq, st);
        if (same) lq = lb;
        // split planes and squared norms
        SplitPlanes pb, pq;
        uint16_t *bh = ws_array<uint16_t>(ctx, (size_t)nb * Kp), *bl = ws_array<uint16_t>(ctx, (size_t)nb * Kp);
        float *bs = ws_array<float>(ctx, (size_t)nb), *n2b = ws_array<float>(ctx, (size_t)nb);
        unsigned *n2b_max = ws_array<unsigned>(ctx, 4);
        unsigned long long *nredo = reinterpret_cast<unsigned long long *>(n2b_max + 2);
        ADAGIO_CUDA(cudaMemsetAsync(n2b_max, 0, 16, st));
        split_rows(dB, nb, m, lb, bh, bl, bs, st);
        pb.hi = bh;
        pb.lo = bl;
        pb.rows = nb;
        pb.Kp = Kp;
        pb.scale = bs;
        pb.scale_stride = 1;
        knn_norms_kernel<<<(unsigned)ceil_div(nb, 8), 256, 0, st>>>(dB, nb, m, lb, n2b, n2b_max);
        ADAGIO_CHECK_LAUNCH();
        const float *n2q = n2b;
        if (same) {
            pq = pb;
        } else {
            uint16_t *qh = ws_array<uint16_t>(ctx, (size_t)nq * Kp), *ql = ws_array<uint16_t>(ctx, (size_t)nq * Kp);
            float *qs = ws_array<float>(ctx, (size_t)nq), *nqq = ws_array<float>(ctx, (size_t)nq);
            split_rows(dQ, nq, m, lq, qh, ql, qs, st);
            pq.hi = qh;
            pq.lo = ql;
            pq.rows = nq;
            pq.Kp = Kp;
            pq.scale = qs;
            pq.scale_stride = 1;
            knn_norms_kernel<<<(unsigned)ceil_div(nq, 8), 256, 0, st>>>(dQ, nq, m, lq, nqq, n2b_max + 1);
            ADAGIO_CHECK_LAUNCH();
            n2q = nqq;
        }
        float *G = ws_array<float>(ctx, (size_t)qrows_max * nb);
        float *part = ws_array<float>(ctx, part_floats);
        int64_t *redo = ws_array<int64_t>(ctx, (size_t)nq);
        double *scratch = ws_array<double>(ctx, (size_t)nb);
        int64_t *didx = out_dev ? idx : ws_array<int64_t>(ctx, (size_t)nq * k);
        double *dd2 = out_dev ? d2 : ws_array<double>(ctx, (size_t)nq * k);

        SelArgs a;
        a.G = G;
        a.Q = dQ;
        a.B = dB;
        a.ldq = lq;
        a.ldb = lb;
        a.n2q = n2q;
        a.n2b = n2b;
        a.n2b_max = n2b_max;
        a.nb = nb;
        a.m = m;
        a.k = k;
        a.exclude_self = exclude_self ? 1 : 0;
        a.idx = didx;
        a.d2 = dd2;
        a.redo = redo;
        a.nredo = nredo;
        for (int64_t q0 = 0; q0 < nq; q0 += block_q) {
            const int64_t rows = std::min<int64_t>(block_q, nq - q0);
            SplitPlanes blk = pq;
            blk.hi = pq.hi + q0 * Kp;
            blk.lo = pq.lo + q0 * Kp;
            blk.rows = rows;
            blk.scale = pq.scale + q0;
            tc_gemm(ctx, blk, pb, (int)rows, (int)nb, nullptr, G, nb, false, part, ctx->dev_status, st);
            a.q0 = q0;
            a.rows = rows;
            knn_select_kernel<<<(unsigned)ceil_div(rows, kSelWarps), 32 * kSelWarps, 0, st>>>(a);
            ADAGIO_CHECK_LAUNCH();
        }
        // rows whose candidate list could not be shown final: an exact search
        unsigned long long hred = 0;
        unsigned hmax[2] = {0u, 0u};
        ADAGIO_CUDA(cudaMemcpyAsync(&hred, nredo, sizeof(hred), cudaMemcpyDeviceToHost, st));
        ADAGIO_CUDA(cudaMemcpyAsync(hmax, n2b_max, sizeof(hmax), cudaMemcpyDeviceToHost, st));
        ADAGIO_CUDA(cudaStreamSynchronize(st));
        // a NaN or infinite squared norm (bits at or above those of +inf)
        if (hmax[0] >= 0x7f800000u || hmax[1] >= 0x7f800000u)
            fail(ADAGIO_E_NONFINITE, "input holds NaN or Inf (or values whose squared norm overflows)");
        if (hred > 0) {
            std::vector<int64_t> rows((size_t)hred);
            ADAGIO_CUDA(cudaMemcpy(rows.data(), redo, hred * sizeof(int64_t), cudaMemcpyDeviceToHost));
            for (int64_t i : rows) {
                knn_exact_dist_kernel<<<(unsigned)ceil_div(nb, 8), 256, 0, st>>>(dQ, lq, dB, lb, i, nb, m,
                                                                                 scratch);
                ADAGIO_CHECK_LAUNCH();
                knn_exact_select_kernel<<<1, 32, 0, st>>>(scratch, i, nb, k, a.exclude_self, didx, dd2);
                ADAGIO_CHECK_LAUNCH();
            }
        }
        ctx->last_knn_redo = (int64_t)hred;
        if (!out_dev) {
            ADAGIO_CUDA(cudaMemcpyAsync(idx, didx, (size_t)nq * k * 8, cudaMemcpyDeviceToHost, st));
            ADAGIO_CUDA(cudaMemcpyAsync(d2, dd2, (size_t)nq * k * 8, cudaMemcpyDeviceToHost, st));
        }
        check_device_status(ctx, st);  // synchronises
        return ADAGIO_OK;
    } catch (const Error &e) {
        ctx->last_error = e.msg;
        return e.code;
    } catch (...) {
        ctx->last_error = "unknown failure";
        return ADAGIO_E_CUDA;
    }
}

extern "C" int64_t adagio_knn_last_exact_rows(const adagio_ctx *ctx) { return ctx ? ctx->last_knn_redo : -1; }
