// Multi-candidate certificate of JL prefixes: several target dimensions of
// Algorithm 1 certified in one pass over the pair tiles.
//
// For a fixed PCA part P (s rows) and JL rows g_1 .. g_k (Lemma 2's +-1 rows),
// the map with the first kc JL rows scales them by 1/sqrt(kc), so its squared
// JL coordinates are k / kc times the first kc squared JL coordinates of the
// k-row map: with Y = [P x ; S_k (I - P^T P) x] (the k-row map's embedding),
// the candidate's squared distance is
//     |dP|^2 + (k / kc) |dJ[:kc]|^2,
// and the Gram sums of the PCA part and of the JL prefixes come out of one
// pass of the tensor tiles: the prefixes end at 64-column chunk boundaries (kc
// a multiple of 64, or k itself).  The full certificate (histogram, mean,
// maximum) is computed for the k-row map; every listed prefix gets a verdict
// from bounds on each pair's distortion: it passes when every pair certainly
// has distortion <= eps, fails when some pair certainly exceeds eps, and is
// left open when the bound of some pair straddles eps (the caller certifies
// that candidate in full).
#include "internal.cuh"
#include "cert.cuh"
#include "tcgemm.cuh"
#include "prep.cuh"
#include "api_guard.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

namespace adagio {

namespace {

// Y' = [Y's PCA part | zeros up to column jo | Y's JL part], row stride ldo.
__global__ void prefix_layout_kernel(const float *__restrict__ Y, int64_t n, int64_t ldy, int s, int jo,
                                     int k, float *__restrict__ out, int64_t ldo) {
    const int64_t r = blockIdx.x;  // rows in x: up to 2^31 - 1 blocks
    const int c = blockIdx.y * blockDim.x + threadIdx.x;
    if (r >= n || c >= ldo) return;
    float v = 0.0f;
    if (c < s)
        v = Y[r * ldy + c];
    else if (c >= jo && c < jo + k)
        v = Y[r * ldy + s + (c - jo)];
    out[r * ldo + c] = v;
}

// The exact distortion (Eq. 2) of queued pair e = (i, j, candidate) under its
// candidate map, one warp per pair: squared differences of the FP32 rows in
// FP64 (differences of two FP32 values are exact in FP64), dy2 = |dP|^2 +
// (k / kc) |dJ[:kc]|^2.  -1 marks x_i == x_j (excluded, as in the certificate).
__global__ void prefix_recompute_kernel(const float *__restrict__ X, int64_t ldx, int d,
                                        const float *__restrict__ Yp, int64_t ldo, int s, int jo, int k,
                                        int4 kc4, const int4 *__restrict__ cq, long long nq,
                                        double *__restrict__ out) {
    const long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= nq) return;
    const int4 e = cq[w];
    const int kc = e.z == 0 ? kc4.x : (e.z == 1 ? kc4.y : (e.z == 2 ? kc4.z : kc4.w));
    const float *xi = X + (int64_t)e.x * ldx, *xj = X + (int64_t)e.y * ldx;
    const float *yi = Yp + (int64_t)e.x * ldo, *yj = Yp + (int64_t)e.y * ldo;
    double sx = 0.0, sp = 0.0, sj = 0.0;
    for (int t = lane; t < d; t += 32) {
        const double v = (double)xi[t] - (double)xj[t];
        sx = fma(v, v, sx);
    }
    for (int t = lane; t < s; t += 32) {
        const double v = (double)yi[t] - (double)yj[t];
        sp = fma(v, v, sp);
    }
    for (int t = lane; t < kc; t += 32) {
        const double v = (double)yi[jo + t] - (double)yj[jo + t];
        sj = fma(v, v, sj);
    }
    for (int o = 16; o > 0; o >>= 1) {
        sx += __shfl_xor_sync(0xffffffffu, sx, o);
        sp += __shfl_xor_sync(0xffffffffu, sp, o);
        sj += __shfl_xor_sync(0xffffffffu, sj, o);
    }
    if (lane == 0) {
        const double dy2 = fma((double)k / (double)kc, sj, sp);
        out[w] = sx == 0.0 ? -1.0 : fabs(sqrt(dy2 / sx) - 1.0);
    }
}

struct CandRecord {  // the device's per-warp verdict record (CandPartial)
    float rmax_hi, rmax_lo, rmin_lo, rmin_hi;
    unsigned long long certain, open;
};
static_assert(sizeof(CandRecord) == 32, "record layout");

}  // namespace

}  // namespace adagio

using namespace adagio;

extern "C" int adagio_distortion_prefixes(adagio_ctx *ctx, const float *X, int64_t n, int d, int64_t ldx,
                                          const float *Y, int s, int k, int64_t ldy, double eps,
                                          const int *kc, int count, int precision, adagio_cert *full,
                                          adagio_prefix_cert *out, void *stream) {
    API_BEGIN(ctx)
    ADAGIO_REQUIRE(X && Y && full && kc && out, "null pointer argument");
    ADAGIO_REQUIRE(n >= 2 && n < (1ll << 31) - 256, "n = %lld out of range [2, 2^31)", (long long)n);
    ADAGIO_REQUIRE(d >= 1 && ldx >= d, "bad d or ldx");
    ADAGIO_REQUIRE(s >= 1 && k >= 1 && ldy >= (int64_t)s + k, "need s >= 1, k >= 1, ldy >= s + k");
    ADAGIO_REQUIRE(count >= 1 && count <= 4, "1 to 4 candidates, got %d", count);
    // the JL part starts at a 64-column boundary (prefixes of 64-multiples)
    // or where its end is one (prefixes k, k - 64, k - 128, ...)
    bool mult64 = true, from_k = true;
    for (int c = 0; c < count; ++c) {
        ADAGIO_REQUIRE(kc[c] >= 1 && kc[c] <= k, "candidate %d keeps %d JL rows: need 1 <= kc <= k = %d", c,
                       kc[c], k);
        mult64 &= kc[c] % 64 == 0 || kc[c] == k;
        from_k &= (k - kc[c]) % 64 == 0;
    }
    ADAGIO_REQUIRE(mult64 || from_k,
                   "the prefixes must all be multiples of 64 (or k), or all differ from k by multiples of 64");
    ADAGIO_REQUIRE(precision == ADAGIO_PREC_FP16X3 || precision == ADAGIO_PREC_BF16X3,
                   "the multi-candidate pass runs on the tensor-core tiles (FP16x3 or BF16x3)");
    ADAGIO_REQUIRE(std::isfinite(eps) && eps > 0.0 && eps < 1.0, "eps must lie in (0, 1), got %g", eps);
    cudaStream_t st = (cudaStream_t)stream;
    const int s_pad = pad64(s);
    const int jo = mult64 ? s_pad : s_pad + (64 - k % 64) % 64;
    const int Kt = jo + k;
    const int64_t ldo = (int64_t)align_up((size_t)Kt, 4);
    const int64_t n_pad = pad_rows(n);
    const int slots = cert_tc_ctas(ctx, n) * cert_tc_slots_per_cta();
    const size_t rec_bytes = (size_t)slots * count * sizeof(CandRecord);
    const unsigned long long cqcap = 1ull << 18;  // open pairs the exact recompute takes
    size_t need = stage_aligned_bytes(ctx, X, n, d, ldx) + stage_aligned_bytes(ctx, Y, n, s + k, ldy) +
                  align_up((size_t)n * ldo * 4, 256) + align_up((size_t)count * n_pad * 16, 256) +
                  align_up(rec_bytes, 256) + certify_bytes(ctx, n, d, Kt, precision) +
                  align_up(cqcap * 16, 256) + align_up(cqcap * 8, 256) + 8192;
    ws_reserve(ctx, need);
    int64_t lx, lyin;
    const float *dX = stage_aligned(ctx, X, n, d, ldx, &lx, st);
    const float *dY = stage_aligned(ctx, Y, n, s + k, ldy, &lyin, st);
    float *Yp = ws_array<float>(ctx, (size_t)n * ldo);
    void *cs = ws_alloc(ctx, (size_t)count * n_pad * 16);
    void *rec = ws_alloc(ctx, rec_bytes);
    int4 *cq = ws_array<int4>(ctx, cqcap);
    double *cqd = ws_array<double>(ctx, cqcap);
    unsigned long long *cqcount = ws_array<unsigned long long>(ctx, 1);
    ADAGIO_CUDA(cudaMemsetAsync(rec, 0, rec_bytes, st));
    ADAGIO_CUDA(cudaMemsetAsync(cqcount, 0, sizeof(unsigned long long), st));
    prefix_layout_kernel<<<dim3((unsigned)n, (unsigned)ceil_div(ldo, 128)), 128, 0, st>>>(dY, n, lyin, s, jo, k,
                                                                                        Yp, ldo);
    ADAGIO_CHECK_LAUNCH();
    MultiSpec ms;
    ms.count = count;
    ms.s = s;
    ms.s_pad = s_pad;
    ms.jo = jo;
    ms.k = k;
    ms.eps = eps;
    for (int c = 0; c < count; ++c) ms.kc[c] = kc[c];
    ms.cs = cs;
    ms.out = rec;
    ms.slots = slots;
    ms.cq = cq;
    ms.cqcount = cqcount;
    ms.cqcap = cqcap;
    CertOptions co;
    co.eps = eps;
    co.lo = 0.0;
    co.hi = 2.0 * eps;
    co.precision = precision;
    co.multi = &ms;
    const int rc = certify(ctx, dX, lx, Yp, ldo, n, d, Kt, co, full, st);
    std::vector<CandRecord> h((size_t)slots * count);
    ADAGIO_CUDA(cudaMemcpy(h.data(), rec, rec_bytes, cudaMemcpyDeviceToHost));
    // the open pairs, decided exactly
    unsigned long long offered = 0;
    ADAGIO_CUDA(cudaMemcpy(&offered, cqcount, sizeof(offered), cudaMemcpyDeviceToHost));
    const long long nq = (long long)std::min(offered, cqcap);
    std::vector<int4> hq((size_t)nq);
    std::vector<double> hd((size_t)nq);
    if (nq > 0) {
        const int4 kc4 = make_int4(kc[0], count > 1 ? kc[1] : 1, count > 2 ? kc[2] : 1, count > 3 ? kc[3] : 1);
        prefix_recompute_kernel<<<(unsigned)ceil_div(nq * 32, 256), 256, 0, st>>>(dX, lx, d, Yp, ldo, s, jo, k, kc4,
                                                                                 cq, nq, cqd);
        ADAGIO_CHECK_LAUNCH();
        ADAGIO_CUDA(cudaMemcpy(hq.data(), cq, sizeof(int4) * (size_t)nq, cudaMemcpyDeviceToHost));
        ADAGIO_CUDA(cudaMemcpy(hd.data(), cqd, sizeof(double) * (size_t)nq, cudaMemcpyDeviceToHost));
    }
    // r = dy2 / dx2 of every counted pair lies in [rmin_lo, rmax_hi]; the
    // largest distortion |sqrt(r) - 1| (Eq. 2) is bracketed by the extremes of
    // the lower and upper bounds (widened by 8 units for the kernel's rounded
    // products and divisions), and by the exact values of the recomputed pairs
    const double w = 8.0 * 5.9604645e-08;
    for (int c = 0; c < count; ++c) {
        adagio_prefix_cert &o = out[c];
        std::memset(&o, 0, sizeof(o));
        o.k = kc[c];
        double rmh = 0.0, rml = 0.0, rnl = INFINITY, rnh = INFINITY;
        unsigned long long open = 0;
        for (int s2 = 0; s2 < slots; ++s2) {
            const CandRecord &r = h[(size_t)s2 * count + c];
            rmh = std::max(rmh, (double)r.rmax_hi);
            rml = std::max(rml, (double)r.rmax_lo);
            rnl = std::min(rnl, (double)r.rmin_lo);
            rnh = std::min(rnh, (double)r.rmin_hi);
            o.violations += r.certain;
            open += r.open;
        }
        double exact_max = -1.0;
        for (long long q = 0; q < nq; ++q) {
            if (hq[(size_t)q].z != c) continue;
            ++o.recomputed;
            const double dq = hd[(size_t)q];
            if (dq < 0.0) continue;  // x_i == x_j
            exact_max = std::max(exact_max, dq);
            if (dq > eps) ++o.violations;
        }
        o.unsettled_pairs = open - o.recomputed;
        const double up_hi = std::sqrt(rmh * (1.0 + w)) - 1.0;
        const double up_lo = 1.0 - std::sqrt(std::max(rnl, 0.0) * (1.0 - w));
        const double lo_hi = std::sqrt(std::max(rml, 0.0) * (1.0 - w)) - 1.0;
        const double lo_lo = 1.0 - std::sqrt(rnh * (1.0 + w));
        o.max_upper = std::isinf(rmh) ? INFINITY : std::max(std::max(up_hi, up_lo), exact_max);
        o.max_lower = std::max({0.0, lo_hi, std::isinf(rnh) ? -1.0 : lo_lo, exact_max});
        o.verdict = o.violations > 0 ? 0 : (o.unsettled_pairs > 0 ? -1 : 1);
    }
    return rc;
    API_END(ctx)
}
