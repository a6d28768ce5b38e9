// K9 + K10: exact recompute of flagged pairs and the certificate finaliser.
//
// K9 takes every pair the tile kernels could not classify with certainty and
// recomputes both squared distances from coordinate differences of the
// ORIGINAL float32 inputs (no centring, no Gram), one warp per pair, in
// double-float arithmetic: each difference is split exactly by TwoSum, each
// square exactly by an FMA-based TwoProduct, and the running sum is kept as
// an unevaluated hi + lo pair (Dekker 1971; Knuth TAOCP vol. 2, 4.2.2).  The
// relative error of the result is a few units of 2^-44, far below the 1e-6
// classification threshold.  The distortion (Eq. 2) and its bin are then
// evaluated in double precision.  A pair with ||x_i - x_j|| == 0 is counted
// as degenerate.
//
// K10 merges the per-CTA partials of both paths in a fixed order, so the
// result does not depend on scheduling (apart from the order of the queue).
#include "internal.cuh"
#include "cert.cuh"

namespace adagio {

namespace {

constexpr int RT = 256;  // recompute block

struct DF {
    float hi, lo;
};

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    float bp = __fsub_rn(s, a);
    float ap = __fsub_rn(s, bp);
    e = __fadd_rn(__fsub_rn(a, ap), __fsub_rn(b, bp));
}

// acc += (a - b)^2 in double-float
__device__ __forceinline__ void add_sq_diff(DF &acc, float a, float b) {
    float d, de;
    two_sum(a, -b, d, de);                 // a - b = d + de exactly
    float p = __fmul_rn(d, d);
    float pe = __fmaf_rn(d, d, -p);        // d*d = p + pe exactly
    float corr = __fmaf_rn(2.0f * d, de, pe);
    float s, e;
    two_sum(acc.hi, p, s, e);
    acc.hi = s;
    acc.lo = __fadd_rn(acc.lo, __fadd_rn(e, corr));
}

__device__ __forceinline__ DF df_add(DF a, DF b) {
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    DF r;
    r.hi = __fadd_rn(s, e);
    r.lo = __fsub_rn(e, __fsub_rn(r.hi, s));
    return r;
}

__device__ __forceinline__ DF warp_sum(DF v) {
    for (int o = 16; o > 0; o >>= 1) {
        DF w;
        w.hi = __shfl_xor_sync(0xffffffffu, v.hi, o);
        w.lo = __shfl_xor_sync(0xffffffffu, v.lo, o);
        v = df_add(v, w);
    }
    return v;
}

__global__ void __launch_bounds__(RT) recompute_kernel(const float *__restrict__ X, int64_t ldx,
                                                        int d, const float *__restrict__ Y,
                                                        int64_t ldy, int m,
                                                        const int2 *__restrict__ queue,
                                                        const unsigned long long *__restrict__ qcount,
                                                        unsigned long long qcap, CertConst cc,
                                                        CertPartial *__restrict__ partials) {
    extern __shared__ unsigned s_hist[];  // [kBins][RT]
    const int tid = threadIdx.x, lane = tid & 31;
    for (int b = 0; b < kBins; ++b) s_hist[b * RT + tid] = 0;
    __syncthreads();
    const unsigned long long qlen = min(*qcount, qcap);
    const long long warps = (long long)gridDim.x * (RT / 32);
    unsigned long long npairs = 0, nviol = 0, nover = 0, ndeg = 0;
    double sum = 0.0;
    float mx = -1.0f;
    int ai = 0x7fffffff, aj = 0x7fffffff;
    const double lo = cc.lo, span = (double)cc.hi - (double)cc.lo;
    for (long long q = (long long)blockIdx.x * (RT / 32) + (tid >> 5); q < (long long)qlen;
         q += warps) {
        const int2 pr = queue[q];
        const float *xi = X + (int64_t)pr.x * ldx, *xj = X + (int64_t)pr.y * ldx;
        const float *yi = Y + (int64_t)pr.x * ldy, *yj = Y + (int64_t)pr.y * ldy;
        DF ax{0.0f, 0.0f}, ay{0.0f, 0.0f};
        for (int k = lane; k < d; k += 32) add_sq_diff(ax, xi[k], xj[k]);
        for (int k = lane; k < m; k += 32) add_sq_diff(ay, yi[k], yj[k]);
        ax = warp_sum(ax);
        ay = warp_sum(ay);
        if (lane == 0) {
            const double dx2 = (double)ax.hi + (double)ax.lo;
            const double dy2 = (double)ay.hi + (double)ay.lo;
            if (dx2 == 0.0) {
                ++ndeg;
            } else {
                const double delta = fabs(sqrt(dy2 / dx2) - 1.0);
                ++npairs;
                sum += delta;
                nviol += delta > (double)cc.eps;
                if (delta < lo || delta >= (double)cc.hi) {
                    ++nover;
                } else {
                    int b = (int)floor((delta - lo) / span * (double)kBins);
                    b = min(max(b, 0), kBins - 1);
                    s_hist[b * RT + tid] += 1u;
                }
                const float df = (float)delta;
                if (better_max(df, pr.x, pr.y, mx, ai, aj)) { mx = df; ai = pr.x; aj = pr.y; }
            }
        }
    }
    __syncthreads();
    write_partial<RT>(partials + blockIdx.x, s_hist, npairs, nviol, nover, 0ull, ndeg, sum, 0.0,
                      mx, 0.0f, ai, aj);
}

__global__ void finalize_kernel(const CertPartial *__restrict__ fast, int nfast,
                                const CertPartial *__restrict__ rec, int nrec,
                                const unsigned long long *__restrict__ qcount,
                                const unsigned *__restrict__ flags, const int *__restrict__ status,
                                const int *__restrict__ stop_flag, CertDevResult *__restrict__ out) {
    const int tid = threadIdx.x;  // 64 threads: one per bin
    unsigned long long h = 0;
    for (int c = 0; c < nfast; ++c) h += fast[c].hist[tid];
    for (int c = 0; c < nrec; ++c) h += rec[c].hist[tid];
    out->hist[tid] = h;
    if (tid == 0) {
        unsigned long long fp = 0, qd = 0, rp = 0, dg = 0, vi = 0, ov = 0;
        double s = 0.0, bs = 0.0;
        float mx = -1.0f, mxb = 0.0f;
        int ai = 0x7fffffff, aj = 0x7fffffff;
        for (int c = 0; c < nfast; ++c) {
            const CertPartial &p = fast[c];
            fp += p.pairs; qd += p.queued; vi += p.violations; ov += p.overflow;
            s += p.sum; bs += p.bound_sum;
            mxb = fmaxf(mxb, p.max_bound);
            if (better_max(p.max, p.argmax_i, p.argmax_j, mx, ai, aj)) {
                mx = p.max; ai = p.argmax_i; aj = p.argmax_j;
            }
        }
        for (int c = 0; c < nrec; ++c) {
            const CertPartial &p = rec[c];
            rp += p.pairs; dg += p.degenerate; vi += p.violations; ov += p.overflow;
            s += p.sum;
            if (better_max(p.max, p.argmax_i, p.argmax_j, mx, ai, aj)) {
                mx = p.max; ai = p.argmax_i; aj = p.argmax_j;
            }
        }
        out->fast_pairs = fp; out->queued = qd; out->recomputed = rp; out->degenerate = dg;
        out->violations = vi; out->overflow = ov; out->sum = s; out->bound_sum = bs;
        out->max = mx; out->max_bound = mxb; out->argmax_i = ai; out->argmax_j = aj;
        out->flags = *flags;
        out->status = status ? *status : 0;
        out->stopped = stop_flag ? *stop_flag : 0;
        out->qlen = *qcount;
    }
}

}  // namespace

void recompute_init() {
    set_max_dyn_smem((const void *)recompute_kernel, (int)((size_t)kBins * RT * sizeof(unsigned)));
}

void launch_recompute(const float *X, int64_t ldx, int d, const float *Y, int64_t ldy, int m,
                      const int2 *queue, const unsigned long long *qcount,
                      unsigned long long qcap, CertConst cc, CertPartial *partials, int grid,
                      cudaStream_t st) {
    const size_t smem = (size_t)kBins * RT * sizeof(unsigned);
    set_max_dyn_smem((const void *)recompute_kernel, (int)smem);
    recompute_kernel<<<grid, RT, smem, st>>>(X, ldx, d, Y, ldy, m, queue, qcount, qcap, cc,
                                            partials);
    ADAGIO_CHECK_LAUNCH();
}

void launch_finalize(const CertPartial *fast, int nfast, const CertPartial *rec, int nrec,
                     const unsigned long long *qcount, const unsigned *flags, const int *status,
                     const int *stop_flag, CertDevResult *out, cudaStream_t st) {
    finalize_kernel<<<1, kBins, 0, st>>>(fast, nfast, rec, nrec, qcount, flags, status, stop_flag,
                                         out);
    ADAGIO_CHECK_LAUNCH();
}

}  // namespace adagio
