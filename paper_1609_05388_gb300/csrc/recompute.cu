// K9 + K10: recompute of flagged pairs (two levels, the second exact) and the
// certificate finaliser.
//
// K9 takes every pair the tile kernels could not classify with certainty and
// recomputes both squared distances from coordinate differences of the
// ORIGINAL float32 inputs (no centring, no Gram), one warp per pair, in two
// levels.  Level 1: each difference rounded once to FP32, its square added
// by FMA into a short FP32 chain (at most 4 terms), each chain added into a
// double-float sum (TwoSum), lanes combined in double-float: the squared
// distance is within 7u (u = 2^-24) of the exact one (2u from the difference,
// 4u from the chain, u from the final rounding), and the distortion within
//     B1 = 7u (1 + rho^2) / (1 + rho) + 12u delta,   rho = sqrt(dy2 / dx2)
// (the numerator error over the denominator, plus the denominator's own
// rounding), taken as 8u and 13u.  The pair is counted from level 1 when B1
// <= 1e-6 (the certificate's band: a count may differ only for pairs within
// 1e-6 of a bin edge or of eps) or when no edge and not eps lies within B1 of
// its distortion.  Otherwise the warp recomputes it at level 2.  Level 2: each
// difference is rounded once to FP32 (relative error <= 2^-24), squared
// exactly by an FMA-based TwoProduct, and the squares are summed as an
// unevaluated hi + lo pair with TwoSum (Dekker 1971; Knuth TAOCP vol. 2,
// 4.2.2).  All terms are positive, so the relative error of each squared
// distance is at most 2^-23 plus the double-float summation error (a few
// units of 2^-44), far below the 1e-6 classification threshold.  Rows are
// read with the widest aligned vector loads (float4, float2 or float).
// The distortion (Eq. 2) is then evaluated without FP64 (slow on this GPU)
// in the cancellation-free form
//     delta = |dy2 - dx2| / (dx2 + sqrt(dx2) sqrt(dy2))
// with the difference dy2 - dx2 taken in double-float and one IEEE FP32
// division and two square roots: its relative error is below 6 * 2^-24
// (under 4e-7 absolute for delta <= 1), inside the 1e-6 band around the
// bin edges and eps where the certificate allows a miscount.  A pair with
// ||x_i - x_j|| == 0 is counted as degenerate.
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

// acc += (a - b)^2 in double-float, the difference rounded once
__device__ __forceinline__ void add_sq_diff(DF &acc, float a, float b) {
    const float d = __fsub_rn(a, b);
    const float p = __fmul_rn(d, d);
    const float pe = __fmaf_rn(d, d, -p);  // d*d = p + pe exactly
    float s, e;
    two_sum(acc.hi, p, s, e);
    acc.hi = s;
    acc.lo = __fadd_rn(acc.lo, __fadd_rn(e, pe));
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

// a - b in double-float
__device__ __forceinline__ DF df_sub(DF a, DF b) {
    DF nb;
    nb.hi = -b.hi;
    nb.lo = -b.lo;
    return df_add(a, nb);
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

template <int V>
struct VecT;
template <>
struct VecT<4> {
    using T = float4;
};
template <>
struct VecT<2> {
    using T = float2;
};
template <>
struct VecT<1> {
    using T = float;
};

__device__ __forceinline__ void add_vec(DF (&c)[4], float4 a, float4 b) {
    add_sq_diff(c[0], a.x, b.x);
    add_sq_diff(c[1], a.y, b.y);
    add_sq_diff(c[2], a.z, b.z);
    add_sq_diff(c[3], a.w, b.w);
}
__device__ __forceinline__ void add_vec(DF (&c)[4], float2 a, float2 b) {
    add_sq_diff(c[0], a.x, b.x);
    add_sq_diff(c[1], a.y, b.y);
}
__device__ __forceinline__ void add_vec(DF (&c)[4], float a, float b) { add_sq_diff(c[0], a, b); }

template <int V>
__device__ __forceinline__ typename VecT<V>::T vec_zero();
template <>
__device__ __forceinline__ float4 vec_zero<4>() { return make_float4(0.0f, 0.0f, 0.0f, 0.0f); }
template <>
__device__ __forceinline__ float2 vec_zero<2>() { return make_float2(0.0f, 0.0f); }
template <>
__device__ __forceinline__ float vec_zero<1>() { return 0.0f; }

// sum over this lane's elements k of (a_k - b_k)^2.  The rows are V-aligned
// and read with V-wide loads in chunks of U loads per row, all of a chunk's
// 2U loads issued before the first is used (a pair is a few dependent L2
// round trips, not one per element); missing entries of the last chunk read
// as zero in both rows and add nothing.  A scalar tail follows.
template <int V>
__device__ __forceinline__ DF sq_dist_lanes(const float *__restrict__ a, const float *__restrict__ b,
                                            int n, int lane) {
    using T = typename VecT<V>::T;
    constexpr int UU = V == 4 ? 4 : (V == 2 ? 8 : 16);  // 64 bytes of each row per lane and chunk
    DF c[4] = {{0.0f, 0.0f}, {0.0f, 0.0f}, {0.0f, 0.0f}, {0.0f, 0.0f}};
    const T *av = reinterpret_cast<const T *>(a), *bv = reinterpret_cast<const T *>(b);
    const int nv = n / V;
    for (int base = lane; base < nv; base += 32 * UU) {
        T x[UU], y[UU];
#pragma unroll
        for (int u = 0; u < UU; ++u) {
            const int v = base + 32 * u;
            x[u] = v < nv ? __ldg(av + v) : vec_zero<V>();
            y[u] = v < nv ? __ldg(bv + v) : vec_zero<V>();
        }
#pragma unroll
        for (int u = 0; u < UU; ++u) add_vec(c, x[u], y[u]);
    }
    for (int k = nv * V + lane; k < n; k += 32) add_sq_diff(c[0], __ldg(a + k), __ldg(b + k));
    return df_add(df_add(c[0], c[1]), df_add(c[2], c[3]));
}

// Level 1 of this lane's share of sum_k (a_k - b_k)^2.  Chain g is the
// coordinates 4g .. 4g + 3: their squares summed by FMA in FP32, the chain
// added into one of two double-float sums.  The chains, their lanes
// (g mod 32), their order and their accumulators depend only on the
// coordinate index, not on the load width V, so rows with any alignment give
// the same bits.  A lane issues all loads of four chains before using them;
// chains past the end read as zero; the n mod 4 last coordinates are
// one-term chains.
template <int V>
__device__ __forceinline__ void load_chain(const float *__restrict__ p, int g, float (&v)[4]) {
    if constexpr (V == 4) {
        const float4 q = __ldg(reinterpret_cast<const float4 *>(p) + g);
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    } else if constexpr (V == 2) {
        const float2 q0 = __ldg(reinterpret_cast<const float2 *>(p) + 2 * g);
        const float2 q1 = __ldg(reinterpret_cast<const float2 *>(p) + 2 * g + 1);
        v[0] = q0.x; v[1] = q0.y; v[2] = q1.x; v[3] = q1.y;
    } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] = __ldg(p + 4 * g + k);
    }
}

__device__ __forceinline__ void df_add_chain(DF &acc, float c) {
    float s, e;
    two_sum(acc.hi, c, s, e);
    acc.hi = s;
    acc.lo = __fadd_rn(acc.lo, e);
}

template <int V>
__device__ __forceinline__ DF sq_dist_lanes_fast(const float *__restrict__ a, const float *__restrict__ b,
                                                 int n, int lane) {
    constexpr int CH = 4;  // chains per lane and chunk
    DF c[2] = {{0.0f, 0.0f}, {0.0f, 0.0f}};
    const int ng = n / 4;
    for (int base = lane; base < ng; base += 32 * CH) {
        float x[CH][4], y[CH][4];
#pragma unroll
        for (int u = 0; u < CH; ++u) {
            const int g = base + 32 * u;
            if (g < ng) {
                load_chain<V>(a, g, x[u]);
                load_chain<V>(b, g, y[u]);
            } else {
#pragma unroll
                for (int k = 0; k < 4; ++k) x[u][k] = y[u][k] = 0.0f;
            }
        }
#pragma unroll
        for (int u = 0; u < CH; ++u) {
            float d = __fsub_rn(x[u][0], y[u][0]), s = __fmul_rn(d, d);
#pragma unroll
            for (int k = 1; k < 4; ++k) {
                d = __fsub_rn(x[u][k], y[u][k]);
                s = __fmaf_rn(d, d, s);
            }
            df_add_chain(c[u & 1], s);
        }
    }
    for (int k = 4 * ng + lane; k < n; k += 32) {
        const float d = __fsub_rn(__ldg(a + k), __ldg(b + k));
        df_add_chain(c[0], __fmul_rn(d, d));
    }
    return df_add(c[0], c[1]);
}

// distortion (Eq. 2) of a pair from its double-float squared distances, in
// the cancellation-free form (FP32 division and square roots, IEEE)
__device__ __forceinline__ float pair_delta(DF ax, DF ay, float &dx2, float &dy2) {
    const DF dd = df_sub(ay, ax);
    dx2 = __fadd_rn(ax.hi, ax.lo);
    dy2 = __fadd_rn(ay.hi, ay.lo);
    const float den = __fmaf_rn(__fsqrt_rn(dx2), __fsqrt_rn(dy2), dx2);
    return __fdiv_rn(fabsf(__fadd_rn(dd.hi, dd.lo)), den);
}

constexpr float kBandR = 1e-6f;  // a count may differ only for pairs this close to an edge or eps

template <int VX, int VY>
__global__ void __launch_bounds__(RT, 3) recompute_kernel(const float *__restrict__ X, int64_t ldx,
                                                        int d, const float *__restrict__ Y,
                                                        int64_t ldy, int m,
                                                        const int2 *__restrict__ queue,
                                                        const unsigned long long *__restrict__ qcount,
                                                        unsigned long long qcap, CertConst cc,
                                                        CertPartial *__restrict__ partials) {
    constexpr int NW = RT / 32;
    __shared__ unsigned s_hist[kBins * NW];  // [bin][warp]: lane 0 of each warp counts
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int e = tid; e < kBins * NW; e += RT) s_hist[e] = 0;
    __syncthreads();
    const unsigned long long qlen = min(*qcount, qcap);
    const long long warps = (long long)gridDim.x * NW;
    unsigned long long npairs = 0, nviol = 0, nover = 0, ndeg = 0;
    double sum = 0.0;
    float mx = -1.0f;
    int ai = 0x7fffffff, aj = 0x7fffffff;
    for (long long q = (long long)blockIdx.x * NW + warp; q < (long long)qlen; q += warps) {
        const int2 pr = queue[q];
        const float *xi = X + (int64_t)pr.x * ldx, *xj = X + (int64_t)pr.y * ldx;
        const float *yi = Y + (int64_t)pr.x * ldy, *yj = Y + (int64_t)pr.y * ldy;
        DF ax = warp_sum(sq_dist_lanes_fast<VX>(xi, xj, d, lane));
        DF ay = warp_sum(sq_dist_lanes_fast<VY>(yi, yj, m, lane));
        float delta = 0.0f;
        int exact = 0;
        if (lane == 0 && ax.hi != 0.0f) {
            float dx2, dy2;
            delta = pair_delta(ax, ay, dx2, dy2);
            const float rho2 = __fdiv_rn(dy2, dx2), rho = __fsqrt_rn(rho2);
            const float u = 5.9604645e-08f;
            const float b1 = u * (8.0f * (1.0f + rho2) / (1.0f + rho) + 13.0f * delta);
            // distance to the nearest bin edge (edges at integer t in [0, 64]) and to eps
            const float t = (delta - cc.lo) * cc.inv_w;
            const float tc = fminf(fmaxf(t, -0.5f), (float)kBins + 0.5f);
            const float dedge = fabsf(tc - rintf(tc)) * cc.w;
            const bool settled = (b1 <= kBandR) || (dedge > b1 && fabsf(delta - cc.eps) > b1);
            exact = settled ? 0 : 1;
        }
        if (__shfl_sync(0xffffffffu, exact, 0)) {
            // level 2 for this pair (rare): exact squares, double-float sums
            ax = warp_sum(sq_dist_lanes<VX>(xi, xj, d, lane));
            ay = warp_sum(sq_dist_lanes<VY>(yi, yj, m, lane));
            float dx2, dy2;
            if (lane == 0) delta = pair_delta(ax, ay, dx2, dy2);
        }
        if (lane == 0) {
            // the squares of the differences sum to zero only if every
            // difference is zero
            if (ax.hi == 0.0f) {
                ++ndeg;
            } else {
                ++npairs;
                sum += (double)delta;
                nviol += delta > cc.eps;
                if (delta < cc.lo || delta >= cc.hi) {
                    ++nover;
                } else {
                    int b = (int)floorf((delta - cc.lo) * cc.inv_w);
                    b = min(max(b, 0), kBins - 1);
                    s_hist[b * NW + warp] += 1u;
                }
                if (better_max(delta, pr.x, pr.y, mx, ai, aj)) { mx = delta; ai = pr.x; aj = pr.y; }
            }
        }
    }
    __syncthreads();
    write_partial<RT, NW>(partials + blockIdx.x, s_hist, npairs, nviol, nover, 0ull, ndeg, sum, 0.0,
                          mx, 0.0f, ai, aj);
}

// Merges the partials of both paths.  Every sum runs over a fixed assignment
// of partials to threads and a fixed reduction tree, so the result does not
// depend on scheduling.
constexpr int FT = 1024;
__global__ void __launch_bounds__(FT) finalize_kernel(const CertPartial *__restrict__ fast, int nfast,
                                                      const CertPartial *__restrict__ rec, int nrec,
                                                      const unsigned long long *__restrict__ qcount,
                                                      const unsigned *__restrict__ flags,
                                                      const int *__restrict__ status,
                                                      const int *__restrict__ stop_flag,
                                                      CertDevResult *__restrict__ out) {
    constexpr int SL = FT / kBins;  // slices per bin
    __shared__ unsigned long long s_h[SL][kBins];
    __shared__ unsigned long long s_u[6][FT / 32];
    __shared__ double s_d[2][FT / 32];
    __shared__ float s_m[2][FT / 32];
    __shared__ int s_i[2][FT / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int ntot = nfast + nrec;
    {
        const int bin = tid % kBins, slice = tid / kBins;
        unsigned long long h = 0;
        for (int c = slice; c < ntot; c += SL) h += c < nfast ? fast[c].hist[bin] : rec[c - nfast].hist[bin];
        s_h[slice][bin] = h;
    }
    unsigned long long u[6] = {0, 0, 0, 0, 0, 0};  // fast pairs, queued, recomputed, degenerate, violations, overflow
    double s = 0.0, bs = 0.0;
    float mx = -1.0f, mxb = 0.0f;
    int ai = 0x7fffffff, aj = 0x7fffffff;
    for (int c = tid; c < ntot; c += FT) {
        const bool f = c < nfast;
        const CertPartial &p = f ? fast[c] : rec[c - nfast];
        if (f) {
            u[0] += p.pairs; u[1] += p.queued;
            bs += p.bound_sum;
            mxb = fmaxf(mxb, p.max_bound);
        } else {
            u[2] += p.pairs; u[3] += p.degenerate;
        }
        u[4] += p.violations; u[5] += p.overflow;
        s += p.sum;
        if (better_max(p.max, p.argmax_i, p.argmax_j, mx, ai, aj)) { mx = p.max; ai = p.argmax_i; aj = p.argmax_j; }
    }
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int q = 0; q < 6; ++q) u[q] += __shfl_xor_sync(0xffffffffu, u[q], o);
        s += __shfl_xor_sync(0xffffffffu, s, o);
        bs += __shfl_xor_sync(0xffffffffu, bs, o);
        mxb = fmaxf(mxb, __shfl_xor_sync(0xffffffffu, mxb, o));
        const float om = __shfl_xor_sync(0xffffffffu, mx, o);
        const int oi = __shfl_xor_sync(0xffffffffu, ai, o);
        const int oj = __shfl_xor_sync(0xffffffffu, aj, o);
        if (better_max(om, oi, oj, mx, ai, aj)) { mx = om; ai = oi; aj = oj; }
    }
    if (lane == 0) {
#pragma unroll
        for (int q = 0; q < 6; ++q) s_u[q][warp] = u[q];
        s_d[0][warp] = s; s_d[1][warp] = bs;
        s_m[0][warp] = mx; s_m[1][warp] = mxb; s_i[0][warp] = ai; s_i[1][warp] = aj;
    }
    __syncthreads();
    if (tid < kBins) {
        unsigned long long h = 0;
        for (int sl = 0; sl < SL; ++sl) h += s_h[sl][tid];
        out->hist[tid] = h;
    }
    if (tid == 0) {
        unsigned long long t[6] = {0, 0, 0, 0, 0, 0};
        double d0 = 0.0, d1 = 0.0;
        float m = -1.0f, mb = 0.0f;
        int bi = 0x7fffffff, bj = 0x7fffffff;
        for (int w = 0; w < FT / 32; ++w) {
            for (int q = 0; q < 6; ++q) t[q] += s_u[q][w];
            d0 += s_d[0][w]; d1 += s_d[1][w];
            mb = fmaxf(mb, s_m[1][w]);
            if (better_max(s_m[0][w], s_i[0][w], s_i[1][w], m, bi, bj)) { m = s_m[0][w]; bi = s_i[0][w]; bj = s_i[1][w]; }
        }
        out->fast_pairs = t[0]; out->queued = t[1]; out->recomputed = t[2]; out->degenerate = t[3];
        out->violations = t[4]; out->overflow = t[5]; out->sum = d0; out->bound_sum = d1;
        out->max = m; out->max_bound = mb; out->argmax_i = bi; out->argmax_j = bj;
        out->flags = *flags;
        out->status = status ? *status : 0;
        out->stopped = stop_flag ? *stop_flag : 0;
        out->qlen = *qcount;
    }
}

}  // namespace

void recompute_init() {}

void launch_recompute(const float *X, int64_t ldx, int d, const float *Y, int64_t ldy, int m,
                      const int2 *queue, const unsigned long long *qcount,
                      unsigned long long qcap, CertConst cc, CertPartial *partials, int grid,
                      cudaStream_t st) {
    // widest vector load every row of the matrix starts aligned to
    auto width = [](const float *p, int64_t ld) {
        const uintptr_t a = reinterpret_cast<uintptr_t>(p);
        if (a % 16 == 0 && ld % 4 == 0) return 4;
        if (a % 8 == 0 && ld % 2 == 0) return 2;
        return 1;
    };
    const int vx = width(X, ldx), vy = width(Y, ldy);
#define ADAGIO_RECOMPUTE(A, B)                                                                    \
    recompute_kernel<A, B><<<grid, RT, 0, st>>>(X, ldx, d, Y, ldy, m, queue, qcount, qcap, cc, partials)
    if (vx == 4) {
        if (vy == 4) ADAGIO_RECOMPUTE(4, 4);
        else if (vy == 2) ADAGIO_RECOMPUTE(4, 2);
        else ADAGIO_RECOMPUTE(4, 1);
    } else if (vx == 2) {
        if (vy == 4) ADAGIO_RECOMPUTE(2, 4);
        else if (vy == 2) ADAGIO_RECOMPUTE(2, 2);
        else ADAGIO_RECOMPUTE(2, 1);
    } else {
        if (vy == 4) ADAGIO_RECOMPUTE(1, 4);
        else if (vy == 2) ADAGIO_RECOMPUTE(1, 2);
        else ADAGIO_RECOMPUTE(1, 1);
    }
#undef ADAGIO_RECOMPUTE
    ADAGIO_CHECK_LAUNCH();
}

void launch_finalize(const CertPartial *fast, int nfast, const CertPartial *rec, int nrec,
                     const unsigned long long *qcount, const unsigned *flags, const int *status,
                     const int *stop_flag, CertDevResult *out, cudaStream_t st) {
    finalize_kernel<<<1, FT, 0, st>>>(fast, nfast, rec, nrec, qcount, flags, status, stop_flag, out);
    ADAGIO_CHECK_LAUNCH();
}

}  // namespace adagio
