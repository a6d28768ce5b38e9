// Shared pieces of the all-pairs distortion certificate (Eq. 2, Eq. 3):
// per-pair classification with an error bound, per-thread statistics, the
// recompute queue and the per-CTA partial record.  Used by the FP32 SIMT tile
// kernel (cert_simt.cu) and the tcgen05 tile kernel (cert_tc.cu).
//
// Fast path.  For a pair (i, j) the tile kernels form the Gram entries
// gx = xc_i . xc_j and gy = yc_i . yc_j of the centred rows and turn them into
//     dx2 = |xc_i|^2 + |xc_j|^2 - 2 gx,   dy2 likewise,
//     rho = sqrt(dy2 / dx2),   delta = |rho - 1|                    (Eq. 2)
// The row statistic (n2, q4, q1) of every row gives a bound on the error of
// dx2:  E = q4_i q4_j + q1_i q1_j + c_r (n2_i + n2_j), where q4 is the row's
// 4-norm times sqrt(2 c4) (product error of the split arithmetic, which
// averages over the K terms) and q1 is its 2-norm times sqrt(2 c_acc)
// (accumulation rounding).  With a = E_x/dx2 and b = E_y/dy2 the distortion
// error is at most B = 0.55 rho (a + b) + 2^-22.
//
// A pair goes to the recompute queue when its bound could change any
// reported quantity: B > 1e-6 and an edge of the histogram (or eps) lies
// within B of delta; or B > 1e-5 (the maximum's tolerance); or the Gram
// values are too ill-conditioned to bound (a or b > 1/8, dx2 <= 0, dy2 <= 0).
// Queued pairs are left out of the fast statistics and added back, exactly,
// by the recompute kernel.
#pragma once

#include <stdint.h>

namespace adagio {

struct __align__(16) RowStat {
    float n2;  // squared 2-norm of the centred row
    float q4;  // sqrt(2 c4) * 4-norm
    float q1;  // sqrt(2 c_acc) * 2-norm
    float pad;
};

// Per-CTA partial statistics (fast path or recompute path).
struct CertPartial {
    unsigned long long hist[kBins];
    unsigned long long pairs;       // pairs classified here (not queued)
    unsigned long long violations;
    unsigned long long overflow;
    unsigned long long degenerate;  // recompute path only
    unsigned long long queued;      // fast path: pairs pushed to the queue
    double sum;                     // sum of distortions
    double bound_sum;               // sum of per-pair error bounds
    float max;                      // max distortion (-1 if none)
    float max_bound;                // error bound of the max pair
    int argmax_i, argmax_j;
};

struct CertConst {
    float lo, hi, w, inv_w;  // histogram range, bin width, 1/width
    float eps;
    float c_r;               // epilogue rounding coefficient
    int lo_is_floor;         // lo <= 0: the lower edge is not a real boundary
};

constexpr float kExempt = 1e-6f;   // histogram/violation exactness threshold
constexpr float kMaxTol = 1e-5f;   // tolerance of the reported maximum
constexpr float kEvalErr = 2.3841858e-07f;  // 2^-22: FP32 evaluation of delta

// Outcome of the fast classification of one pair.
enum PairClass { PAIR_SKIP = 0, PAIR_OK = 1, PAIR_QUEUE = 2 };

struct FastPair {
    float delta;
    float bound;
    int bin;        // -1 = overflow
    int violation;
};

// Classify one pair from its Gram entries.  Returns PAIR_OK with `out` filled,
// or PAIR_QUEUE when the pair must be recomputed exactly.
__device__ __forceinline__ int classify_pair(float gx, float gy, const RowStat &xi,
                                             const RowStat &xj, const RowStat &yi,
                                             const RowStat &yj, const CertConst &cc,
                                             FastPair &out) {
    float dx2 = (xi.n2 + xj.n2) - 2.0f * gx;
    float dy2 = (yi.n2 + yj.n2) - 2.0f * gy;
    float ex = fmaf(xi.q4, xj.q4, fmaf(xi.q1, xj.q1, cc.c_r * (xi.n2 + xj.n2)));
    float ey = fmaf(yi.q4, yj.q4, fmaf(yi.q1, yj.q1, cc.c_r * (yi.n2 + yj.n2)));
    // ill-conditioned or non-positive: cannot bound the ratio
    if (!(dx2 > 8.0f * ex) || !(dy2 > 8.0f * ey)) return PAIR_QUEUE;
    float a = __fdividef(ex, dx2);
    float b = __fdividef(ey, dy2);
    float rho = sqrtf(dy2 / dx2);
    float delta = fabsf(rho - 1.0f);
    float bound = fmaf(0.55f * rho, a + b, kEvalErr * fmaxf(rho, 1.0f));
    if (bound > kMaxTol) return PAIR_QUEUE;
    float t = (delta - cc.lo) * cc.inv_w;
    if (bound > kExempt) {
        // distance to the nearest histogram edge, to eps
        float tn = rintf(t);
        bool edge_real = !(cc.lo_is_floor && tn <= 0.0f) && tn <= (float)kBins;
        bool near_edge = edge_real && fabsf(t - tn) * cc.w < bound;
        bool near_eps = fabsf(delta - cc.eps) < bound;
        if (near_edge || near_eps) return PAIR_QUEUE;
    }
    out.delta = delta;
    out.bound = bound;
    out.violation = delta > cc.eps;
    if (delta < cc.lo || delta >= cc.hi) {
        out.bin = -1;
    } else {
        int bin = (int)floorf(t);
        out.bin = min(max(bin, 0), kBins - 1);
    }
    return PAIR_OK;
}

// Lexicographic (max, then smallest (i, j)) comparison used by every max merge.
__device__ __forceinline__ bool better_max(float m1, int i1, int j1, float m2, int i2, int j2) {
    if (m1 != m2) return m1 > m2;
    if (i1 != i2) return (unsigned)i1 < (unsigned)i2;
    return (unsigned)j1 < (unsigned)j2;
}

// Block-wide reduction of per-thread statistics into one CertPartial slot.
// `s_hist` holds HS histogram slots per bin laid out [bin][slot] (u32; one
// slot per thread when HS = NT, one per warp when HS = NT / 32), so both the
// per-pair increment and this fold are bank-conflict free.  Must be called by
// every thread of the block; ends with a __syncthreads().
template <int NT, int HS = NT>
__device__ void write_partial(CertPartial *dst, const unsigned *s_hist, unsigned long long pairs,
                              unsigned long long viol, unsigned long long over,
                              unsigned long long queued, unsigned long long degen, double sum,
                              double bsum, float mx, float mxb, int ai, int aj) {
    constexpr int NW = NT / 32;
    __shared__ unsigned long long r_u[5][NW];
    __shared__ double r_d[2][NW];
    __shared__ float r_m[2][NW];
    __shared__ int r_i[2][NW];
    __shared__ unsigned long long r_h[kBins];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long u[5] = {pairs, viol, over, queued, degen};
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int q = 0; q < 5; ++q) u[q] += __shfl_xor_sync(0xffffffffu, u[q], o);
        sum += __shfl_xor_sync(0xffffffffu, sum, o);
        bsum += __shfl_xor_sync(0xffffffffu, bsum, o);
        float om = __shfl_xor_sync(0xffffffffu, mx, o);
        float ob = __shfl_xor_sync(0xffffffffu, mxb, o);
        int oi = __shfl_xor_sync(0xffffffffu, ai, o);
        int oj = __shfl_xor_sync(0xffffffffu, aj, o);
        if (better_max(om, oi, oj, mx, ai, aj)) {
            mx = om; mxb = ob; ai = oi; aj = oj;
        }
    }
    if (lane == 0) {
#pragma unroll
        for (int q = 0; q < 5; ++q) r_u[q][warp] = u[q];
        r_d[0][warp] = sum; r_d[1][warp] = bsum;
        r_m[0][warp] = mx; r_m[1][warp] = mxb; r_i[0][warp] = ai; r_i[1][warp] = aj;
    }
    if (threadIdx.x < kBins) r_h[threadIdx.x] = 0;
    __syncthreads();
    for (int b = 0; b < kBins; ++b) {
        unsigned long long v = threadIdx.x < HS ? s_hist[b * HS + threadIdx.x] : 0u;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0 && v) atomicAdd(&r_h[b], v);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t[5] = {0, 0, 0, 0, 0};
        double d0 = 0, d1 = 0;
        float m = -1.0f, mb = 0.0f;
        int bi = 0x7fffffff, bj = 0x7fffffff;
        for (int w = 0; w < NW; ++w) {
            for (int q = 0; q < 5; ++q) t[q] += r_u[q][w];
            d0 += r_d[0][w]; d1 += r_d[1][w];
            if (better_max(r_m[0][w], r_i[0][w], r_i[1][w], m, bi, bj)) {
                m = r_m[0][w]; mb = r_m[1][w]; bi = r_i[0][w]; bj = r_i[1][w];
            }
        }
        dst->pairs = t[0]; dst->violations = t[1]; dst->overflow = t[2];
        dst->queued = t[3]; dst->degenerate = t[4];
        dst->sum = d0; dst->bound_sum = d1;
        dst->max = m; dst->max_bound = mb; dst->argmax_i = bi; dst->argmax_j = bj;
    }
    if (threadIdx.x < kBins) dst->hist[threadIdx.x] = r_h[threadIdx.x];
    __syncthreads();
}

// Warp-aggregated push of the flagged pairs of this warp step onto the queue.
// Every lane of the warp must call it (flag may be false).
__device__ __forceinline__ void queue_push(bool flag, int i, int j, int2 *queue,
                                           unsigned long long *qcount, unsigned long long qcap) {
    unsigned mask = __ballot_sync(0xffffffffu, flag);
    if (mask == 0) return;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(mask) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(qcount, (unsigned long long)__popc(mask));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (flag) {
        unsigned long long pos = base + __popc(mask & ((1u << lane) - 1u));
        if (pos < qcap) queue[pos] = make_int2(i, j);
    }
}

// Maps a linear index over the upper triangle (including the diagonal) of a
// T x T tile grid to (I, J), I <= J, row by row.
__device__ __forceinline__ void tri_index(long long t, int T, int &I, int &J) {
    // offset(I) = I*T - I*(I-1)/2 ; solve offset(I) <= t < offset(I+1)
    double b = 2.0 * T + 1.0;
    double disc = b * b - 8.0 * (double)t;
    int i = (int)floor((b - sqrt(fmax(disc, 0.0))) * 0.5);
    i = max(0, min(i, T - 1));
    long long off = (long long)i * T - (long long)i * (i - 1) / 2;
    while (off > t) {
        --i;
        off = (long long)i * T - (long long)i * (i - 1) / 2;
    }
    while (i + 1 < T) {
        long long nxt = (long long)(i + 1) * T - (long long)(i + 1) * i / 2;
        if (nxt > t) break;
        ++i;
        off = nxt;
    }
    I = i;
    J = i + (int)(t - off);
}

}  // namespace adagio
