// K8 (tensor-core path): all-pairs distortion tiles on tcgen05.
//
// Persistent CTAs walk tiles (I, J), I <= J, of the pair matrix in the band
// order of the schedule table (bands of tile rows, so the I-tiles of a band
// stay in L2 while the J-tiles stream).  For every tile they form
//     Gy = Yc[I] Yc[J]^T   and   Gx = Xc[I] Xc[J]^T
// from 2-term split planes (hi + lo, FP16 or BF16, power-of-two scaled) with
// three products hi.hi + hi.lo + lo.hi per K chunk, accumulated in FP32 in
// tensor memory chunk by chunk, and hand the sums to the epilogue
// (cert_common.cuh), which classifies every pair (Eq. 2), accumulates max /
// histogram / counts and queues the pairs that need the recompute.
//
// Two variants share the code:
//   single  one CTA per 128 x 128 tile (tcgen05 cta_group::1, M = N = 128)
//   pair    a cluster of two CTAs per 256 x 128 tile (cta_group::2, M = 256,
//           N = 128): each CTA loads its own 128 rows of the I block and half
//           of the 128 J rows, the leader CTA issues the MMAs for both, and
//           each CTA's tensor memory receives its own 128 x 128 quarter-tile.
//           Per multiply-add this moves 25 % fewer bytes through L2 and
//           shared memory than the single variant (the MMA reads 6 KB of
//           operands per 128 x 128 x 16 step instead of 8 KB).
//
// Roles (320 threads per CTA):
//   warp 0      TMA producer: 4 planes (A hi/lo, B hi/lo) of 64 K-elements per
//               stage, 128-byte swizzle
//   warp 1      TMEM owner (512 columns = 2 chunk slots of 128 + 256 staging
//               columns) and, in the single CTA or the pair's leader, MMA
//               issuer: tcgen05.mma kind::f16, K = 16.  Every 64-element K
//               step goes to a fresh slot, cross products (hi.lo, lo.hi)
//               first and the 4 hi.hi products last: the FP32 accumulator
//               loses up to one unit in the last place per MMA (it
//               truncates), so this bounds the full-size roundings to 4 per
//               chunk
//   warps 2..9  epilogue: two warps per TMEM lane quarter, 64 columns each;
//               they drain every slot into register running sums (round to
//               nearest) and classify their 64 pairs at the end of a tile,
//               without data-dependent branches
// The producer (in a pair, the leader's producer, which hands every decision
// to the peer's producer through its shared memory) decides the tile
// sequence and sends it down the pipeline (a tile index per first stage, -1
// to stop, forwarded through a slot), so early exit needs no grid-wide
// barrier, and the epilogue warps never wait on one another.  Every wait is
// bounded: on timeout the role records a status word and leaves, the
// producers drain their in-flight copies, the MMA warp waits for its last
// commit, and TMEM is freed.
#include <cuda.h>

#include "internal.cuh"
#include "cert.cuh"
#include "tc_ptx.cuh"

#include <cmath>
#include <type_traits>
#include <vector>

namespace adagio {

using namespace tc;

namespace {

// Epilogue warps: 8 (two per TMEM lane quarter, 64 columns each) or 12 (three
// per quarter: 48, 40 and 40 columns)
constexpr int kEpiWarps = 8;
static_assert(kEpiWarps == 8 || kEpiWarps == 12, "8 or 12 epilogue warps");
constexpr int kThreads = 64 + 32 * kEpiWarps;               // producer, MMA, epilogue
constexpr int kSlots = 2;                                   // TMEM chunk accumulators
constexpr int kTile = 128;
constexpr int kKStep = 64;                                  // fp16 elements per stage row
constexpr uint32_t kAPlane = kTile * kKStep * 2;            // 16 KB: 128 rows of one plane
constexpr uint32_t kStageCol = kSlots * kTile;              // finished Gram sums (gx | gy)
constexpr uint32_t kTmemCols = kStageCol + 2 * kTile;       // 512
static_assert(kTmemCols == 512, "TMEM holds 512 columns");
constexpr int kPiece = 8;                                   // columns classified per step
// Histogram counters in shared memory: 64 bins plus an overflow bin (64),
// one u32 counter per (bin, tile row), shared by the two epilogue warps of a
// lane quarter (atomic adds; lane l of a warp always hits bank l).
constexpr int kHBins = kBins + 1;
constexpr int kHRows = kTile;
// Candidates of the multi-candidate certificate served by one pass.
constexpr int kMaxCand = 4;

// A JL-prefix candidate's verdict data, per epilogue warp.  Its pairs are
// judged on r = |f(x_i) - f(x_j)|^2 / |x_i - x_j|^2: the distortion of Eq. 2
// is |sqrt(r) - 1|, so it exceeds eps exactly when r lies outside
// [(1 - eps)^2, (1 + eps)^2], and error bounds on the two squared distances
// bound r without a square root or a division per pair.
struct CandPartial {
    float rmax_hi, rmax_lo;            // largest upper / lower bound on a pair's r
    float rmin_lo, rmin_hi;            // smallest lower / upper bound on a pair's r
    unsigned long long certain, open;  // pairs certainly beyond eps / on an open side
};
// Bound coefficient: with s = ex / dx2 + ey / dy2 <= 1/8 the square root of
// the ratio moves by at most ((1 - s)^(-1/2) - 1) <= 0.5523 s relative; the
// kernel carries ex, ey pre-multiplied by 0.56 (the row statistics' q4 by
// sqrt(0.56), the (n2_i + n2_j) coefficients by 0.56).
constexpr float kBoundCoef = 0.56f;
constexpr float kCondMax = kBoundCoef * 0.125f;

// JL-prefix candidates of one pass (the multi-candidate certificate): Y holds
// the PCA part in its first py_chunks 64-column chunks and k JL columns after
// it; candidate c keeps the first kc JL columns, scaled by sqrt(k / kc), and
// is complete after Y chunk end[c].
struct TcMulti {
    int count;                 // candidates (0: none)
    int py_chunks;             // Y chunks of the PCA part
    int end[kMaxCand];         // last Y chunk of each candidate's prefix
    float lam[kMaxCand];       // k / kc
    // raw bound coefficients (rounded up): the (n2_i + n2_j) terms of the X
    // side, the PCA part and the whole prefix, and 2^-24 for g - gP
    float cxr, cypr, cycr[kMaxCand], u2r;
    float kraw;                // 1 / 0.56 rounded up: raw q4 from the sqrt(0.56)-scaled ones
    // thresholds on r (rounding slack included): certainly beyond eps when
    // r > uv or r < lv, certainly within when lf <= r <= uf
    float uv, lv, uf, lf;
    long long n_pad;           // rows of each candidate's statistics
    int4 *cq;                  // open pairs (i, j, candidate) for the exact recompute
    unsigned long long *cqcount, cqcap;
    // [count][n_pad] interleaved by row pair (2q, 2q+1): element 2q = the two
    // |yP|^2 and the two q4 of the PCA part, element 2q + 1 = the two |yJc|^2
    // and the two q4 of the whole prefix (q4 times sqrt(0.56))
    const ulonglong2 *cs;
    CandPartial *out;          // [gridDim.x * kEpiWarps][count]
};

struct TcArgs {
    const float4 *rs;          // per row: (|xc|^2, |yc|^2, sqrt(0.56) q4x, sqrt(0.56) q4y)
    // the same statistics interleaved by column pair (2q, 2q+1): element 2q =
    // (|xc|^2, |xc|^2, |yc|^2, |yc|^2), element 2q+1 = the two q4x, the two q4y
    const ulonglong2 *rs2;
    float cx, cy;              // 0.56 x bound coefficients of (n2_i + n2_j) per side
    const float *scale_x, *scale_y;
    const uint32_t *sched;     // (I << 16) | J per tile (pair variant: I counts 256-row blocks)
    long long ntp;
    int n, kx_steps, ky_steps;
    uint32_t idesc;
    CertConst cc;
    int eps_bin;               // standard range: eps is the lower edge of this bin
    CertPartial *partials;     // [gridDim.x * kEpiWarps], one slot per epilogue warp
    int2 *queue;
    unsigned long long *qcount, qcap;
    int *stop_flag;
    int *status;
    float4 *dump;              // optional: (dx2, dy2, ex, ey) of 128 x 128 tile units
    long long dump_tiles;      // u = q * dump_stride, q < dump_tiles, into slot q
    long long dump_stride;
    TcMulti multi;             // JL-prefix candidates (the multi-candidate kernel only)
};

// Shared-memory layout of one CTA.  The pair variant loads half of the J rows
// per CTA, so its stages are smaller and there are four of them.
template <bool PAIR, bool MULTI = false>
struct Layout {
    // the multi-candidate kernel trades a stage for its per-thread verdict data
    static constexpr int kStages = PAIR ? 4 : (MULTI ? 2 : 3);
    static constexpr int kBRows = PAIR ? kTile / 2 : kTile;                   // J rows loaded here
    static constexpr uint32_t kBPlane = kBRows * kKStep * 2;
    static constexpr uint32_t kStageBytes = 2 * kAPlane + 2 * kBPlane;
    static constexpr uint32_t kTxBytes = PAIR ? 2 * kStageBytes : kStageBytes;  // per full barrier
    static constexpr uint32_t stages = 0;
    static constexpr uint32_t hist = kStages * kStageBytes;                  // u32 [65][128]
    static constexpr uint32_t bars = hist + kHBins * kHRows * 4;
    static constexpr uint32_t cmd = bars + 256;                               // int [16]
    static constexpr uint32_t dec = cmd + 64;                                 // int [4]
    static constexpr uint32_t tmem_ptr = dec + 16;
    static constexpr uint32_t totals = tmem_ptr + 16;                         // WarpTotals [8]
    static constexpr uint32_t cand = totals + 64 * kEpiWarps;                 // CandRun fields per thread
    static constexpr uint32_t total = cand + (MULTI ? kMaxCand * (4 * 4 + 2 * 8) * 32 * kEpiWarps : 0);
    static constexpr size_t smem = total + 1024;                              // + alignment slack
    static_assert(smem <= 232448, "tile kernel exceeds the 227 KB shared-memory limit");
    static_assert(totals % 8 == 0, "per-warp totals need 8-byte alignment");
    static_assert(kStageBytes % 1024 == 0 && kBPlane % 1024 == 0, "stage buffers need 1 KB alignment");
    static_assert((2 * kStages + 2 * kSlots + 6) * 8 <= 256, "barriers exceed their area");
};

// Folds the CTA's histogram counters into this epilogue warp's partial, once
// every epilogue warp has finished: warp ew takes bins ew, ew + 8, ...
// (the overflow bin 64 falls to warp 0).  With the standard range (STD) the
// violations come from the bins too: eps is the lower edge of bin eps_bin,
// so delta > eps <=> bin >= eps_bin (up to pairs within rounding of eps,
// which the exactness band exempts), and the overflow pairs lie above eps.
template <bool STD>
__device__ __forceinline__ void fold_hist(const uint32_t *s_hist, int ew, int eps_bin,
                                          CertPartial *dst) {
    const int lane = threadIdx.x & 31;
    unsigned long long pairs = 0, viol = 0, over = 0;
    for (int b = ew; b < kHBins; b += kEpiWarps) {
        const uint32_t *c = s_hist + b * kHRows;
        unsigned long long v = (unsigned long long)c[lane] + c[lane + 32] + c[lane + 64] + c[lane + 96];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        pairs += v;
        if (b == kBins) over = v;
        else dst->hist[b] = v;
        if (STD && b >= eps_bin) viol += v;
    }
    if (lane == 0) {
        dst->pairs += pairs;
        dst->overflow = over;
        if (STD) dst->violations = viol;
    }
    __syncwarp();
}

// a0 += b0, a1 += b1 in one packed FP32 instruction (each lane rounded to
// nearest, the same bits as two scalar adds)
__device__ __forceinline__ void add2_f32(float &a0, float &a1, uint32_t b0, uint32_t b1) {
    asm("{\n\t.reg .b64 ra, rb;\n\tmov.b64 ra, {%0, %1};\n\tmov.b64 rb, {%2, %3};\n\t"
        "add.rn.f32x2 ra, ra, rb;\n\tmov.b64 {%0, %1}, ra;\n\t}"
        : "+f"(a0), "+f"(a1)
        : "r"(b0), "r"(b1));
}

// this warp's TMEM columns into registers, one wait
__device__ __forceinline__ void tmem_ld_cols(uint32_t ta, uint32_t (&v)[40]) { tmem_ld40_wait(ta, v); }
__device__ __forceinline__ void tmem_ld_cols(uint32_t ta, uint32_t (&v)[48]) { tmem_ld48_wait(ta, v); }
__device__ __forceinline__ void tmem_ld_cols(uint32_t ta, uint32_t (&v)[64]) { tmem_ld64_wait(ta, v); }

struct EpiConst {
    float m2sx, m2sy;      // -2 / scale^2 of the split planes
    float cx, cy;          // 0.56 x bound coefficients of (n2_i + n2_j) per side
    float inv_w, t0, w;    // t = delta * inv_w + t0 = (delta - lo) / w
    float tlo;             // lowest t at which an edge is real, minus 0.5
    float eps;
};

// Statistics one epilogue thread keeps over the pairs of one tile row.
struct RowAcc {
    float sum;     // sum of the distortions of the pairs counted here
    float mxb;     // largest error bound among them
    float mx;      // largest distortion among them (0: possibly none)
    int mp;        // the piece (8 columns) where mx was first reached
    int viol;      // delta > eps (ranges where eps is not a bin edge)
};

// Per-warp running totals of the epilogue, in shared memory (lane 0 owns them).
struct WarpTotals {
    unsigned long long violations, queued;
    double sum, bound_sum;
    float max, max_bound;
    int argmax_i, argmax_j;
};

static_assert(sizeof(WarpTotals) <= 64, "per-warp totals exceed their shared-memory slot");

// The fast value of one pair from its Gram entries (Eq. 2), shared by the
// classification and the argmax search so that both see the same bits.  With
// p = dx2 dy2 and r = 1/sqrt(p):
//   delta = |sqrt(dy2 / dx2) - 1| = |dy2 - dx2| / (dx2 + p r)   (no cancellation)
// ex, ey (0.56 x the Gram error bounds, q4_i q4_j + c (n2_i + n2_j)) give
//   s = (ex dy2 + ey dx2) r^2 = 0.56 (ex / dx2 + ey / dy2),
//   B = rho s + 1.25e-6 delta + 1e-9,  rho = dy2 r,
// a bound on the distortion's error when s <= 0.56 / 8 and dx2, dy2 > 0 (the
// last two terms cover the approximate reciprocal square root and division,
// and the rounding of t and of the bin edges, about 2e-7 delta).
// The fast value counts when, in addition,
//   B <= min(1e-5, max(1e-6, distance of delta to the nearest real bin edge
//                      (and, off the standard range, to eps)))
// i.e. B is within the maximum's tolerance, and either B <= 1e-6 or no edge
// lies within B of delta; every other pair is recomputed.  A NaN Gram entry
// (how the caller marks a column that is not a real pair) fails the test.
struct PairVal {
    float delta, B, t;
    bool ok;
};

template <bool STD, bool DUMP>
__device__ __forceinline__ PairVal pair_value(float gx, float gy, const float4 ri, const float4 rj,
                                              const EpiConst &k, float4 *dump) {
    const float sx = __fadd_rn(ri.x, rj.x), sy = __fadd_rn(ri.y, rj.y);
    const float dx2 = fmaf(k.m2sx, gx, sx), dy2 = fmaf(k.m2sy, gy, sy);
    const float ex = fmaf(ri.z, rj.z, __fmul_rn(k.cx, sx)), ey = fmaf(ri.w, rj.w, __fmul_rn(k.cy, sy));
    if (DUMP) *dump = make_float4(dx2, dy2, ex * (1.0f / kBoundCoef), ey * (1.0f / kBoundCoef));
    const float pp = __fmul_rn(dx2, dy2);
    const float r = rsqrtf(pp);
    PairVal v;
    v.delta = __fdividef(fabsf(__fsub_rn(dy2, dx2)), fmaf(pp, r, dx2));
    const float rho = __fmul_rn(dy2, r);
    const float sab = __fmul_rn(fmaf(ex, dy2, __fmul_rn(ey, dx2)), __fmul_rn(r, r));
    v.B = fmaf(rho, sab, fmaf(1.25e-6f, v.delta, 1e-9f));
    v.t = STD ? __fmul_rn(v.delta, k.inv_w) : fmaf(v.delta, k.inv_w, k.t0);
    // distance to the nearest real edge: edges lie at integer t in [tlo + 0.5, 64]
    const float tc = fminf(fmaxf(v.t, k.tlo), (float)kBins + 0.5f);
    const float dedge = __fmul_rn(fabsf(__fsub_rn(tc, rintf(tc))), k.w);
    const float near = STD ? dedge : fminf(dedge, fabsf(__fsub_rn(v.delta, k.eps)));
    const float lim = fminf(kMaxTol, fmaxf(kExempt, near));
    v.ok = (fminf(dx2, dy2) > 0.0f) & (sab <= kCondMax) & (v.B <= lim);
    return v;
}

// Two FP32 values in one 64-bit register pair, for the packed (f32x2)
// instructions: each lane is rounded to nearest exactly like the scalar
// instruction, so a packed evaluation gives the scalar one's bits.
typedef unsigned long long f2;

__device__ __forceinline__ f2 pk2(float a, float b) {
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void upk2(f2 v, float &a, float &b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ f2 fadd2(f2 a, f2 b) {
    f2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2 fsub2(f2 a, f2 b) {
    f2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2 fmul2(f2 a, f2 b) {
    f2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
// a b + c, one rounding per lane
__device__ __forceinline__ f2 ffma2(f2 a, f2 b, f2 c) {
    f2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}

// A JL-prefix candidate's running data in one epilogue thread while it
// judges one tile row.  nrmh = -(largest upper bound on a pair's r) and rnl =
// smallest lower bound, each in both lanes of a packed value; rml and rnh are
// the other-side bounds of the pairs that set those records (lower bounds on
// the largest distortion that some pair certainly has).
struct CandRun {
    f2 nrmh, rnl;
    float rml, rnh;
    unsigned certain, open;
};
// The row's statistics for one candidate, each twice: the X row's |xc|^2 and
// q4 (times kraw, so the X bound comes out raw), the candidate's |yP|^2,
// PCA-part q4, |yJc|^2 and whole-prefix q4.
struct CandRow {
    f2 nx, qx, nP, qP, nJ, qT;
};
// The candidate's constants, each twice.
struct CandK {
    f2 m2sx, m2sy, cxr, lam, cypr, cyc, u2r, nuf, lf;
};

// Entry c of a candidate array in the kernel parameters, read with constant
// indices (a computed index would copy the parameters to local memory).
template <typename T>
__device__ __forceinline__ T cand_sel(const T (&v)[kMaxCand], int c) {
    static_assert(kMaxCand == 4, "cand_sel selects among four");
    return c == 0 ? v[0] : (c == 1 ? v[1] : (c == 2 ? v[2] : v[3]));
}

// Bounds xl <= dx2 <= xh and yl <= dy2 <= yh of two pairs (columns j, j + 1
// of one row) under one candidate, yl returned negated.  gx, gP, g: the
// pairs' X Gram sums, PCA-part Y sums and running prefix sums; xa, xb: the
// columns' pair-interleaved X statistics (|xc|^2 pair, q4x pair); ca, cb: the
// candidate's.  dy2 = dP + lam dJ with dP from gP and dJ from g - gP; its
// error bound eP + lam (eT + eP + u2 sT) takes the PCA part's bound eP, the
// whole prefix's eT (the error of g) and the rounding of g - gP.
__device__ __forceinline__ void cand_bounds2(f2 gx, f2 gP, f2 g, const CandRow &ri, const ulonglong2 xa,
                                             const ulonglong2 xb, const ulonglong2 ca, const ulonglong2 cb,
                                             const CandK &K, f2 &xl, f2 &xh, f2 &yh, f2 &nyl) {
    const f2 sx = fadd2(ri.nx, xa.x);
    const f2 dx2 = ffma2(K.m2sx, gx, sx);
    const f2 ex = ffma2(ri.qx, xb.x, fmul2(K.cxr, sx));
    const f2 sP = fadd2(ri.nP, ca.x), sJ = fadd2(ri.nJ, cb.x), sT = fadd2(sP, sJ);
    const f2 dP = ffma2(K.m2sy, gP, sP);
    const f2 dJ = ffma2(K.m2sy, fsub2(g, gP), sJ);
    const f2 dy2 = ffma2(K.lam, dJ, dP);
    const f2 eP = ffma2(ri.qP, ca.y, fmul2(K.cypr, sP));
    const f2 eT = ffma2(ri.qT, cb.y, fmul2(K.cyc, sT));
    const f2 ey = ffma2(K.lam, ffma2(K.u2r, sT, fadd2(eT, eP)), eP);
    xl = fsub2(dx2, ex);
    xh = fadd2(dx2, ex);
    yh = fadd2(dy2, ey);
    nyl = fsub2(ey, dy2);
}

// The distortion of Eq. 2 is |sqrt(r) - 1| for r = dy2 / dx2, so a pair with
// xl > 0 certainly stays within eps when yh <= uf xl and yl >= lf xh
// ((1 + eps)^2 and (1 - eps)^2 with 32 units of rounding slack).  The common
// path tests that and the two running records of r with four fused
// multiply-adds per pair (each sign exact): 2 bits per column pair, set where
// a valid pair needs the full test.
__device__ __forceinline__ unsigned cand_fast2(f2 xl, f2 xh, f2 yh, f2 nyl, bool v0, bool v1, const CandK &K,
                                               const CandRun &a) {
    const f2 C = ffma2(K.nuf, xl, yh);      // yh - uf xl
    const f2 D = ffma2(K.lf, xh, nyl);      // lf xh - yl
    const f2 E1 = ffma2(a.nrmh, xl, yh);    // yh - rmh xl
    const f2 E3 = ffma2(a.rnl, xh, nyl);    // rnl xh - yl
    float c0, c1, d0, d1, e0, e1, f0, f1;
    upk2(C, c0, c1);
    upk2(D, d0, d1);
    upk2(E1, e0, e1);
    upk2(E3, f0, f1);
    // a NaN (only from 0 x inf) compares false below and goes to the full test
    const bool ok0 = (c0 <= 0.0f) & (d0 <= 0.0f) & (e0 <= 0.0f) & (f0 <= 0.0f);
    const bool ok1 = (c1 <= 0.0f) & (d1 <= 0.0f) & (e1 <= 0.0f) & (f1 <= 0.0f);
    return (v0 & !ok0 ? 1u : 0u) | (v1 & !ok1 ? 2u : 0u);
}

// The full test of one pair: it certainly exceeds eps when yl > uv xh or
// yh < lv xl, certainly does not when the common-path conditions hold, and is
// open otherwise.  An open pair (i, j) goes to the candidates' queue, where an
// exact recompute decides it; a pair with xl <= 0 (possibly x_i == x_j, which
// the certificate excludes) is always open.  Only an open pair the full queue
// cannot take leaves the largest r unbounded.
__device__ __forceinline__ void cand_slow(float xl, float xh, float yh, float nyl, int i, int j, int c,
                                          const TcMulti &m, CandRun &a) {
    const float yl = -nyl;
    const bool pos = xl > 0.0f;
    const bool viol = pos & ((fmaf(-m.uv, xh, yl) > 0.0f) | (fmaf(m.lv, xl, -yh) > 0.0f));
    const bool fine = pos & (fmaf(-m.uf, xl, yh) <= 0.0f) & (fmaf(m.lf, xh, -yl) <= 0.0f);
    const bool open = !viol & !fine;
    a.certain += viol ? 1u : 0u;
    a.open += open ? 1u : 0u;
    bool queued = false;
    if (open) {
        const unsigned long long q = atomicAdd(m.cqcount, 1ull);
        if (q < m.cqcap) {
            m.cq[q] = make_int4(i, j, c, 0);
            queued = true;
        }
    }
    float nrmh, rnl, u;
    upk2(a.nrmh, nrmh, u);
    upk2(a.rnl, rnl, u);
    if (!pos) {
        if (!queued) nrmh = -INFINITY;
    } else {
        if (fmaf(nrmh, xl, yh) > 0.0f) {  // a new largest upper bound
            nrmh = fminf(nrmh, -__fdiv_ru(yh, xl));
            a.rml = fmaxf(a.rml, __fdiv_rd(yl, xh));
        }
        if (fmaf(rnl, xh, -yl) > 0.0f) {  // a new smallest lower bound
            rnl = fminf(rnl, fmaxf(__fdiv_rd(yl, xh), 0.0f));
            a.rnh = fminf(a.rnh, __fdiv_ru(yh, xl));
        }
    }
    a.nrmh = pk2(nrmh, nrmh);
    a.rnl = pk2(rnl, rnl);
}

// The row's statistics and the kernel constants, each twice (one per lane of
// a packed value).
struct RowPk {
    f2 n2x, n2y, q4x, q4y;
};
struct EpiPk {
    f2 m2sx, m2sy, cx, cy, inv_w, t0, w, c_rel, c_abs;
};

// pair_value for the two columns of a column pair: `ja` holds their
// (|xc|^2, |yc|^2) and `jb` their scaled q4 pairs (the pair-interleaved row
// statistics).  The same operations as pair_value, two lanes at a time, so
// both return the same bits for the same pair.
template <bool STD, bool DUMP>
__device__ __forceinline__ void pair_value2(f2 gx, f2 gy, const RowPk &ri, const ulonglong2 ja,
                                            const ulonglong2 jb, const EpiConst &k, const EpiPk &kp,
                                            PairVal (&v)[2], float4 *dump) {
    const f2 sx = fadd2(ri.n2x, ja.x), sy = fadd2(ri.n2y, ja.y);
    const f2 dx2 = ffma2(kp.m2sx, gx, sx), dy2 = ffma2(kp.m2sy, gy, sy);
    const f2 ex = ffma2(ri.q4x, jb.x, fmul2(kp.cx, sx)), ey = ffma2(ri.q4y, jb.y, fmul2(kp.cy, sy));
    float dx[2], dy[2];
    upk2(dx2, dx[0], dx[1]);
    upk2(dy2, dy[0], dy[1]);
    if (DUMP) {
        float e[2], f[2];
        upk2(ex, e[0], e[1]);
        upk2(ey, f[0], f[1]);
        for (int q = 0; q < 2; ++q)
            dump[q] = make_float4(dx[q], dy[q], e[q] * (1.0f / kBoundCoef), f[q] * (1.0f / kBoundCoef));
    }
    const f2 pp = fmul2(dx2, dy2);
    float pq[2], num[2], den[2];
    upk2(pp, pq[0], pq[1]);
    const f2 r = pk2(rsqrtf(pq[0]), rsqrtf(pq[1]));
    upk2(fsub2(dy2, dx2), num[0], num[1]);
    upk2(ffma2(pp, r, dx2), den[0], den[1]);
    const f2 delta = pk2(__fdividef(fabsf(num[0]), den[0]), __fdividef(fabsf(num[1]), den[1]));
    const f2 rho = fmul2(dy2, r);
    const f2 sab = fmul2(ffma2(ex, dy2, fmul2(ey, dx2)), fmul2(r, r));
    const f2 B = ffma2(rho, sab, ffma2(kp.c_rel, delta, kp.c_abs));
    const f2 t = STD ? fmul2(delta, kp.inv_w) : ffma2(delta, kp.inv_w, kp.t0);
    float tq[2], sq[2];
    upk2(delta, v[0].delta, v[1].delta);
    upk2(B, v[0].B, v[1].B);
    upk2(t, tq[0], tq[1]);
    upk2(sab, sq[0], sq[1]);
    float tc[2], rn[2];
    for (int q = 0; q < 2; ++q) {
        v[q].t = tq[q];
        // distance to the nearest real edge: edges lie at integer t in [tlo + 0.5, 64]
        tc[q] = fminf(fmaxf(tq[q], k.tlo), (float)kBins + 0.5f);
        rn[q] = rintf(tc[q]);
    }
    float dd[2], de[2];
    upk2(fsub2(pk2(tc[0], tc[1]), pk2(rn[0], rn[1])), dd[0], dd[1]);
    upk2(fmul2(pk2(fabsf(dd[0]), fabsf(dd[1])), kp.w), de[0], de[1]);
    for (int q = 0; q < 2; ++q) {
        const float near = STD ? de[q] : fminf(de[q], fabsf(__fsub_rn(v[q].delta, k.eps)));
        const float lim = fminf(kMaxTol, fmaxf(kExempt, near));
        v[q].ok = (fminf(dx[q], dy[q]) > 0.0f) & (sq[q] <= kCondMax) & (v[q].B <= lim);
    }
}

// Classifies the kPiece pairs (i, j0 + c0 + c) of one tile row, without
// data-dependent branches, so the compiler interleaves the independent
// pairs.  Counted pairs go into their histogram bin (bin 64: outside the
// range) and the row statistics; the others set bit c of q8 (the piece's
// queue mask).
template <bool DUMP, bool STD>
__device__ __forceinline__ void classify_piece(const float (&gx)[kPiece], const float (&gy)[kPiece],
                                               const float4 ri, const ulonglong2 *__restrict__ rsj2,
                                               const EpiConst &k, uint32_t *hrow, RowAcc &a,
                                               float &pm, uint32_t &q8, float4 *dump_row) {
    const RowPk rp{pk2(ri.x, ri.x), pk2(ri.y, ri.y), pk2(ri.z, ri.z), pk2(ri.w, ri.w)};
    const EpiPk kp{pk2(k.m2sx, k.m2sx), pk2(k.m2sy, k.m2sy), pk2(k.cx, k.cx),   pk2(k.cy, k.cy),
                   pk2(k.inv_w, k.inv_w), pk2(k.t0, k.t0),   pk2(k.w, k.w),     pk2(1.25e-6f, 1.25e-6f),
                   pk2(1e-9f, 1e-9f)};
#pragma unroll
    for (int c = 0; c < kPiece; c += 2) {
        PairVal v[2];
        pair_value2<STD, DUMP>(pk2(gx[c], gx[c + 1]), pk2(gy[c], gy[c + 1]), rp, __ldg(rsj2 + c),
                               __ldg(rsj2 + c + 1), k, kp, v, DUMP ? dump_row + c : nullptr);
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            q8 |= v[q].ok ? 0u : (1u << (c + q));
            int bin;
            if (STD) {
                bin = min((int)v[q].t, kBins);
            } else {
                bin = ((v[q].t >= 0.0f) & (v[q].t < (float)kBins)) ? (int)v[q].t : kBins;
                a.viol += (v[q].ok & (v[q].delta > k.eps)) ? 1 : 0;
            }
            atomicAdd(hrow + bin * kHRows, v[q].ok ? 1u : 0u);
            const float dok = v[q].ok ? v[q].delta : 0.0f;
            a.sum = __fadd_rn(a.sum, dok);
            pm = fmaxf(pm, dok);
            a.mxb = fmaxf(a.mxb, v[q].ok ? v[q].B : 0.0f);
        }
    }
}

// ---------------------------------------------------------------- the kernel
template <bool DUMP, bool PAIR, bool STD, bool MULTI = false>
__global__ void __launch_bounds__(kThreads, 1)
    cert_tc_kernel(const __grid_constant__ CUtensorMap map_xh, const __grid_constant__ CUtensorMap map_xl,
                   const __grid_constant__ CUtensorMap map_yh, const __grid_constant__ CUtensorMap map_yl,
                   const __grid_constant__ CUtensorMap bmap_xh, const __grid_constant__ CUtensorMap bmap_xl,
                   const __grid_constant__ CUtensorMap bmap_yh, const __grid_constant__ CUtensorMap bmap_yl,
                   TcArgs p) {
    using L = Layout<PAIR, MULTI>;
    constexpr int kStages = L::kStages;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    // 1024-byte alignment of the stage buffers (128-byte swizzle atoms), by
    // an offset from the shared array so the address space stays known; the
    // offset is the same in both CTAs of a pair, which the MMA relies on
    uint8_t *smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    const uint32_t sbase = smem_u32(smem);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // identity: the pair's two CTAs share a tile sequence; rank 0 leads
    const uint32_t rank = PAIR ? cluster_ctarank() : 0u;
    const bool leader = rank == 0;

    uint32_t *s_hist = reinterpret_cast<uint32_t *>(smem + L::hist);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + L::bars);
    int *s_cmd = reinterpret_cast<int *>(smem + L::cmd);  // [kStages] stage, [kStages + s] slot
    int *s_dec = reinterpret_cast<int *>(smem + L::dec);  // pair: the leader's decisions for the peer
    uint32_t *s_tmem = reinterpret_cast<uint32_t *>(smem + L::tmem_ptr);
    const uint32_t bar_full = smem_u32(bars);                 // [kStages]
    const uint32_t bar_empty = bar_full + 8 * kStages;        // [kStages]
    const uint32_t bar_sfull = bar_empty + 8 * kStages;       // [kSlots]
    const uint32_t bar_sempty = bar_sfull + 8 * kSlots;       // [kSlots]
    const uint32_t bar_done = bar_sempty + 8 * kSlots;        // MMA drain
    const uint32_t bar_dfull = bar_done + 8;                  // [2] pair: decision posted (peer)
    const uint32_t bar_dempty = bar_dfull + 16;               // [2] pair: decision taken (leader)
    const uint32_t bar_epi = bar_dempty + 16;                 // every epilogue thread is done

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(bar_full + 8 * s, 1);
            mbar_init(bar_empty + 8 * s, 1);
        }
        for (int s = 0; s < kSlots; ++s) {
            mbar_init(bar_sfull + 8 * s, 1);
            // one arrival per epilogue warp (of both CTAs of a pair)
            // every epilogue thread arrives (a pair: one arrival per warp of both CTAs)
            mbar_init(bar_sempty + 8 * s, PAIR ? 2 * kEpiWarps : kEpiWarps);
        }
        mbar_init(bar_done, 1);
        for (int q = 0; q < 2; ++q) {
            mbar_init(bar_dfull + 8 * q, 1);
            mbar_init(bar_dempty + 8 * q, 1);
        }
        mbar_init(bar_epi, 32 * kEpiWarps);
        for (int q = 0; q < 16; ++q) s_cmd[q] = 0;
        for (int q = 0; q < 4; ++q) s_dec[q] = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    for (int e = threadIdx.x; e < kHBins * kHRows; e += kThreads) s_hist[e] = 0;
    if (warp == 1) {
        if (PAIR) {
            // collective with the peer CTA's warp 1: the same columns in both
            asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                             smem_u32(s_tmem)),
                         "r"(kTmemCols)
                         : "memory");
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
        } else {
            asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                             smem_u32(s_tmem)),
                         "r"(kTmemCols)
                         : "memory");
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
        }
    }
    tc_fence_before();
    // a pair: no CTA touches the other's barriers before both are initialised
    if (PAIR)
        cluster_sync();
    else
        __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *s_tmem;
    const int ksteps = p.ky_steps + p.kx_steps;

    if (warp == 0) {
        // ------------------------------------------------------ TMA producer
        // Both CTAs of a pair load the same stages of the same tiles: each its
        // own 128 I rows and its half of the J rows; every copy completes on
        // the leader's full barrier, which expects the bytes of both.
        int stage = 0;
        uint32_t phase = 0;
        bool ok = true;
        uint32_t issued_parity[kStages];
        bool issued[kStages];
        for (int s = 0; s < kStages; ++s) issued[s] = false, issued_parity[s] = 0;
        const uint32_t full_tgt = PAIR ? mapa(bar_full, 0) : bar_full;
        long long t = PAIR ? (long long)cluster_id_x() : (long long)blockIdx.x;
        for (long long k = 0; ok; ++k, t += PAIR ? (long long)ncluster_x() : (long long)gridDim.x) {
            bool stop;
            const int q = (int)(k & 1);
            const uint32_t use = (uint32_t)(k >> 1) & 1u;
            if (leader) {
                stop = t >= p.ntp;
                if (!stop && p.stop_flag) {
                    int f = 0;
                    if (lane == 0) f = *(volatile int *)p.stop_flag;
                    stop = __shfl_sync(0xffffffffu, f, 0) != 0;
                }
                if (PAIR) {
                    // post the decision in the peer's shared memory (decision
                    // slot q, once the peer has taken the one posted two tiles ago)
                    ok = warp_wait<true>(bar_dempty + 8 * q, use ^ 1u, p.status, 1);
                    if (!ok) break;
                    if (lane == 0) {
                        st_cluster_u32(mapa(smem_u32(s_dec + q), 1), stop ? 0xFFFFFFFFu : 1u);
                        mbar_arrive_cluster(mapa(bar_dfull + 8 * q, 1));
                    }
                    __syncwarp();
                }
            } else {
                ok = warp_wait<true>(bar_dfull + 8 * q, use, p.status, 1);
                if (!ok) break;
                int dec = 0;
                if (lane == 0) {
                    dec = ((volatile int *)s_dec)[q];
                    mbar_arrive_cluster(mapa(bar_dempty + 8 * q, 0));
                }
                stop = __shfl_sync(0xffffffffu, dec, 0) < 0;
            }
            if (stop) {
                if (leader) {
                    if (lane == 0 && mbar_wait<PAIR>(bar_empty + 8 * stage, phase ^ 1, p.status, 1)) {
                        s_cmd[stage] = -1;
                        mbar_arrive(bar_full + 8 * stage);
                    }
                    // the empty wait proved the stage's last copy was consumed,
                    // and the stop arrive moved its full barrier one phase on:
                    // nothing of this stage is left to drain
                    issued[stage] = false;
                }
                __syncwarp();
                break;
            }
            const uint32_t packed = p.sched[t];
            const int I = (int)(packed >> 16), J = (int)(packed & 0xFFFF);
            const int arow = PAIR ? I * 2 * kTile + (int)rank * kTile : I * kTile;
            const int brow = J * kTile + (int)rank * L::kBRows;
            for (int ks = 0; ks < ksteps; ++ks) {
                ok = warp_wait<PAIR>(bar_empty + 8 * stage, phase ^ 1, p.status, 1);
                if (!ok) break;
                if (lane == 0) {
                    if (leader) {
                        if (ks == 0) s_cmd[stage] = (int)t;
                        mbar_arrive_expect_tx(bar_full + 8 * stage, L::kTxBytes);
                    }
                    const uint32_t bar = full_tgt + 8 * stage;
                    const uint32_t dst = sbase + L::stages + stage * L::kStageBytes;
                    const bool is_y = ks >= p.kx_steps;
                    const int k0 = (is_y ? ks - p.kx_steps : ks) * kKStep;
                    const CUtensorMap *mh = is_y ? &map_yh : &map_xh;
                    const CUtensorMap *ml = is_y ? &map_yl : &map_xl;
                    const CUtensorMap *bh = is_y ? &bmap_yh : &bmap_xh;
                    const CUtensorMap *bl = is_y ? &bmap_yl : &bmap_xl;
                    tma_load_2d<PAIR>(dst, mh, k0, arow, bar);
                    tma_load_2d<PAIR>(dst + kAPlane, ml, k0, arow, bar);
                    tma_load_2d<PAIR>(dst + 2 * kAPlane, bh, k0, brow, bar);
                    tma_load_2d<PAIR>(dst + 2 * kAPlane + L::kBPlane, bl, k0, brow, bar);
                }
                __syncwarp();
                issued[stage] = true;
                issued_parity[stage] = phase;
                if (++stage == kStages) {
                    stage = 0;
                    phase ^= 1;
                }
            }
        }
        // drain: every issued copy must have landed before the CTA can exit.
        // The leader's full barriers count the copies of both CTAs; the peer
        // waits until the MMA has consumed its last copies (every started
        // tile is consumed whole).
        if (lane == 0)
            for (int s = 0; s < kStages; ++s)
                if (issued[s]) {
                    if (leader)
                        mbar_wait<PAIR>(bar_full + 8 * s, issued_parity[s], p.status, 1);
                    else
                        mbar_wait<true>(bar_empty + 8 * s, issued_parity[s], p.status, 1);
                }
        __syncwarp();
    } else if (warp == 1) {
        // ------------------------------------------------------- MMA issuer
        // Every K step accumulates into a fresh TMEM slot (128 columns): first
        // the 8 small cross-term products (hi.lo, lo.hi), then the 4 large
        // hi.hi products, so only 4 FP32 accumulator roundings per chunk act
        // on full-size partial sums.  The epilogue drains the slot.  In a pair
        // only the leader issues; the peer's warp 1 only holds TMEM.
        if (leader) {
            int stage = 0, slot = 0;
            uint32_t phase = 0, sphase = 0;
            bool any = false;
            bool ok = true;
            while (ok) {
                int t = -1;
                ok = warp_wait<PAIR>(bar_full + 8 * stage, phase, p.status, 2);
                if (!ok) break;
                if (lane == 0) t = s_cmd[stage];
                t = __shfl_sync(0xffffffffu, t, 0);
                if (t < 0) {
                    // forward the stop to the epilogues through the next slot;
                    // the plain (release) arrive publishes the stop word
                    if (lane == 0 && mbar_wait<PAIR>(bar_sempty + 8 * slot, sphase ^ 1, p.status, 2)) {
                        s_cmd[kStages + slot] = -1;
                        if (PAIR) st_cluster_u32(mapa(smem_u32(s_cmd + kStages + slot), 1), 0xFFFFFFFFu);
                        mbar_arrive(bar_sfull + 8 * slot);
                        if (PAIR) mbar_arrive_cluster(mapa(bar_sfull + 8 * slot, 1));
                    }
                    __syncwarp();
                    break;
                }
                for (int ks = 0; ks < ksteps; ++ks) {
                    if (ks > 0) {
                        ok = warp_wait<PAIR>(bar_full + 8 * stage, phase, p.status, 2);
                        if (!ok) break;
                    }
                    ok = warp_wait<PAIR>(bar_sempty + 8 * slot, sphase ^ 1, p.status, 2);
                    if (!ok) break;
                    tc_fence_after();
                    // the descriptors are warp-uniform values; one elected
                    // lane issues the MMAs and the commits
                    const uint32_t d = tmem_base + (uint32_t)(slot * kTile);
                    const uint32_t a0 = sbase + L::stages + stage * L::kStageBytes;
                    const uint64_t ah = sw128_desc(a0), al = sw128_desc(a0 + kAPlane);
                    const uint64_t bh = sw128_desc(a0 + 2 * kAPlane);
                    const uint64_t bl = sw128_desc(a0 + 2 * kAPlane + L::kBPlane);
                    if (elect_one()) {
#pragma unroll
                        for (int kk = 0; kk < kKStep / 16; ++kk) {
                            const uint64_t off = (uint64_t)(kk * 32) >> 4;  // 16 elements = 32 bytes
                            tc_mma<PAIR>(d, ah + off, bl + off, p.idesc, kk == 0 ? 0u : 1u);
                            tc_mma<PAIR>(d, al + off, bh + off, p.idesc, 1u);
                        }
#pragma unroll
                        for (int kk = 0; kk < kKStep / 16; ++kk) {
                            const uint64_t off = (uint64_t)(kk * 32) >> 4;
                            tc_mma<PAIR>(d, ah + off, bh + off, p.idesc, 1u);
                        }
                        tc_commit<PAIR>(bar_empty + 8 * stage);
                        tc_commit<PAIR>(bar_sfull + 8 * slot);
                        any = true;
                    }
                    __syncwarp();
                    if (++stage == kStages) {
                        stage = 0;
                        phase ^= 1;
                    }
                    if (++slot == kSlots) {
                        slot = 0;
                        sphase ^= 1;
                    }
                }
            }
            // all issued MMAs must be complete before TMEM is released
            any = __shfl_sync(0xffffffffu, any ? 1 : 0, 0) != 0;
            if (lane == 0 && any) {
                tc_commit_local<PAIR>(bar_done);
                mbar_wait(bar_done, 0, p.status, 2);
            }
            __syncwarp();
        }
    } else {
        // --------------------------------------------------------- epilogue
        // Three warps per TMEM lane quarter (warp % 4), i.e. tile row r; warp
        // part h of the quarter owns columns [col0, col0 + NC) of the tile
        // (48, 40, 40 columns).  The K chunks of a tile come X first, then Y.
        // The chunks are summed in registers: the X sums are parked in the
        // TMEM staging columns at the first Y chunk, the Y sums in the running
        // columns at the end of the tile, and the tile is then pending.  The
        // classification of a tile is software-pipelined into the next one: it
        // runs piece by piece between the next tile's X-chunk drains, while the
        // MMA warp computes that tile, and is finished at the next tile's first
        // Y chunk, before its X sums overwrite the staging columns.
        const int ew = warp - 2;                 // 0 .. kEpiWarps - 1
        const int quarter = warp & 3;
        const int h = ew >> 2;                   // part of the quarter: 0, 1, 2
        const int col0 = kEpiWarps == 8 ? 64 * h : (h == 0 ? 0 : (h == 1 ? 48 : 88));
        const int r = quarter * 32 + lane;       // tile row of this thread
        const uint32_t lane_addr = (uint32_t)(quarter * 32) << 16;
        const uint32_t gx_stage = tmem_base + lane_addr + kStageCol + (uint32_t)col0;
        const uint32_t gy_run = gx_stage + kTile;
        // the slot-drained barrier is the leader's
        const uint32_t sempty_tgt = PAIR ? mapa(bar_sempty, 0) : bar_sempty;
        auto epilogue = [&](auto ncols) {
        constexpr int NC = decltype(ncols)::value;
        constexpr int NP = NC / kPiece;          // pieces of a tile row
        CertPartial *mine = p.partials + (size_t)blockIdx.x * kEpiWarps + ew;
        int slot = 0;
        uint32_t sphase = 0;
        EpiConst k;
        {
            const float sx = *p.scale_x, sy = *p.scale_y;
            k.m2sx = -2.0f / (sx * sx);
            k.m2sy = -2.0f / (sy * sy);
            k.cx = p.cx;
            k.cy = p.cy;
            k.inv_w = p.cc.inv_w;
            k.t0 = -p.cc.lo * p.cc.inv_w;
            k.w = p.cc.w;
            // with lo <= 0 the lower edge is no boundary (distortions are >= 0)
            k.tlo = p.cc.lo_is_floor ? 0.5f : -0.5f;
            k.eps = p.cc.eps;
        }
        WarpTotals *wt = reinterpret_cast<WarpTotals *>(smem + L::totals) + ew;
        if (lane == 0) {
            wt->violations = wt->queued = 0;
            wt->sum = wt->bound_sum = 0.0;
            wt->max = -1.0f;
            wt->max_bound = 0.0f;
            wt->argmax_i = wt->argmax_j = 0x7fffffff;
        }
        uint32_t *hrow = s_hist + r;  // bin b of this tile row at hrow[b * kHRows]
        // the tile waiting for (or in) classification
        bool pend = false, pend_full = false;
        int pend_pieces = 0;
        long long pend_u = 0;
        int pend_i = 0, pend_j0 = 0;
        float4 pend_ri = make_float4(0.f, 0.f, 0.f, 0.f);
        unsigned long long pend_vmask = 0ull, qmask = 0ull;
        RowAcc acc{0.0f, 0.0f, -1.0f, 0, 0};

        // the pending tile's Gram entries of one piece (NaN where not a pair)
        auto load_piece = [&](int c0, float (&px)[kPiece], float (&py)[kPiece]) {
            uint32_t ux[kPiece], uy[kPiece];
            tmem_ld8x2_wait(gx_stage + c0, gy_run + c0, ux, uy);
            if (pend_full) {
#pragma unroll
                for (int c = 0; c < kPiece; ++c) {
                    px[c] = __uint_as_float(ux[c]);
                    py[c] = __uint_as_float(uy[c]);
                }
            } else {
                // this piece's valid-pair bits; bit c is a constant after unrolling
                const uint32_t v8 = (uint32_t)(pend_vmask >> c0) & 0xFFu;
#pragma unroll
                for (int c = 0; c < kPiece; ++c) {
                    const bool valid = (v8 >> c) & 1u;
                    px[c] = valid ? __uint_as_float(ux[c]) : __int_as_float(0x7fc00000);
                    py[c] = __uint_as_float(uy[c]);
                }
            }
        };
        // classifies the next 8-column piece of the pending tile
        auto classify_next = [&]() {
            const int c0 = pend_pieces * kPiece;
            float px[kPiece], py[kPiece];
            load_piece(c0, px, py);
            uint32_t q8 = 0u;
            float pm = -1.0f;
            if (DUMP && p.dump && pend_u % p.dump_stride == 0 && pend_u / p.dump_stride < p.dump_tiles) {
                float4 *drow = p.dump + (size_t)(pend_u / p.dump_stride) * kTile * kTile + r * kTile +
                               col0 + c0;
                classify_piece<DUMP, STD>(px, py, pend_ri, p.rs2 + pend_j0 + c0, k, hrow, acc, pm, q8, drow);
            } else {
                classify_piece<false, STD>(px, py, pend_ri, p.rs2 + pend_j0 + c0, k, hrow, acc, pm, q8,
                                           nullptr);
            }
            const bool better = pm > acc.mx;
            acc.mx = better ? pm : acc.mx;
            acc.mp = better ? pend_pieces : acc.mp;
            qmask |= (unsigned long long)q8 << c0;
            ++pend_pieces;
        };
        // the first column at or after piece `from` of this lane's row where a
        // counted pair has distortion `target` (-1: none); every lane takes
        // part (the TMEM loads are warp-wide), lane `who` searches
        auto find_column = [&](int from, float target, int who) -> int {
            int found = -1;
            for (int piece = from; piece < NP; ++piece) {
                const int c0 = piece * kPiece;
                float px[kPiece], py[kPiece];
                load_piece(c0, px, py);
#pragma unroll
                for (int c = 0; c < kPiece; ++c) {
                    const PairVal v = pair_value<STD, false>(px[c], py[c], pend_ri,
                                                             __ldg(p.rs + pend_j0 + c0 + c), k, nullptr);
                    if (found < 0 && v.ok && v.delta == target) found = c0 + c;
                }
                found = __shfl_sync(0xffffffffu, found, who);
                if (found >= 0) break;
            }
            return found;
        };
        // queue pushes and warp totals of the fully classified pending tile
        auto finish_pending = [&]() {
            while (pend_pieces < NP) classify_next();
            qmask &= pend_vmask;
            int nq = __popcll(qmask);
            const int nok = __popcll(pend_vmask & ~qmask);
            while (__any_sync(0xffffffffu, qmask != 0ull)) {
                const bool has = qmask != 0ull;
                const int c = has ? __ffsll((long long)qmask) - 1 : 0;
                if (has) qmask &= qmask - 1;
                queue_push(has, pend_i, pend_j0 + c, p.queue, p.qcount, p.qcap);
            }
            float sum = acc.sum, mxb = acc.mxb, tmax = acc.mx;
            // >= the sum of the row's bounds
            float bsum = __fmul_rn((float)nok, acc.mxb);
            int viol = acc.viol;
            for (int o = 16; o > 0; o >>= 1) {
                if (!STD) viol += __shfl_xor_sync(0xffffffffu, viol, o);
                nq += __shfl_xor_sync(0xffffffffu, nq, o);
                sum += __shfl_xor_sync(0xffffffffu, sum, o);
                bsum += __shfl_xor_sync(0xffffffffu, bsum, o);
                mxb = fmaxf(mxb, __shfl_xor_sync(0xffffffffu, mxb, o));
                tmax = fmaxf(tmax, __shfl_xor_sync(0xffffffffu, tmax, o));
            }
            // the maximum and its pair: searched for only when this tile can
            // hold the warp's maximum (ties included: the lexicographically
            // smallest pair wins).  Rows grow with the lane, so the first lane
            // whose row holds a counted pair at tmax has the smallest i.
            float wmax = -1.0f;
            int wi = 0x7fffffff, wj = 0x7fffffff;
            if (lane == 0) {
                wmax = wt->max;
                wi = wt->argmax_i;
                wj = wt->argmax_j;
            }
            wmax = __shfl_sync(0xffffffffu, wmax, 0);
            if (tmax >= wmax) {
                unsigned cand = __ballot_sync(0xffffffffu, acc.mx == tmax);
                while (cand) {
                    const int l = __ffs(cand) - 1;
                    cand &= cand - 1;
                    const int from = __shfl_sync(0xffffffffu, acc.mp, l);
                    const int c = find_column(from, tmax, l);
                    if (c >= 0) {
                        const int fi = __shfl_sync(0xffffffffu, pend_i, l);
                        const int fj = pend_j0 + c;
                        wi = __shfl_sync(0xffffffffu, wi, 0);
                        wj = __shfl_sync(0xffffffffu, wj, 0);
                        if (lane == 0 && better_max(tmax, fi, fj, wmax, wi, wj)) {
                            wt->max = tmax;
                            wt->argmax_i = fi;
                            wt->argmax_j = fj;
                        }
                        break;
                    }
                }
            }
            if (lane == 0) {
                if (!STD) wt->violations += (unsigned)viol;
                wt->queued += (unsigned)nq;
                wt->sum += (double)sum;
                wt->bound_sum += (double)bsum;
                wt->max_bound = fmaxf(wt->max_bound, mxb);
                // a certain violation: a counted pair with delta - B > eps
                // (its B is at most the maximum's tolerance)
                if (p.stop_flag && tmax > k.eps + kMaxTol) atomicExch(p.stop_flag, 1);
            }
            pend = false;
        };

        // the producer's static tile sequence; its entries are read a tile
        // ahead, so the row statistic a tile needs at its end is requested at
        // its start and neither load's latency is exposed
        long long t = PAIR ? (long long)cluster_id_x() : (long long)blockIdx.x;
        const long long tstep = PAIR ? (long long)ncluster_x() : (long long)gridDim.x;
        uint32_t nxt_packed = t < p.ntp ? __ldg(p.sched + t) : 0u;
        bool ok = true;
        // the JL-prefix candidates' verdict data (multi-candidate kernel): per
        // epilogue thread and candidate in shared memory, field f of
        // candidate c at [(c * F + f) * 256 + et]: -rmax_hi, rmax_lo,
        // rmin_lo, rmin_hi (CandRun), then the two counts
        const int et = ew * 32 + lane;
        float *s_cr = reinterpret_cast<float *>(smem + L::cand);  // rmh, rml, rnl, rnh
        unsigned long long *s_cn =
            reinterpret_cast<unsigned long long *>(smem + L::cand + kMaxCand * 4 * 32 * kEpiWarps * 4);
        if constexpr (MULTI) {
            for (int c = 0; c < p.multi.count; ++c) {
                s_cr[(c * 4 + 0) * 32 * kEpiWarps + et] = 0.0f;
                s_cr[(c * 4 + 1) * 32 * kEpiWarps + et] = 0.0f;
                s_cr[(c * 4 + 2) * 32 * kEpiWarps + et] = INFINITY;
                s_cr[(c * 4 + 3) * 32 * kEpiWarps + et] = INFINITY;
                s_cn[(c * 2 + 0) * 32 * kEpiWarps + et] = 0ull;
                s_cn[(c * 2 + 1) * 32 * kEpiWarps + et] = 0ull;
            }
        }
        // every pair of this thread's row of the current tile under candidate
        // c: the tile's X sums and PCA-part sums are in the staging and running
        // columns, its running Y sums in the TMEM columns at tg
        auto cand_check = [&](int c, uint32_t tg, uint32_t packed, int ib, float4 ri) {
            const TcMulti &m = p.multi;
            const int J = (int)(packed & 0xFFFF);
            const int i = ib * kTile + r;
            const int j0 = J * kTile + col0;
            const bool full = (ib < J) && (J * kTile + kTile <= p.n);
            const ulonglong2 *cs = m.cs + (size_t)c * (size_t)m.n_pad;
            const float lam_c = cand_sel(m.lam, c), cyc_c = cand_sel(m.cycr, c);
            CandRow cr;
            {
                const ulonglong2 a = __ldg(cs + (i & ~1)), b = __ldg(cs + (i | 1));
                float v0, v1;
                const bool odd = (i & 1) != 0;
                upk2(a.x, v0, v1);
                cr.nP = pk2(odd ? v1 : v0, odd ? v1 : v0);
                upk2(a.y, v0, v1);
                cr.qP = pk2(odd ? v1 : v0, odd ? v1 : v0);
                upk2(b.x, v0, v1);
                cr.nJ = pk2(odd ? v1 : v0, odd ? v1 : v0);
                upk2(b.y, v0, v1);
                cr.qT = pk2(odd ? v1 : v0, odd ? v1 : v0);
                cr.nx = pk2(ri.x, ri.x);
                const float qx = __fmul_ru(ri.z, m.kraw);
                cr.qx = pk2(qx, qx);
            }
            const int base = c * 4 * 32 * kEpiWarps + et;
            CandRun a;
            {
                const float f0 = s_cr[base], f2v = s_cr[base + 64 * kEpiWarps];
                a.nrmh = pk2(f0, f0);
                a.rnl = pk2(f2v, f2v);
                a.rml = s_cr[base + 32 * kEpiWarps];
                a.rnh = s_cr[base + 96 * kEpiWarps];
                a.certain = a.open = 0u;
            }
            CandK K;
            K.m2sx = pk2(k.m2sx, k.m2sx);
            K.m2sy = pk2(k.m2sy, k.m2sy);
            K.cxr = pk2(m.cxr, m.cxr);
            K.lam = pk2(lam_c, lam_c);
            K.cypr = pk2(m.cypr, m.cypr);
            K.cyc = pk2(cyc_c, cyc_c);
            K.u2r = pk2(m.u2r, m.u2r);
            K.nuf = pk2(-m.uf, -m.uf);
            K.lf = pk2(m.lf, m.lf);
            // pieces in a loop, not unrolled: the check's code stays small
            // enough for the instruction cache beside the main epilogue
#pragma unroll 1
            for (int pc = 0; pc < NP; ++pc) {
                uint32_t ux[kPiece], uy[kPiece], ug[kPiece];
                tmem_ld8x3_wait(gx_stage + pc * kPiece, gy_run + pc * kPiece, tg + pc * kPiece, ux, uy, ug);
                // the piece's pairs on the common path, branch-free; the
                // few that need the full test are redone below
                unsigned flag = 0u;
#pragma unroll
                for (int q = 0; q < kPiece; q += 2) {
                    const int cc = pc * kPiece + q;
                    const int j = j0 + cc;
                    const bool v0 = full || ((i < j) && (j < p.n));
                    const bool v1 = full || ((i < j + 1) && (j + 1 < p.n));
                    f2 xl, xh, yh, nyl;
                    cand_bounds2(pk2(__uint_as_float(ux[q]), __uint_as_float(ux[q + 1])),
                                 pk2(__uint_as_float(uy[q]), __uint_as_float(uy[q + 1])),
                                 pk2(__uint_as_float(ug[q]), __uint_as_float(ug[q + 1])), cr, __ldg(p.rs2 + j), __ldg(p.rs2 + j + 1), __ldg(cs + j), __ldg(cs + j + 1), K,
                                 xl, xh, yh, nyl);
                    flag |= cand_fast2(xl, xh, yh, nyl, v0, v1, K, a) << q;
                }
                if (__any_sync(0xffffffffu, flag != 0u)) {
#pragma unroll
                    for (int q = 0; q < kPiece; q += 2) {
                        if (flag & (3u << q)) {
                            const int cc = pc * kPiece + q;
                            const int j = j0 + cc;
                            f2 xl, xh, yh, nyl;
                            cand_bounds2(pk2(__uint_as_float(ux[q]), __uint_as_float(ux[q + 1])),
                                         pk2(__uint_as_float(uy[q]), __uint_as_float(uy[q + 1])),
                                         pk2(__uint_as_float(ug[q]), __uint_as_float(ug[q + 1])), cr,
                                         __ldg(p.rs2 + j), __ldg(p.rs2 + j + 1),
                                         __ldg(cs + j), __ldg(cs + j + 1), K, xl, xh, yh, nyl);
                            float l0, l1, h0, h1, y0, y1, n0, n1;
                            upk2(xl, l0, l1);
                            upk2(xh, h0, h1);
                            upk2(yh, y0, y1);
                            upk2(nyl, n0, n1);
                            if (flag & (1u << q)) cand_slow(l0, h0, y0, n0, i, j, c, m, a);
                            if (flag & (2u << q)) cand_slow(l1, h1, y1, n1, i, j + 1, c, m, a);
                        }
                    }
                }
            }
            {
                float f0, u;
                upk2(a.nrmh, f0, u);
                s_cr[base] = f0;
                s_cr[base + 32 * kEpiWarps] = a.rml;
                upk2(a.rnl, f0, u);
                s_cr[base + 64 * kEpiWarps] = f0;
                s_cr[base + 96 * kEpiWarps] = a.rnh;
                s_cn[(c * 2 + 0) * 32 * kEpiWarps + et] += a.certain;
                s_cn[(c * 2 + 1) * 32 * kEpiWarps + et] += a.open;
            }
        };
        // this warp's NC sums into TMEM columns starting at `dst`
        auto park = [&](const float (&v)[NC], uint32_t dst) {
#pragma unroll
            for (int qd = 0; qd < NC / 16; ++qd) {
                uint32_t u[16];
#pragma unroll
                for (int c = 0; c < 16; ++c) u[c] = __float_as_uint(v[qd * 16 + c]);
                tmem_st16(dst + qd * 16, u);
            }
            if constexpr (NC % 16 != 0) {
                uint32_t u[8];
#pragma unroll
                for (int c = 0; c < 8; ++c) u[c] = __float_as_uint(v[NC - 8 + c]);
                tmem_st8(dst + NC - 8, u);
            }
            tmem_wait_st();
        };
        while (ok) {
            const uint32_t cur_packed = nxt_packed;
            nxt_packed = t + tstep < p.ntp ? __ldg(p.sched + t + tstep) : 0u;
            // this CTA's 128-row block of the tile and the row statistic of this thread's row
            const int cur_ib = PAIR ? 2 * (int)(cur_packed >> 16) + (int)rank : (int)(cur_packed >> 16);
            const float4 cur_ri = __ldg(p.rs + cur_ib * kTile + r);
            // the tile's X sums, then (once they are parked) its Y sums
            float g[NC];
#pragma unroll
            for (int c = 0; c < NC; ++c) g[c] = 0.0f;
            bool stop = false;
            for (int ks = 0; ks < ksteps; ++ks) {
                ok = warp_wait<PAIR>(bar_sfull + 8 * slot, sphase, p.status, 3);
                if (!ok) break;
                tc_fence_after();
                if (ks == 0) {
                    int cmdv = 0;
                    if (lane == 0) cmdv = s_cmd[kStages + slot];
                    if (__shfl_sync(0xffffffffu, cmdv, 0) < 0) {
                        stop = true;
                        break;
                    }
                }
                if (ks == p.kx_steps) {
                    // the first Y chunk: the pending tile's classification ends
                    // here (it reads the staging columns), then the X sums are
                    // parked there and the registers take the Y sums
                    if (pend) finish_pending();
                    park(g, gx_stage);
                    if constexpr (MULTI) {
                        // the column statistics the candidates' checks read
                        // (8 lines of 128 bytes each per array), into L1
                        // while the PCA chunks are computed
                        const int jp = (int)(cur_packed & 0xFFFF) * kTile + col0 + (lane & 7) * 8;
                        if (lane < 8) asm volatile("prefetch.global.L1 [%0];" ::"l"(p.rs2 + jp));
                        if ((lane >> 3) < p.multi.count)
                            asm volatile("prefetch.global.L1 [%0];" ::"l"(p.multi.cs + (size_t)(lane >> 3) *
                                                                                     (size_t)p.multi.n_pad + jp));
                    }
#pragma unroll
                    for (int c = 0; c < NC; ++c) g[c] = 0.0f;
                }
                // the chunk's Gram partial sums, added in order (round to
                // nearest; the packed adds round each lane like scalar adds)
                const uint32_t ta = tmem_base + lane_addr + (uint32_t)(slot * kTile + col0);
                {
                    uint32_t v[NC];
                    tmem_ld_cols(ta, v);
#pragma unroll
                    for (int c = 0; c < NC; c += 2) add2_f32(g[c], g[c + 1], v[c], v[c + 1]);
                }
                if constexpr (MULTI) {
                    if (ks >= p.kx_steps) {
                        const int yc = ks - p.kx_steps;
                        // the PCA part's Gram sums, kept beside the running ones
                        if (yc + 1 == p.multi.py_chunks) park(g, gy_run);
                        bool due = false;
                        for (int c = 0; c < p.multi.count; ++c) due |= yc == cand_sel(p.multi.end, c);
                        if (due) {
                            // the running sums go to this warp's columns of the
                            // drained slot (released only after the checks), so
                            // the checks run with their registers free
                            park(g, ta);
                            // one call site: the check is large, and its copies
                            // would crowd the instruction cache
#pragma unroll 1
                            for (int c = 0; c < p.multi.count; ++c)
                                if (yc == cand_sel(p.multi.end, c)) cand_check(c, ta, cur_packed, cur_ib, cur_ri);
                            uint32_t v[NC];
                            tmem_ld_cols(ta, v);
#pragma unroll
                            for (int c = 0; c < NC; ++c) g[c] = __uint_as_float(v[c]);
                        }
                    }
                }
                // the slot is drained: one arrival per warp (a pair: on the
                // leader's barrier)
                tc_fence_before();
                __syncwarp();
                if (PAIR) {
                    if (lane == 0) mbar_arrive_cluster(sempty_tgt + 8 * slot);
                } else {
                    if (lane == 0) mbar_arrive(bar_sempty + 8 * slot);
                }
                if (++slot == kSlots) {
                    slot = 0;
                    sphase ^= 1;
                }
                // the previous tile's pieces, spread evenly over the X chunks
                while (ks < p.kx_steps && pend && pend_pieces < NP &&
                       pend_pieces * p.kx_steps < (ks + 1) * NP)
                    classify_next();
            }
            if (!ok || stop) break;
            // ---- park the Y sums in the running columns; the tile is now pending
            park(g, gy_run);
            const int J = (int)(cur_packed & 0xFFFF);
            const int Ib = cur_ib;
            pend = true;
            pend_pieces = 0;
            pend_u = PAIR ? 2 * t + (long long)rank : t;
            pend_i = Ib * kTile + r;
            pend_ri = cur_ri;
            pend_j0 = J * kTile + col0;
            // the 64 column statistics the classification reads, one lane per
            // pair of rows: in L1 by the time the next tile's drains begin
            asm volatile("prefetch.global.L1 [%0];" ::"l"(p.rs + pend_j0 + (lane * NC) / 32));
            pend_vmask = ~0ull;
            pend_full = (Ib < J) && (J * kTile + kTile <= p.n);
            if (!pend_full) {
                // diagonal, below-diagonal or ragged tile: columns that are not
                // pairs i < j < n get a NaN Gram entry and their queue bit is cleared
                for (int c = 0; c < NC; ++c) {
                    const int j = pend_j0 + c;
                    if (!((pend_i < j) & (j < p.n))) pend_vmask &= ~(1ull << c);
                }
            }
            qmask = 0ull;
            acc = RowAcc{0.0f, 0.0f, -1.0f, 0, 0};
            t += tstep;
        }
        // the last tile (its sums are complete in TMEM)
        if (ok && pend) finish_pending();
        // every epilogue thread is done with the shared histogram counters
        mbar_arrive(bar_epi);
        mbar_wait(bar_epi, 0, p.status, 4);
        // ---- this warp's partial: its share of the histogram and its totals
        fold_hist<STD>(s_hist, ew, p.eps_bin, mine);
        if (lane == 0) {
            if (!STD) mine->violations = wt->violations;
            mine->queued = wt->queued;
            mine->degenerate = 0;
            mine->sum = wt->sum;
            mine->bound_sum = wt->bound_sum;
            mine->max = wt->max;
            mine->max_bound = wt->max_bound;
            mine->argmax_i = wt->argmax_i;
            mine->argmax_j = wt->argmax_j;
        }
        if constexpr (MULTI) {
            for (int c = 0; c < p.multi.count; ++c) {
                const int base = c * 4 * 32 * kEpiWarps + et;
                float rmh = -s_cr[base], rml = s_cr[base + 32 * kEpiWarps];
                float rnl = s_cr[base + 64 * kEpiWarps], rnh = s_cr[base + 96 * kEpiWarps];
                unsigned long long ce = s_cn[(c * 2 + 0) * 32 * kEpiWarps + et];
                unsigned long long op = s_cn[(c * 2 + 1) * 32 * kEpiWarps + et];
                for (int o = 16; o > 0; o >>= 1) {
                    rmh = fmaxf(rmh, __shfl_xor_sync(0xffffffffu, rmh, o));
                    rml = fmaxf(rml, __shfl_xor_sync(0xffffffffu, rml, o));
                    rnl = fminf(rnl, __shfl_xor_sync(0xffffffffu, rnl, o));
                    rnh = fminf(rnh, __shfl_xor_sync(0xffffffffu, rnh, o));
                    ce += __shfl_xor_sync(0xffffffffu, ce, o);
                    op += __shfl_xor_sync(0xffffffffu, op, o);
                }
                if (lane == 0) {
                    CandPartial &cp = p.multi.out[((size_t)blockIdx.x * kEpiWarps + ew) * p.multi.count + c];
                    cp.rmax_hi = rmh;
                    cp.rmax_lo = rml;
                    cp.rmin_lo = rnl;
                    cp.rmin_hi = rnh;
                    cp.certain = ce;
                    cp.open = op;
                }
            }
        }
            };
        if constexpr (kEpiWarps == 8) {
            epilogue(std::integral_constant<int, 64>{});
        } else {
            if (h == 0)
                epilogue(std::integral_constant<int, 48>{});
            else
                epilogue(std::integral_constant<int, 40>{});
        }
    }

    tc_fence_before();
    // a pair: both CTAs are done with each other's barriers and shared memory
    if (PAIR)
        cluster_sync();
    else
        __syncthreads();
    tc_fence_after();
    if (warp == 1) {
        if (PAIR)
            asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                         "r"(kTmemCols)
                         : "memory");
        else
            asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                         "r"(kTmemCols)
                         : "memory");
    }
    if (PAIR) cluster_sync();
}

// (|xc|^2, |yc|^2, sqrt(0.56) q4x, sqrt(0.56) q4y) per row: the q4 terms of
// the Gram bounds carry the kernel's bound coefficient (rounded up)
// and the same interleaved by column pair into out2 (see TcArgs::rs2)
__global__ void pack_row_stats(const RowStat *__restrict__ rx, const RowStat *__restrict__ ry,
                               int64_t n_pad, float4 *__restrict__ out, float *__restrict__ out2) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const float sc = 0.74833152f;  // sqrt(0.56) = 0.748331477..., rounded up
    if (r >= n_pad) return;
    const float4 v = make_float4(rx[r].n2, ry[r].n2, sc * rx[r].q4, sc * ry[r].q4);
    out[r] = v;
    float *e = out2 + (r & ~1ll) * 4 + (r & 1);  // element 2q starts at float 8q
    e[0] = v.x;
    e[2] = v.y;
    e[4] = v.z;
    e[6] = v.w;
}

// Row statistics of the JL-prefix candidates (TcMulti::cs): row r of Y,
// centred by the preparation's column means in FP32 like the split planes, in
// FP64 sums: the PCA part's squared norm and 4-norm coefficient, and per
// candidate the squared norm of its JL prefix and the 4-norm coefficient of
// the whole prefix (PCA part and JL prefix), q4 = sqrt(2 c4) ||.||_4 (rounded
// up).  Written interleaved by row pair; rows past n get zeros.
__global__ void cand_stats_kernel(const float *__restrict__ Y, int64_t n, int64_t n_pad, int64_t ldy,
                                  const float *__restrict__ mu, int s, int jo, int count, int4 kc4,
                                  double q4scale, float *__restrict__ cs) {
    const int lane = threadIdx.x & 31;
    const int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (r >= n_pad) return;
    const int kc[4] = {kc4.x, kc4.y, kc4.z, kc4.w};
    double p2 = 0.0, p4 = 0.0;
    if (r < n)
        for (int c = lane; c < s; c += 32) {
            const double v = __fsub_rn(Y[r * ldy + c], mu[c]);
            p2 = fma(v, v, p2);
            p4 = fma(v * v, v * v, p4);
        }
    for (int o = 16; o > 0; o >>= 1) {
        p2 += __shfl_xor_sync(0xffffffffu, p2, o);
        p4 += __shfl_xor_sync(0xffffffffu, p4, o);
    }
    for (int q = 0; q < count; ++q) {
        double j2 = 0.0, j4 = 0.0;
        if (r < n)
            for (int t = lane; t < kc[q]; t += 32) {
                const double v = __fsub_rn(Y[r * ldy + jo + t], mu[jo + t]);
                j2 = fma(v, v, j2);
                j4 = fma(v * v, v * v, j4);
            }
        for (int o = 16; o > 0; o >>= 1) {
            j2 += __shfl_xor_sync(0xffffffffu, j2, o);
            j4 += __shfl_xor_sync(0xffffffffu, j4, o);
        }
        if (lane == 0) {
            // element 2q' (two floats per field) holds rows 2q', 2q' + 1
            float *e = cs + (int64_t)q * n_pad * 4 + (r & ~1ll) * 4 + (r & 1);
            e[0] = (float)p2;
            e[2] = __double2float_ru(q4scale * sqrt(sqrt(p4)));
            e[4] = (float)j2;
            e[6] = __double2float_ru(q4scale * sqrt(sqrt(p4 + j4)));
        }
    }
}

// Band orders of the upper triangle.  Single: bands of `band` tile rows; in a
// band, J runs left to right and I over the band's rows with I <= J, so the
// band's I tiles stay in L2 while the J tiles stream.  Pair: tiles of 256 I
// rows x 128 J rows (I counts 256-row blocks), bands of band / 2 such blocks
// (the same rows), J >= 2 I (the tiles that hold pairs i < j).
std::vector<uint32_t> band_schedule(int T, int band) {
    std::vector<uint32_t> s;
    s.reserve((size_t)T * (T + 1) / 2);
    for (int b0 = 0; b0 < T; b0 += band) {
        const int b1 = std::min(T, b0 + band);
        for (int J = b0; J < T; ++J)
            for (int I = b0; I < b1 && I <= J; ++I) s.push_back(((uint32_t)I << 16) | (uint32_t)J);
    }
    return s;
}

std::vector<uint32_t> band_schedule_pair(int T, int band) {
    const int T2 = T / 2, band2 = std::max(1, band / 2);
    std::vector<uint32_t> s;
    s.reserve((size_t)T2 * (T2 + 1));
    for (int b0 = 0; b0 < T2; b0 += band2) {
        const int b1 = std::min(T2, b0 + band2);
        for (int J = 2 * b0; J < T; ++J)
            for (int I = b0; I < b1 && 2 * I <= J; ++I) s.push_back(((uint32_t)I << 16) | (uint32_t)J);
    }
    return s;
}

}  // namespace

// 128-row tile blocks of a prepared matrix of n rows
static int tile_blocks(int64_t n) { return (int)(pad_rows(n) / kTile); }

// raises the kernels' dynamic shared-memory limit (once per device)
void cert_tc_init() {
    set_max_dyn_smem((const void *)cert_tc_kernel<true, false, true>, (int)Layout<false>::smem);
    set_max_dyn_smem((const void *)cert_tc_kernel<false, false, true>, (int)Layout<false>::smem);
    set_max_dyn_smem((const void *)cert_tc_kernel<false, false, false>, (int)Layout<false>::smem);
    set_max_dyn_smem((const void *)cert_tc_kernel<true, true, true>, (int)Layout<true>::smem);
    set_max_dyn_smem((const void *)cert_tc_kernel<false, true, true>, (int)Layout<true>::smem);
    set_max_dyn_smem((const void *)cert_tc_kernel<false, true, false>, (int)Layout<true>::smem);
    set_max_dyn_smem((const void *)cert_tc_kernel<false, false, true, true>, (int)Layout<false, true>::smem);
}

static cudaLaunchConfig_t pair_config(unsigned ctas, cudaStream_t st, cudaLaunchAttribute *at) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(ctas);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = Layout<true>::smem;
    cfg.stream = st;
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cfg;
}

// CTA pairs of the pair variant that can be resident at once (0: none; the
// single variant is used), queried once per context
static int pair_capacity(adagio_ctx *ctx) {
    if (ctx->tc_pair_clusters >= 0) return ctx->tc_pair_clusters;
    cert_tc_init();
    cudaLaunchAttribute at[1];
    cudaLaunchConfig_t cfg = pair_config((unsigned)(ctx->num_sms / 2 * 2), nullptr, at);
    int nc = 0;
    if (cudaOccupancyMaxActiveClusters(&nc, (const void *)cert_tc_kernel<false, true, true>, &cfg) != cudaSuccess) {
        cudaGetLastError();
        nc = 0;
    }
    ctx->tc_pair_clusters = std::max(0, std::min(nc, ctx->num_sms / 2));
    return ctx->tc_pair_clusters;
}

int tc_size_class(int64_t n) {
    int c = 0;
    while ((1ll << c) < tile_blocks(n)) ++c;
    return c;
}

// The tile configuration that certifies n points: the context's explicit
// setting (adagio_set_tile_kernel), else what the autotuner found for n's
// size class, else one CTA per tile (measured faster on the MNIST-shaped
// workload: its epilogue, not the operand traffic the pair saves, limits the
// tile rate) with bands of 8 tile rows.  The pair needs rows padded to 256
// and resident CTA pairs.
TileConfig tc_config(adagio_ctx *ctx, int64_t n) {
    TileConfig c{1, 8};
    auto it = ctx->tc_tuned.find(tc_size_class(n));
    if (it != ctx->tc_tuned.end()) c = TileConfig{it->second.variant, it->second.band};
    if (ctx->tc_variant != 0) c.variant = ctx->tc_variant;
    if (ctx->tc_band != 0) c.band = ctx->tc_band;
    if (c.variant == 2 && (pad_rows(n) % (2 * kTile) != 0 || pair_capacity(ctx) == 0)) c.variant = 1;
    return c;
}

int tc_variant(adagio_ctx *ctx, int64_t n) { return tc_config(ctx, n).variant; }

bool tc_pair_supported(adagio_ctx *ctx) { return pair_capacity(ctx) > 0; }

// Per-context cache of the device copy of a schedule, by tile-block count,
// variant and band, resident for the context's lifetime (built on first use:
// a synchronous upload, so callers that capture graphs make it resident first
// with tc_prepare).
static const uint32_t *schedule_for(adagio_ctx *ctx, int T, TileConfig cfg, long long *count) {
    const int key = (T << 10) | (cfg.band << 2) | cfg.variant;
    const int variant = cfg.variant;
    auto it = ctx->tc_sched.find(key);
    if (it != ctx->tc_sched.end()) {
        *count = variant == 2 ? (long long)(T / 2) * (T / 2 + 1) : (long long)T * (T + 1) / 2;
        return it->second;
    }
    std::vector<uint32_t> s = variant == 2 ? band_schedule_pair(T, cfg.band) : band_schedule(T, cfg.band);
    uint32_t *dev = nullptr;
    ADAGIO_CUDA(cudaMalloc(&dev, s.size() * sizeof(uint32_t)));
    cudaError_t e = cudaMemcpy(dev, s.data(), s.size() * sizeof(uint32_t), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(dev);
        ADAGIO_CUDA(e);
    }
    ctx->tc_sched[key] = dev;
    *count = (long long)s.size();
    return dev;
}

void tc_prepare(adagio_ctx *ctx, int64_t n) {
    long long c;
    (void)schedule_for(ctx, tile_blocks(n), tc_config(ctx, n), &c);
}

int cert_tc_slots_per_cta() { return kEpiWarps; }

// CTAs of one certificate launch: one per SM (the shared-memory footprint
// allows one), never more than there are tiles, so that small problems of a
// batch leave SMs to the others
int cert_tc_ctas(adagio_ctx *ctx, int64_t n) {
    const long long T = tile_blocks(n);
    if (tc_variant(ctx, n) == 2) {
        const long long tiles = (T / 2) * (T / 2 + 1);
        return 2 * (int)std::min<long long>(pair_capacity(ctx), tiles);
    }
    const long long tiles = T * (T + 1) / 2;
    return (int)std::min<long long>(ctx->num_sms, tiles);
}

// 128-row block coordinates (I, J) of 128 x 128 tile unit u (the unit index
// of the per-pair dump): the u-th tile of the single schedule, or CTA u % 2
// of the (u / 2)-th tile of the pair schedule
void tc_tile_coords(adagio_ctx *ctx, int64_t n, long long u, int *I, int *J) {
    const int T = tile_blocks(n);
    const TileConfig cfg = tc_config(ctx, n);
    if (cfg.variant == 2) {
        const std::vector<uint32_t> s = band_schedule_pair(T, cfg.band);
        const uint32_t v = s.at((size_t)(u >> 1));
        *I = 2 * (int)(v >> 16) + (int)(u & 1);
        *J = (int)(v & 0xFFFF);
    } else {
        const std::vector<uint32_t> s = band_schedule(T, cfg.band);
        const uint32_t v = s.at((size_t)u);
        *I = (int)(v >> 16);
        *J = (int)(v & 0xFFFF);
    }
}

bool launch_cert_tc(const CertLaunch &L, int precision, cudaStream_t st) {
    const PrepMat &x = *L.x, &y = *L.y;
    if (!x.hi || !y.hi) return false;
    if (x.n_pad / kTile >= 65536) return false;
    TileConfig cfg = tc_config(L.ctx, x.n);
    // a shard, and the multi-candidate pass, run the single-CTA kernel
    const bool sharded = L.t_end >= 0;
    const bool multi = L.multi && L.multi->count > 0;
    if (sharded || multi) cfg.variant = 1;
    const bool pair = cfg.variant == 2;
    if (pair && (x.n_pad % (2 * kTile) != 0 || y.n_pad != x.n_pad))
        fail(ADAGIO_E_CUDA, "internal: pair tiles need rows padded to 256 (n_pad %lld)",
             (long long)x.n_pad);
    const bool bf16 = precision == ADAGIO_PREC_BF16X3;
    const int brows = pair ? Layout<true>::kBRows : Layout<false>::kBRows;
    const CUtensorMap mxh = plane_map(x.hi, x.n_pad, x.Kp16, kKStep, kTile, bf16);
    const CUtensorMap mxl = plane_map(x.lo, x.n_pad, x.Kp16, kKStep, kTile, bf16);
    const CUtensorMap myh = plane_map(y.hi, y.n_pad, y.Kp16, kKStep, kTile, bf16);
    const CUtensorMap myl = plane_map(y.lo, y.n_pad, y.Kp16, kKStep, kTile, bf16);
    const CUtensorMap bxh = plane_map(x.hi, x.n_pad, x.Kp16, kKStep, brows, bf16);
    const CUtensorMap bxl = plane_map(x.lo, x.n_pad, x.Kp16, kKStep, brows, bf16);
    const CUtensorMap byh = plane_map(y.hi, y.n_pad, y.Kp16, kKStep, brows, bf16);
    const CUtensorMap byl = plane_map(y.lo, y.n_pad, y.Kp16, kKStep, brows, bf16);
    TcArgs a;
    a.rs = reinterpret_cast<const float4 *>(L.rs_xy);
    a.rs2 = reinterpret_cast<const ulonglong2 *>(reinterpret_cast<const float4 *>(L.rs_xy) + x.n_pad);
    pack_row_stats<<<(unsigned)ceil_div(x.n_pad, 256), 256, 0, st>>>(
        x.rs, y.rs, x.n_pad, (float4 *)L.rs_xy, (float *)(reinterpret_cast<float4 *>(L.rs_xy) + x.n_pad));
    ADAGIO_CHECK_LAUNCH();
    // ex = q4_i q4_j + (c_acc + c_r)(n2_i + n2_j) dominates the split model's
    // q1 term, because 2 |a| |b| <= |a|^2 + |b|^2; the kernel takes it times
    // the bound coefficient 0.56 (q4 scaled by sqrt(0.56) in the row stats)
    a.cx = kBoundCoef * (x.bm.cacc + L.cc.c_r);
    a.cy = kBoundCoef * (y.bm.cacc + L.cc.c_r);
    a.scale_x = x.scale;
    a.scale_y = y.scale;
    const int T = (int)(x.n_pad / kTile);
    if (sharded) {
        // the band order restricted to tiles [t_begin, t_end) of the
        // row-major triangle; uploaded into the call's workspace
        std::vector<uint32_t> s;
        for (uint32_t e : band_schedule(T, cfg.band)) {
            const long long I = e >> 16, J = e & 0xFFFF;
            const long long t = I * T - I * (I - 1) / 2 + (J - I);
            if (t >= L.t_begin && t < L.t_end) s.push_back(e);
        }
        uint32_t *dev = ws_array<uint32_t>(L.ctx, std::max<size_t>(s.size(), 1));
        ADAGIO_CUDA(cudaMemcpy(dev, s.data(), s.size() * sizeof(uint32_t), cudaMemcpyHostToDevice));
        a.sched = dev;
        a.ntp = (long long)s.size();
    } else {
        a.sched = schedule_for(L.ctx, T, cfg, &a.ntp);
    }
    a.n = (int)x.n;
    a.kx_steps = x.Kp16 / kKStep;
    a.ky_steps = y.Kp16 / kKStep;
    // instruction descriptor, kind::f16: D = F32 (bits 4-5 = 1), A/B format
    // F16 = 0 / BF16 = 1 (bits 7-9, 10-12), K-major A and B, N >> 3 at bit
    // 17, M >> 4 at bit 24 (M = 256 for the pair: 128 rows per CTA)
    const uint32_t fmt = bf16 ? 1u : 0u;
    const uint32_t M = pair ? 2 * kTile : kTile;
    a.idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(kTile >> 3) << 17) | ((M >> 4) << 24);
    a.cc = L.cc;
    a.partials = L.partials;
    a.queue = L.queue;
    a.qcount = L.qcount;
    a.qcap = L.qcap;
    a.stop_flag = L.stop_flag;
    a.status = L.status;
    a.dump = reinterpret_cast<float4 *>(L.dump);
    a.dump_tiles = L.dump_tiles;
    a.dump_stride = std::max(1ll, L.dump_stride);
    // the standard range: lo = 0 and eps on a bin edge (the default [0, 2 eps)
    // puts it on edge 32); then the violations are read off the histogram
    const double span = (double)L.cc.hi - (double)L.cc.lo;
    const double te = ((double)L.cc.eps - (double)L.cc.lo) / span * kBins;
    const long eb = std::lround(te);
    const bool std_range = L.cc.lo == 0.0f && eb >= 1 && eb <= kBins && std::fabs(te - (double)eb) <= 1e-6;
    a.eps_bin = std_range ? (int)eb : kBins;
    if (L.dump && !std_range) fail(ADAGIO_E_CUDA, "internal: the per-pair dump needs the standard range");
    a.multi = TcMulti{};
    if (multi) {
        const MultiSpec &ms = *L.multi;
        if (!std_range || L.dump || sharded || !L.ysrc)
            fail(ADAGIO_E_CUDA, "internal: the multi-candidate pass needs the standard range, whole");
        TcMulti &mt = a.multi;
        mt.count = ms.count;
        mt.py_chunks = ms.s_pad / kKStep;
        // raw coefficients, rounded up: the same error model as the pair
        // bound of the full certificate, without its 0.56 linearisation factor
        const double cr = L.cc.c_r;
        auto up = [](double v) { return std::nextafter((float)v, INFINITY); };
        mt.cxr = up((double)x.bm.cacc + cr);
        mt.cypr = up((double)bound_model(precision, ms.s_pad).cacc + cr);
        for (int c = 0; c < kMaxCand; ++c) {
            mt.end[c] = 0;
            mt.lam[c] = 1.0f;
            mt.cycr[c] = 0.0f;
        }
        for (int c = 0; c < ms.count; ++c) {
            mt.end[c] = (ms.jo + ms.kc[c] - 1) / kKStep;
            mt.lam[c] = (float)ms.k / (float)ms.kc[c];
            mt.cycr[c] = up((double)bound_model(precision, (mt.end[c] + 1) * kKStep).cacc + cr);
        }
        mt.u2r = up(5.9604645e-08);
        mt.kraw = up(1.0 / (double)kBoundCoef);
        // thresholds on r from the caller's eps in FP64, with 32 units of
        // slack for the roundings of the bounds and of these products
        const double e1 = (1.0 + ms.eps) * (1.0 + ms.eps), e0 = (1.0 - ms.eps) * (1.0 - ms.eps);
        const double sl = 32.0 * 5.9604645e-08;
        mt.uv = up(e1 * (1.0 + sl));
        mt.lv = std::nextafter((float)(e0 * (1.0 - sl)), 0.0f);
        mt.uf = std::nextafter((float)(e1 * (1.0 - sl)), 0.0f);
        mt.lf = up(e0 * (1.0 + sl));
        mt.cs = reinterpret_cast<const ulonglong2 *>(ms.cs);
        mt.cq = reinterpret_cast<int4 *>(ms.cq);
        mt.cqcount = ms.cqcount;
        mt.cqcap = ms.cqcap;
        // a certificate whose recompute queue overflowed runs the tiles again:
        // each launch starts the candidates' queue afresh (their records are
        // written, not added)
        ADAGIO_CUDA(cudaMemsetAsync(ms.cqcount, 0, sizeof(unsigned long long), st));
        mt.out = reinterpret_cast<CandPartial *>(ms.out);
        mt.n_pad = y.n_pad;
        const int4 kc4 = make_int4(ms.kc[0], ms.kc[1], ms.kc[2], ms.kc[3]);
        const double q4scale = std::sqrt(2.0 * (double)y.bm.c4) * (1.0 + 1e-6);
        cand_stats_kernel<<<(unsigned)ceil_div(y.n_pad, 8), 256, 0, st>>>(
            L.ysrc, y.n, y.n_pad, L.ldy_src, y.mu, ms.s, ms.jo, ms.count, kc4, q4scale,
            reinterpret_cast<float *>(ms.cs));
        ADAGIO_CHECK_LAUNCH();
    }
    ADAGIO_CUDA(cudaMemsetAsync(L.partials, 0, sizeof(CertPartial) * L.grid, st));
    cert_tc_init();
    const unsigned ctas = (unsigned)(L.grid / kEpiWarps);
    if (pair) {
        cudaLaunchAttribute at[1];
        const cudaLaunchConfig_t cfg = pair_config(ctas, st, at);
        if (L.dump)
            ADAGIO_CUDA(cudaLaunchKernelEx(&cfg, cert_tc_kernel<true, true, true>, mxh, mxl, myh, myl, bxh,
                                           bxl, byh, byl, a));
        else if (std_range)
            ADAGIO_CUDA(cudaLaunchKernelEx(&cfg, cert_tc_kernel<false, true, true>, mxh, mxl, myh, myl, bxh,
                                           bxl, byh, byl, a));
        else
            ADAGIO_CUDA(cudaLaunchKernelEx(&cfg, cert_tc_kernel<false, true, false>, mxh, mxl, myh, myl, bxh,
                                           bxl, byh, byl, a));
    } else {
        const size_t sm = Layout<false>::smem;
        if (multi)
            cert_tc_kernel<false, false, true, true><<<ctas, kThreads, Layout<false, true>::smem, st>>>(
                mxh, mxl, myh, myl, bxh, bxl, byh, byl, a);
        else if (L.dump)
            cert_tc_kernel<true, false, true><<<ctas, kThreads, sm, st>>>(mxh, mxl, myh, myl, bxh, bxl, byh,
                                                                          byl, a);
        else if (std_range)
            cert_tc_kernel<false, false, true><<<ctas, kThreads, sm, st>>>(mxh, mxl, myh, myl, bxh, bxl, byh,
                                                                           byl, a);
        else
            cert_tc_kernel<false, false, false><<<ctas, kThreads, sm, st>>>(mxh, mxl, myh, myl, bxh, bxl,
                                                                            byh, byl, a);
    }
    ADAGIO_CHECK_LAUNCH();
    return true;
}

}  // namespace adagio
