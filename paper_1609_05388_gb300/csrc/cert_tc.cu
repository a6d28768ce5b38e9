// K8 (tensor-core path): all-pairs distortion tiles on tcgen05.
//
// One persistent CTA per SM walks 128 x 128 tiles (I, J), I <= J, of the
// pair matrix in the band order of the schedule table (bands of 8 tile rows,
// so the I-tiles of a band stay in L2 while the J-tiles stream).  For every
// tile it forms
//     Gy = Yc[I] Yc[J]^T   and   Gx = Xc[I] Xc[J]^T
// from 2-term split planes (hi + lo, FP16 or BF16, power-of-two scaled) with
// three products hi.hi + hi.lo + lo.hi per K chunk, accumulated in FP32 in
// tensor memory chunk by chunk, and hands the sums to the epilogue (cert_common.cuh),
// which classifies every pair (Eq. 2), accumulates max / histogram / counts
// and queues the pairs that need the exact recompute.
//
// Roles (320 threads):
//   warp 0      TMA producer: 4 planes (A hi/lo, B hi/lo) of 64 K-elements per
//               stage, 3 stages of 64 KB, 128-byte swizzle
//   warp 1      TMEM owner (512 columns = 4 chunk slots of 128) and MMA issuer:
//               tcgen05.mma kind::f16, M = N = 128, K = 16.  Every 64-element K
//               step goes to a fresh slot, cross products (hi.lo, lo.hi) first
//               and the 4 hi.hi products last: the FP32 accumulator loses up to
//               one unit in the last place per MMA (it truncates), so this
//               bounds the full-size roundings to 4 per chunk
//   warps 2..9  epilogue: two warps per TMEM lane quarter, 64 columns each;
//               they drain every slot into register running sums (round to
//               nearest) and classify their 64 pairs at the end of a tile,
//               without data-dependent branches
// The producer decides the tile sequence and sends it down the pipeline (a
// tile index per first stage, -1 to stop, forwarded through a slot), so early
// exit needs no CTA-wide barrier, and the epilogue warps never wait on one
// another.  Every wait is bounded: on timeout the role records a status word
// and leaves, the producer drains its in-flight copies, the MMA warp waits
// for its last commit, and TMEM is freed.
#include <cuda.h>

#include "internal.cuh"
#include "cert.cuh"

#include <mutex>
#include <vector>

namespace adagio {

namespace {

constexpr int kEpiWarps = 8;                                // two per TMEM lane quarter
constexpr int kThreads = 64 + 32 * kEpiWarps;               // producer, MMA, epilogue
constexpr int kStages = 3;
constexpr int kSlots = 2;                                   // TMEM chunk accumulators
constexpr int kTile = 128;
constexpr int kKStep = 64;                                  // fp16 elements per stage row
constexpr int kEpiCols = 64;                                // columns per epilogue warp
constexpr uint32_t kPlaneBytes = kTile * kKStep * 2;        // 16 KB
constexpr uint32_t kStageBytes = 4 * kPlaneBytes;           // 64 KB
constexpr uint32_t kStageCol = kSlots * kTile;              // finished Gram sums (gx | gy)
constexpr uint32_t kTmemCols = kStageCol + 2 * kTile;       // 512
static_assert(kTmemCols == 512, "TMEM holds 512 columns");
constexpr int kPiece = 8;                                   // columns classified per step
constexpr int kPieces = kEpiCols / kPiece;
constexpr int kHistFlushTiles = 1000;                       // u16 counters: <= 64 per tile
// per-thread histogram: two 16-bit bin counters per 32-bit word
constexpr int kHistWords = kBins / 2;
constexpr long long kSpinLimit = 4000000000ll;              // clock64 cycles (~2 s)

struct TcArgs {
    const float4 *rs;          // per row: (|xc|^2, |yc|^2, q4x, q4y)
    float cx, cy;              // bound coefficients of (n2_i + n2_j) per side
    const float *scale_x, *scale_y;
    const uint32_t *sched;     // (I << 16) | J per tile pair
    long long ntp;
    int n, kx_steps, ky_steps;
    uint32_t idesc;
    CertConst cc;
    CertPartial *partials;     // [gridDim.x * kEpiWarps], one slot per epilogue warp
    int2 *queue;
    unsigned long long *qcount, qcap;
    int *stop_flag;
    int *status;
    float4 *dump;              // optional: (dx2, dy2, ex, ey) of tile pairs t < dump_tiles
    long long dump_tiles;
};

struct SmemLayout {
    static constexpr uint32_t stages = 0;
    static constexpr uint32_t hist = kStages * kStageBytes;                  // u32 [32][256]
    static constexpr uint32_t bars = hist + kHistWords * 32 * kEpiWarps * 4;
    static constexpr uint32_t cmd = bars + 256;                               // int [16]
    static constexpr uint32_t tmem_ptr = cmd + 64;
    static constexpr uint32_t totals = tmem_ptr + 16;                         // WarpTotals [8]
    static constexpr uint32_t total = totals + 64 * kEpiWarps;
};
constexpr size_t kSmemBytes = SmemLayout::total + 1024;   // + alignment slack
static_assert(kSmemBytes <= 232448, "tile kernel exceeds the 227 KB shared-memory limit");
static_assert(SmemLayout::totals % 8 == 0, "per-warp totals need 8-byte alignment");

// ------------------------------------------------------------------ PTX glue
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred P1;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2;\n\t"
        "selp.b32 %0, 1, 0, P1;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for the completion of the phase with the given parity.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int *status, int code) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (true) {
        if (mbar_try_wait(bar, parity)) return true;
        if (clock64() - t0 > kSpinLimit) {
            atomicCAS(status, 0, code);
            return false;
        }
    }
}

// Warp-uniform bounded wait: lane 0 waits, every lane gets the outcome.
__device__ __forceinline__ bool warp_wait(uint32_t bar, uint32_t parity, int *status, int code) {
    int ok = 0;
    if ((threadIdx.x & 31) == 0) ok = mbar_wait(bar, parity, status, code) ? 1 : 0;
    return __shfl_sync(0xffffffffu, ok, 0) != 0;
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y,
                                            uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// SW128 K-major shared-memory matrix descriptor (tcgen05 format): start
// address >> 4, leading byte offset 16 (unused for swizzled K-major), stride
// byte offset 1024 (one 8-row x 128-byte swizzle atom), version 1, 128B swizzle.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)(16 >> 4) << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

__device__ __forceinline__ void tc_mma(uint32_t dtmem, uint64_t adesc, uint64_t bdesc,
                                       uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void tc_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

// 16 consecutive TMEM columns of this warp's lane quarter into registers.
// The wait is part of the same statement, so no use of the registers can be
// scheduled before the asynchronous load has completed.
__device__ __forceinline__ void tmem_ld16_wait(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
}

// 64 consecutive TMEM columns (four x16 loads) with one wait.
__device__ __forceinline__ void tmem_ld64_wait(uint32_t taddr, uint32_t (&r)[64]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%64];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%65];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%32, %33, %34, %35, %36, %37, %38, %39, %40, %41, %42, %43, %44, %45, %46, %47}, [%66];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%48, %49, %50, %51, %52, %53, %54, %55, %56, %57, %58, %59, %60, %61, %62, %63}, [%67];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]), "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]), "=r"(r[40]), "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]), "=r"(r[48]), "=r"(r[49]), "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]), "=r"(r[55]), "=r"(r[56]), "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]), "=r"(r[61]), "=r"(r[62]), "=r"(r[63])
        : "r"(taddr), "r"(taddr + 16), "r"(taddr + 32), "r"(taddr + 48)
        : "memory");
}

// Two 32-column pieces (at ta and tb; two x16 loads each) with one wait.
__device__ __forceinline__ void tmem_ld32x2_wait(uint32_t ta, uint32_t tb, uint32_t (&a)[32],
                                                 uint32_t (&b)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%64];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%65];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%32, %33, %34, %35, %36, %37, %38, %39, %40, %41, %42, %43, %44, %45, %46, %47}, [%66];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%48, %49, %50, %51, %52, %53, %54, %55, %56, %57, %58, %59, %60, %61, %62, %63}, [%67];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(a[0]), "=r"(a[1]), "=r"(a[2]), "=r"(a[3]), "=r"(a[4]), "=r"(a[5]), "=r"(a[6]), "=r"(a[7]), "=r"(a[8]), "=r"(a[9]), "=r"(a[10]), "=r"(a[11]), "=r"(a[12]), "=r"(a[13]), "=r"(a[14]), "=r"(a[15]), "=r"(a[16]), "=r"(a[17]), "=r"(a[18]), "=r"(a[19]), "=r"(a[20]), "=r"(a[21]), "=r"(a[22]), "=r"(a[23]), "=r"(a[24]), "=r"(a[25]), "=r"(a[26]), "=r"(a[27]), "=r"(a[28]), "=r"(a[29]), "=r"(a[30]), "=r"(a[31]), "=r"(b[0]), "=r"(b[1]), "=r"(b[2]), "=r"(b[3]), "=r"(b[4]), "=r"(b[5]), "=r"(b[6]), "=r"(b[7]), "=r"(b[8]), "=r"(b[9]), "=r"(b[10]), "=r"(b[11]), "=r"(b[12]), "=r"(b[13]), "=r"(b[14]), "=r"(b[15]), "=r"(b[16]), "=r"(b[17]), "=r"(b[18]), "=r"(b[19]), "=r"(b[20]), "=r"(b[21]), "=r"(b[22]), "=r"(b[23]), "=r"(b[24]), "=r"(b[25]), "=r"(b[26]), "=r"(b[27]), "=r"(b[28]), "=r"(b[29]), "=r"(b[30]), "=r"(b[31])
        : "r"(ta), "r"(ta + 16), "r"(tb), "r"(tb + 16)
        : "memory");
}

// Two 16-column pieces (at ta and tb) with one wait.
__device__ __forceinline__ void tmem_ld16x2_wait(uint32_t ta, uint32_t tb, uint32_t (&a)[16],
                                                 uint32_t (&b)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%32];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%33];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(a[0]), "=r"(a[1]), "=r"(a[2]), "=r"(a[3]), "=r"(a[4]), "=r"(a[5]), "=r"(a[6]), "=r"(a[7]), "=r"(a[8]), "=r"(a[9]), "=r"(a[10]), "=r"(a[11]), "=r"(a[12]), "=r"(a[13]), "=r"(a[14]), "=r"(a[15]), "=r"(b[0]), "=r"(b[1]), "=r"(b[2]), "=r"(b[3]), "=r"(b[4]), "=r"(b[5]), "=r"(b[6]), "=r"(b[7]), "=r"(b[8]), "=r"(b[9]), "=r"(b[10]), "=r"(b[11]), "=r"(b[12]), "=r"(b[13]), "=r"(b[14]), "=r"(b[15])
        : "r"(ta), "r"(tb)
        : "memory");
}

// Two 8-column pieces (at ta and tb) with one wait.
__device__ __forceinline__ void tmem_ld8x2_wait(uint32_t ta, uint32_t tb, uint32_t (&a)[8],
                                                uint32_t (&b)[8]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7}, [%16];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 "
        "{%8, %9, %10, %11, %12, %13, %14, %15}, [%17];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(a[0]), "=r"(a[1]), "=r"(a[2]), "=r"(a[3]), "=r"(a[4]), "=r"(a[5]), "=r"(a[6]), "=r"(a[7]), "=r"(b[0]), "=r"(b[1]), "=r"(b[2]), "=r"(b[3]), "=r"(b[4]), "=r"(b[5]), "=r"(b[6]), "=r"(b[7])
        : "r"(ta), "r"(tb)
        : "memory");
}

// 16 registers into 16 consecutive TMEM columns of this warp's lane quarter.
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&v)[16]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
        "{%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16};"
        :
        : "r"(taddr), "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15])
        : "memory");
}

__device__ __forceinline__ void tmem_wait_st() {
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// Folds this warp's 32 per-thread counters of every bin into its partial
// (the bins and their total, part of `pairs`).
__device__ __forceinline__ void fold_hist(uint32_t *s_hist, int ew, CertPartial *dst) {
    const int lane = threadIdx.x & 31;
    unsigned long long pairs = 0;
    for (int w = 0; w < kHistWords; ++w) {
        uint32_t *c = s_hist + w * (32 * kEpiWarps) + ew * 32 + lane;
        const uint32_t v = *c;
        *c = 0;
        unsigned a = v & 0xFFFFu, b = v >> 16;
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, o);
            b += __shfl_xor_sync(0xffffffffu, b, o);
        }
        if (lane == 0) {
            dst->hist[2 * w] += a;
            dst->hist[2 * w + 1] += b;
            pairs += a + b;
        }
    }
    if (lane == 0) dst->pairs += pairs;
    __syncwarp();
}

struct EpiConst {
    float m2sx, m2sy;      // -2 / scale^2 of the split planes
    float cx, cy;          // bound coefficients of (n2_i + n2_j) per side
    float inv_w, t0, w;    // t = delta * inv_w + t0 = (delta - lo) / w
    float eps;
};

// Statistics one epilogue thread keeps over the pairs of one tile row.
struct RowAcc {
    float sum, bsum, mxb, mx;
    int viol, over, certain, arg;
};

// Per-warp running totals of the epilogue, in shared memory (lane 0 owns them).
struct WarpTotals {
    unsigned long long violations, overflow, queued;
    double sum, bound_sum;
    float max, max_bound;
    int argmax_i, argmax_j;
};

static_assert(sizeof(WarpTotals) <= 64, "per-warp totals exceed their shared-memory slot");

// Classifies the kPiece pairs (i, j0 + c0 + c) of one tile row from their Gram
// entries (Eq. 2), without data-dependent branches, so the compiler
// interleaves the independent pairs.  With p = dx2 dy2 and r = 1/sqrt(p):
//   delta = |sqrt(dy2 / dx2) - 1| = |dy2 - dx2| / (dx2 + p r)   (no cancellation)
// The Gram error bounds are ex = q4x_i q4x_j + cx (n2x_i + n2x_j), likewise ey,
// and the distortion error is at most
//   B = 0.55 rho (ex / dx2 + ey / dy2) + 1e-6 delta + 1e-9,  rho = dy2 r,
// written as 0.55 dy2 r^3 (ex dy2 + ey dx2) + ...; the last two terms cover
// the approximate reciprocal square root and reciprocal.  The fast value is
// used when the Gram values are well enough conditioned to bound
// (dx2 > 8 ex and dy2 > 8 ey) and
//   B <= min(1e-5, max(1e-6, distance of delta to the nearest bin edge or eps)),
// i.e. B is within the maximum's tolerance, and either B <= 1e-6 or no edge
// and not eps lies within B of delta; every other pair is flagged in qmask for
// the exact recompute.  A NaN Gram entry (how the caller marks a column that
// is not a real pair) fails the test: the pair is flagged and adds nothing to
// the statistics, and the caller clears its qmask bit.
template <bool DUMP>
__device__ __forceinline__ void classify_piece(const float (&gx)[kPiece], const float (&gy)[kPiece],
                                               const float4 ri, const float4 *__restrict__ rsj,
                                               int c0, const EpiConst &k, uint32_t *hrow, RowAcc &a,
                                               unsigned long long &qmask, float4 *dump_row) {
#pragma unroll
    for (int c = 0; c < kPiece; ++c) {
        const float4 rj = __ldg(rsj + c);
        const float sx = ri.x + rj.x, sy = ri.y + rj.y;
        const float dx2 = fmaf(k.m2sx, gx[c], sx), dy2 = fmaf(k.m2sy, gy[c], sy);
        const float ex = fmaf(ri.z, rj.z, k.cx * sx), ey = fmaf(ri.w, rj.w, k.cy * sy);
        if (DUMP) dump_row[c] = make_float4(dx2, dy2, ex, ey);
        const float pp = dx2 * dy2;
        const float r = rsqrtf(pp);
        const float delta = __fdividef(fabsf(dy2 - dx2), fmaf(pp, r, dx2));
        const float B = fmaf((0.55f * dy2) * (r * r * r), fmaf(ex, dy2, ey * dx2),
                             fmaf(1e-6f, delta, 1e-9f));
        const float t = fmaf(delta, k.inv_w, k.t0);
        // distance to the nearest real edge: edges lie at integer t in [0, 64]
        const float tc = fminf(fmaxf(t, -0.5f), (float)kBins + 0.5f);
        const float dedge = fabsf(tc - rintf(tc)) * k.w;
        const float lim = fminf(kMaxTol, fmaxf(kExempt, fminf(dedge, fabsf(delta - k.eps))));
        const float cond = fminf(fmaf(-8.0f, ex, dx2), fmaf(-8.0f, ey, dy2));
        const bool ok = (cond > 0.0f) & (B <= lim);
        qmask |= ok ? 0ull : (1ull << (c0 + c));
        const bool in_range = (t >= 0.0f) & (t < (float)kBins);
        const bool binned = ok & in_range;
        const int bin = (int)t;
        // pairs not counted in a bin add 0 (to bin 0's word)
        atomicAdd(hrow + (binned ? (bin >> 1) : 0) * (32 * kEpiWarps),
                  binned ? (1u << ((bin & 1) << 4)) : 0u);
        const bool viol = ok & (delta > k.eps);
        a.over += (ok & !in_range) ? 1 : 0;
        a.viol += viol ? 1 : 0;
        a.certain += (viol & (delta - B > k.eps)) ? 1 : 0;
        const float bok = ok ? B : 0.0f;
        a.sum += ok ? delta : 0.0f;
        a.bsum += bok;
        a.mxb = fmaxf(a.mxb, bok);
        const bool better = ok & (delta > a.mx);
        a.mx = better ? delta : a.mx;
        a.arg = better ? c0 + c : a.arg;
    }
}

// ---------------------------------------------------------------- the kernel
template <bool DUMP>
__global__ void __launch_bounds__(kThreads, 1)
    cert_tc_kernel(const __grid_constant__ CUtensorMap map_xh, const __grid_constant__ CUtensorMap map_xl,
                   const __grid_constant__ CUtensorMap map_yh, const __grid_constant__ CUtensorMap map_yl,
                   TcArgs p) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    // 1024-byte alignment of the stage buffers (128-byte swizzle atoms), by
    // an offset from the shared array so the address space stays known
    uint8_t *smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    const uint32_t sbase = smem_u32(smem);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    uint32_t *s_hist = reinterpret_cast<uint32_t *>(smem + SmemLayout::hist);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + SmemLayout::bars);
    int *s_cmd = reinterpret_cast<int *>(smem + SmemLayout::cmd);  // [kStages] stage, [kStages + s] slot
    uint32_t *s_tmem = reinterpret_cast<uint32_t *>(smem + SmemLayout::tmem_ptr);
    const uint32_t bar_full = smem_u32(bars);                 // [kStages]
    const uint32_t bar_empty = bar_full + 8 * kStages;        // [kStages]
    const uint32_t bar_sfull = bar_empty + 8 * kStages;       // [kSlots]
    const uint32_t bar_sempty = bar_sfull + 8 * kSlots;       // [kSlots]
    const uint32_t bar_done = bar_sempty + 8 * kSlots;        // MMA drain

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(bar_full + 8 * s, 1);
            mbar_init(bar_empty + 8 * s, 1);
        }
        for (int s = 0; s < kSlots; ++s) {
            mbar_init(bar_sfull + 8 * s, 1);
            mbar_init(bar_sempty + 8 * s, 32 * kEpiWarps);
        }
        mbar_init(bar_done, 1);
        for (int q = 0; q < 16; ++q) s_cmd[q] = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    for (int e = threadIdx.x; e < kHistWords * 32 * kEpiWarps; e += kThreads) s_hist[e] = 0;
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(s_tmem)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *s_tmem;
    const int ksteps = p.ky_steps + p.kx_steps;

    if (warp == 0) {
        // ------------------------------------------------------ TMA producer
        int stage = 0;
        uint32_t phase = 0;
        bool ok = true;
        uint32_t issued_parity[kStages];
        bool issued[kStages];
        for (int s = 0; s < kStages; ++s) issued[s] = false, issued_parity[s] = 0;
        long long t = blockIdx.x;
        while (ok) {
            bool stop = t >= p.ntp;
            if (!stop && p.stop_flag) {
                int f = 0;
                if (lane == 0) f = *(volatile int *)p.stop_flag;
                stop = __shfl_sync(0xffffffffu, f, 0) != 0;
            }
            if (stop) {
                if (lane == 0 && mbar_wait(bar_empty + 8 * stage, phase ^ 1, p.status, 1)) {
                    s_cmd[stage] = -1;
                    mbar_arrive(bar_full + 8 * stage);
                }
                // the empty wait proved the stage's last copy was consumed, and
                // the stop arrive moved its full barrier one phase on: nothing
                // of this stage is left to drain
                issued[stage] = false;
                __syncwarp();
                break;
            }
            const uint32_t packed = p.sched[t];
            const int I = (int)(packed >> 16), J = (int)(packed & 0xFFFF);
            for (int ks = 0; ks < ksteps; ++ks) {
                ok = warp_wait(bar_empty + 8 * stage, phase ^ 1, p.status, 1);
                if (!ok) break;
                if (lane == 0) {
                    if (ks == 0) s_cmd[stage] = (int)t;
                    const uint32_t bar = bar_full + 8 * stage;
                    mbar_arrive_expect_tx(bar, kStageBytes);
                    const uint32_t dst = sbase + SmemLayout::stages + stage * kStageBytes;
                    const bool is_y = ks >= p.kx_steps;
                    const int k0 = (is_y ? ks - p.kx_steps : ks) * kKStep;
                    const CUtensorMap *mh = is_y ? &map_yh : &map_xh;
                    const CUtensorMap *ml = is_y ? &map_yl : &map_xl;
                    tma_load_2d(dst, mh, k0, I * kTile, bar);
                    tma_load_2d(dst + kPlaneBytes, ml, k0, I * kTile, bar);
                    tma_load_2d(dst + 2 * kPlaneBytes, mh, k0, J * kTile, bar);
                    tma_load_2d(dst + 3 * kPlaneBytes, ml, k0, J * kTile, bar);
                }
                __syncwarp();
                issued[stage] = true;
                issued_parity[stage] = phase;
                if (++stage == kStages) {
                    stage = 0;
                    phase ^= 1;
                }
            }
            t += gridDim.x;
        }
        // drain: every issued copy must have landed before the CTA can exit
        if (lane == 0)
            for (int s = 0; s < kStages; ++s)
                if (issued[s]) mbar_wait(bar_full + 8 * s, issued_parity[s], p.status, 1);
        __syncwarp();
    } else if (warp == 1) {
        // ------------------------------------------------------- MMA issuer
        // Every K step accumulates into a fresh TMEM slot (128 columns): first
        // the 8 small cross-term products (hi.lo, lo.hi), then the 4 large
        // hi.hi products, so only 4 FP32 accumulator roundings per chunk act
        // on full-size partial sums.  The epilogue drains the slot.
        int stage = 0, slot = 0;
        uint32_t phase = 0, sphase = 0;
        bool any = false;
        bool ok = true;
        while (ok) {
            int t = -1;
            ok = warp_wait(bar_full + 8 * stage, phase, p.status, 2);
            if (!ok) break;
            if (lane == 0) t = s_cmd[stage];
            t = __shfl_sync(0xffffffffu, t, 0);
            if (t < 0) {
                // forward the stop to the epilogue through the next slot; the
                // plain arrive releases the store of the stop word
                if (lane == 0 && mbar_wait(bar_sempty + 8 * slot, sphase ^ 1, p.status, 2)) {
                    s_cmd[kStages + slot] = -1;
                    mbar_arrive(bar_sfull + 8 * slot);
                }
                __syncwarp();
                break;
            }
            for (int ks = 0; ks < ksteps; ++ks) {
                if (ks > 0) {
                    ok = warp_wait(bar_full + 8 * stage, phase, p.status, 2);
                    if (!ok) break;
                }
                ok = warp_wait(bar_sempty + 8 * slot, sphase ^ 1, p.status, 2);
                if (!ok) break;
                tc_fence_after();
                if (lane == 0) {
                    const uint32_t d = tmem_base + (uint32_t)(slot * kTile);
                    const uint32_t a0 = sbase + SmemLayout::stages + stage * kStageBytes;
                    const uint64_t ah = sw128_desc(a0), al = sw128_desc(a0 + kPlaneBytes);
                    const uint64_t bh = sw128_desc(a0 + 2 * kPlaneBytes);
                    const uint64_t bl = sw128_desc(a0 + 3 * kPlaneBytes);
#pragma unroll
                    for (int kk = 0; kk < kKStep / 16; ++kk) {
                        const uint64_t off = (uint64_t)(kk * 32) >> 4;  // 16 elements = 32 bytes
                        tc_mma(d, ah + off, bl + off, p.idesc, kk == 0 ? 0u : 1u);
                        tc_mma(d, al + off, bh + off, p.idesc, 1u);
                    }
#pragma unroll
                    for (int kk = 0; kk < kKStep / 16; ++kk) {
                        const uint64_t off = (uint64_t)(kk * 32) >> 4;
                        tc_mma(d, ah + off, bh + off, p.idesc, 1u);
                    }
                    tc_commit(bar_empty + 8 * stage);
                    tc_commit(bar_sfull + 8 * slot);
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
            tc_commit(bar_done);
            mbar_wait(bar_done, 0, p.status, 2);
        }
        __syncwarp();
    } else {
        // --------------------------------------------------------- epilogue
        // Warp e owns TMEM lane quarter (warp % 4), i.e. tile row r, and the
        // column half h of the tile.  The K chunks of a tile come X first, then
        // Y.  The X chunks are summed in registers (gx); the Y chunks are summed
        // in this warp's TMEM running columns (gy, read + add + write back).  At
        // the end of a tile gx is parked in the TMEM staging columns.  The
        // classification of a tile is software-pipelined into the next one: it
        // runs piece by piece between the next tile's X-chunk drains, while the
        // MMA warp computes that tile, and is finished before the next tile's Y
        // chunks overwrite the running columns.
        const int ew = warp - 2;                 // 0..7
        const int quarter = warp & 3;
        const int h = ew >> 2;                   // column half
        const int r = quarter * 32 + lane;       // tile row of this thread
        const uint32_t lane_addr = (uint32_t)(quarter * 32) << 16;
        const uint32_t gx_stage = tmem_base + lane_addr + kStageCol + (uint32_t)(h * kEpiCols);
        const uint32_t gy_run = gx_stage + kTile;
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
            k.eps = p.cc.eps;
        }
        WarpTotals *wt = reinterpret_cast<WarpTotals *>(smem + SmemLayout::totals) + ew;
        if (lane == 0) {
            wt->violations = wt->overflow = wt->queued = 0;
            wt->sum = wt->bound_sum = 0.0;
            wt->max = -1.0f;
            wt->max_bound = 0.0f;
            wt->argmax_i = wt->argmax_j = 0x7fffffff;
        }
        uint32_t *hrow = s_hist + ew * 32 + lane;  // bins 2w, 2w+1 at hrow[w * 256]
        int tiles_since_flush = 0;
        // the tile waiting for (or in) classification
        bool pend = false;
        int pend_pieces = 0;
        long long pend_t = 0;
        int pend_i = 0, pend_j0 = 0;
        float4 pend_ri = make_float4(0.f, 0.f, 0.f, 0.f);
        unsigned long long pend_vmask = 0ull, qmask = 0ull;
        RowAcc acc{0.0f, 0.0f, 0.0f, -1.0f, 0, 0, 0, 0};

        // classifies the next 8-column piece of the pending tile
        auto classify_next = [&]() {
            const int c0 = pend_pieces * kPiece;
            uint32_t ux[kPiece], uy[kPiece];
            tmem_ld8x2_wait(gx_stage + c0, gy_run + c0, ux, uy);
            float px[kPiece], py[kPiece];
#pragma unroll
            for (int c = 0; c < kPiece; ++c) {
                const bool valid = (pend_vmask >> (c0 + c)) & 1ull;
                px[c] = valid ? __uint_as_float(ux[c]) : __int_as_float(0x7fc00000);
                py[c] = __uint_as_float(uy[c]);
            }
            if (DUMP && p.dump && pend_t < p.dump_tiles) {
                float4 *drow = p.dump + (size_t)pend_t * kTile * kTile + r * kTile + h * kEpiCols + c0;
                classify_piece<DUMP>(px, py, pend_ri, p.rs + pend_j0 + c0, c0, k, hrow, acc, qmask, drow);
            } else {
                classify_piece<false>(px, py, pend_ri, p.rs + pend_j0 + c0, c0, k, hrow, acc, qmask,
                                      nullptr);
            }
            ++pend_pieces;
        };
        // queue pushes and warp totals of the fully classified pending tile
        auto finish_pending = [&]() {
            while (pend_pieces < kPieces) classify_next();
            qmask &= pend_vmask;
            int nq = __popcll(qmask);
            while (__any_sync(0xffffffffu, qmask != 0ull)) {
                const bool has = qmask != 0ull;
                const int c = has ? __ffsll((long long)qmask) - 1 : 0;
                if (has) qmask &= qmask - 1;
                queue_push(has, pend_i, pend_j0 + c, p.queue, p.qcount, p.qcap);
            }
            int aj_t = pend_j0 + acc.arg, ai_t = pend_i;
            for (int o = 16; o > 0; o >>= 1) {
                acc.viol += __shfl_xor_sync(0xffffffffu, acc.viol, o);
                acc.over += __shfl_xor_sync(0xffffffffu, acc.over, o);
                acc.certain += __shfl_xor_sync(0xffffffffu, acc.certain, o);
                nq += __shfl_xor_sync(0xffffffffu, nq, o);
                acc.sum += __shfl_xor_sync(0xffffffffu, acc.sum, o);
                acc.bsum += __shfl_xor_sync(0xffffffffu, acc.bsum, o);
                acc.mxb = fmaxf(acc.mxb, __shfl_xor_sync(0xffffffffu, acc.mxb, o));
                const float om = __shfl_xor_sync(0xffffffffu, acc.mx, o);
                const int oi = __shfl_xor_sync(0xffffffffu, ai_t, o);
                const int oj = __shfl_xor_sync(0xffffffffu, aj_t, o);
                if (better_max(om, oi, oj, acc.mx, ai_t, aj_t)) { acc.mx = om; ai_t = oi; aj_t = oj; }
            }
            if (lane == 0) {
                wt->violations += (unsigned)acc.viol;
                wt->overflow += (unsigned)acc.over;
                wt->queued += (unsigned)nq;
                wt->sum += (double)acc.sum;
                wt->bound_sum += (double)acc.bsum;
                wt->max_bound = fmaxf(wt->max_bound, acc.mxb);
                if (acc.mx >= 0.0f && better_max(acc.mx, ai_t, aj_t, wt->max, wt->argmax_i, wt->argmax_j)) {
                    wt->max = acc.mx;
                    wt->argmax_i = ai_t;
                    wt->argmax_j = aj_t;
                }
                // a certain violation: delta - B > eps for some pair
                if (p.stop_flag && acc.certain > 0) atomicExch(p.stop_flag, 1);
            }
            pend = false;
            if (++tiles_since_flush == kHistFlushTiles) {
                tiles_since_flush = 0;
                fold_hist(s_hist, ew, mine);
            }
        };

        long long t = blockIdx.x;               // the producer's static tile sequence
        bool ok = true;
        while (ok) {
            float gx[kEpiCols];
#pragma unroll
            for (int c = 0; c < kEpiCols; ++c) gx[c] = 0.0f;
            bool stop = false;
            for (int ks = 0; ks < ksteps; ++ks) {
                ok = warp_wait(bar_sfull + 8 * slot, sphase, p.status, 3);
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
                const uint32_t ta = tmem_base + lane_addr + (uint32_t)(slot * kTile + h * kEpiCols);
                if (ks < p.kx_steps) {
                    // X chunk: registers, all 64 columns behind one wait
                    uint32_t v[64];
                    tmem_ld64_wait(ta, v);
#pragma unroll
                    for (int c = 0; c < kEpiCols; ++c) gx[c] += __uint_as_float(v[c]);
                } else {
                    // Y chunk: the running columns (the first Y chunk starts them)
                    if (ks == p.kx_steps && pend) finish_pending();
                    const bool first = ks == p.kx_steps;
#pragma unroll
                    for (int hh = 0; hh < kEpiCols / 32; ++hh) {
                        uint32_t v[32], w[32];
                        if (first) {
                            tmem_ld16x2_wait(ta + hh * 32, ta + hh * 32 + 16,
                                             *reinterpret_cast<uint32_t(*)[16]>(v),
                                             *reinterpret_cast<uint32_t(*)[16]>(v + 16));
                        } else {
                            tmem_ld32x2_wait(ta + hh * 32, gy_run + hh * 32, v, w);
#pragma unroll
                            for (int c = 0; c < 32; ++c)
                                v[c] = __float_as_uint(__uint_as_float(v[c]) + __uint_as_float(w[c]));
                        }
                        tmem_st16(gy_run + hh * 32, *reinterpret_cast<uint32_t(*)[16]>(v));
                        tmem_st16(gy_run + hh * 32 + 16, *reinterpret_cast<uint32_t(*)[16]>(v + 16));
                    }
                    tmem_wait_st();
                }
                tc_fence_before();
                mbar_arrive(bar_sempty + 8 * slot);
                if (++slot == kSlots) {
                    slot = 0;
                    sphase ^= 1;
                }
                // one piece of the previous tile between X-chunk drains
                if (ks < p.kx_steps && pend && pend_pieces < kPieces) classify_next();
            }
            if (!ok || stop) break;
            // this tile's Y chunks have started the running columns, so the
            // previous tile is finished (kx_steps >= 1 always precedes them)
            // ---- park gx in the staging columns; the tile is now pending
#pragma unroll
            for (int qd = 0; qd < kEpiCols / 16; ++qd) {
                uint32_t vx[16];
#pragma unroll
                for (int c = 0; c < 16; ++c) vx[c] = __float_as_uint(gx[qd * 16 + c]);
                tmem_st16(gx_stage + qd * 16, vx);
            }
            tmem_wait_st();
            const uint32_t packed = p.sched[t];
            const int I = (int)(packed >> 16), J = (int)(packed & 0xFFFF);
            pend = true;
            pend_pieces = 0;
            pend_t = t;
            pend_i = I * kTile + r;
            pend_ri = __ldg(p.rs + pend_i);
            pend_j0 = J * kTile + h * kEpiCols;
            // the 64 column statistics the classification reads, one lane per
            // pair of rows: in L1 by the time the next tile's drains begin
            asm volatile("prefetch.global.L1 [%0];" ::"l"(p.rs + pend_j0 + 2 * lane));
            pend_vmask = ~0ull;
            if (!((I < J) && (J * kTile + kTile <= p.n))) {
                // diagonal or ragged tile: columns that are not pairs i < j < n
                // get a NaN Gram entry and their queue bit is cleared
                for (int c = 0; c < kEpiCols; ++c) {
                    const int j = pend_j0 + c;
                    if (!((pend_i < j) & (j < p.n))) pend_vmask &= ~(1ull << c);
                }
            }
            qmask = 0ull;
            acc = RowAcc{0.0f, 0.0f, 0.0f, -1.0f, 0, 0, 0, 0};
            t += gridDim.x;
        }
        // the last tile (its sums are complete in TMEM)
        if (ok && pend) finish_pending();
        // ---- this warp's partial: the rest of its histogram and its totals
        fold_hist(s_hist, ew, mine);
        if (lane == 0) {
            mine->violations = wt->violations;
            mine->queued = wt->queued;
            mine->overflow = wt->overflow;
            mine->pairs += wt->overflow;  // fold_hist added the binned pairs
            mine->degenerate = 0;
            mine->sum = wt->sum;
            mine->bound_sum = wt->bound_sum;
            mine->max = wt->max;
            mine->max_bound = wt->max_bound;
            mine->argmax_i = wt->argmax_i;
            mine->argmax_j = wt->argmax_j;
        }
    }

    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                     "r"(kTmemCols)
                     : "memory");
    }
}

__global__ void pack_row_stats(const RowStat *__restrict__ rx, const RowStat *__restrict__ ry,
                               int64_t n_pad, float4 *__restrict__ out) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n_pad) out[r] = make_float4(rx[r].n2, ry[r].n2, rx[r].q4, ry[r].q4);
}

// ------------------------------------------------------------------ host side
using EncodeFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                              const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                              const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                              CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn encode_fn() {
    static EncodeFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeFn>(p);
    });
    if (!fn) fail(ADAGIO_E_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
    return fn;
}

CUtensorMap plane_map(const uint16_t *plane, int64_t rows, int cols, bool bf16) {
    CUtensorMap m;
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
    const cuuint32_t box[2] = {(cuuint32_t)kKStep, (cuuint32_t)kTile};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = encode_fn()(&m, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16,
                             2, const_cast<uint16_t *>(plane), dims, strides, box, estr,
                             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) fail(ADAGIO_E_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return m;
}

// Band order of the upper triangle: bands of kBand tile rows; in a band, J
// runs left to right and I over the band's rows with I <= J.
constexpr int kBand = 8;

std::vector<uint32_t> band_schedule(int T) {
    std::vector<uint32_t> s;
    s.reserve((size_t)T * (T + 1) / 2);
    for (int b0 = 0; b0 < T; b0 += kBand) {
        const int b1 = std::min(T, b0 + kBand);
        for (int J = b0; J < T; ++J)
            for (int I = b0; I < b1 && I <= J; ++I) s.push_back(((uint32_t)I << 16) | (uint32_t)J);
    }
    return s;
}

}  // namespace

// Per-context cache of the device copy of the schedule.
// The schedule of T tile rows, resident on the device for the context's
// lifetime (built on first use: a synchronous upload, so callers that capture
// graphs make it resident first with tc_prepare).
static const uint32_t *schedule_for(adagio_ctx *ctx, int T) {
    auto it = ctx->tc_sched.find(T);
    if (it != ctx->tc_sched.end()) return it->second;
    std::vector<uint32_t> s = band_schedule(T);
    uint32_t *dev = nullptr;
    ADAGIO_CUDA(cudaMalloc(&dev, s.size() * sizeof(uint32_t)));
    cudaError_t e = cudaMemcpy(dev, s.data(), s.size() * sizeof(uint32_t), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(dev);
        ADAGIO_CUDA(e);
    }
    ctx->tc_sched[T] = dev;
    return dev;
}

void tc_prepare(adagio_ctx *ctx, int T) { (void)schedule_for(ctx, T); }

// CTAs of one certificate launch: one per SM (the shared-memory footprint
// allows one), never more than there are tiles, so that small problems of a
// batch leave SMs to the others
int cert_tc_ctas(adagio_ctx *ctx, int64_t n) {
    const long long T = (n + kTile - 1) / kTile;
    const long long tiles = T * (T + 1) / 2;
    return (int)std::min<long long>(ctx->num_sms, tiles);
}

void tc_tile_coords(int T, long long t, int *I, int *J) {
    const std::vector<uint32_t> s = band_schedule(T);
    const uint32_t v = s.at((size_t)t);
    *I = (int)(v >> 16);
    *J = (int)(v & 0xFFFF);
}

// raises the kernels' dynamic shared-memory limit (once per device)
void cert_tc_init() {
    set_max_dyn_smem((const void *)cert_tc_kernel<true>, (int)kSmemBytes);
    set_max_dyn_smem((const void *)cert_tc_kernel<false>, (int)kSmemBytes);
}

bool launch_cert_tc(const CertLaunch &L, int precision, cudaStream_t st) {
    const PrepMat &x = *L.x, &y = *L.y;
    if (!x.hi || !y.hi) return false;
    if (x.n_pad / kTile >= 65536) return false;
    const bool bf16 = precision == ADAGIO_PREC_BF16X3;
    const CUtensorMap mxh = plane_map(x.hi, x.n_pad, x.Kp16, bf16);
    const CUtensorMap mxl = plane_map(x.lo, x.n_pad, x.Kp16, bf16);
    const CUtensorMap myh = plane_map(y.hi, y.n_pad, y.Kp16, bf16);
    const CUtensorMap myl = plane_map(y.lo, y.n_pad, y.Kp16, bf16);
    TcArgs a;
    a.rs = reinterpret_cast<const float4 *>(L.rs_xy);
    pack_row_stats<<<(unsigned)ceil_div(x.n_pad, 256), 256, 0, st>>>(x.rs, y.rs, x.n_pad,
                                                                     (float4 *)L.rs_xy);
    ADAGIO_CHECK_LAUNCH();
    // ex = q4_i q4_j + (c_acc + c_r)(n2_i + n2_j) dominates the split model's
    // q1 term, because 2 |a| |b| <= |a|^2 + |b|^2
    a.cx = x.bm.cacc + L.cc.c_r;
    a.cy = y.bm.cacc + L.cc.c_r;
    a.scale_x = x.scale;
    a.scale_y = y.scale;
    const int T = (int)(x.n_pad / kTile);
    a.sched = schedule_for(L.ctx, T);
    a.ntp = (long long)T * (T + 1) / 2;
    a.n = (int)x.n;
    a.kx_steps = x.Kp16 / kKStep;
    a.ky_steps = y.Kp16 / kKStep;
    // instruction descriptor, kind::f16: D = F32 (bits 4-5 = 1), A/B format
    // F16 = 0 / BF16 = 1 (bits 7-9, 10-12), K-major A and B, N >> 3 at bit
    // 17, M >> 4 at bit 24
    const uint32_t fmt = bf16 ? 1u : 0u;
    a.idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(kTile >> 3) << 17) |
              ((uint32_t)(kTile >> 4) << 24);
    a.cc = L.cc;
    a.partials = L.partials;
    a.queue = L.queue;
    a.qcount = L.qcount;
    a.qcap = L.qcap;
    a.stop_flag = L.stop_flag;
    a.status = L.status;
    a.dump = reinterpret_cast<float4 *>(L.dump);
    a.dump_tiles = L.dump_tiles;
    ADAGIO_CUDA(cudaMemsetAsync(L.partials, 0, sizeof(CertPartial) * L.grid, st));
    cert_tc_init();
    if (L.dump)
        cert_tc_kernel<true><<<L.grid / kEpiWarps, kThreads, kSmemBytes, st>>>(mxh, mxl, myh, myl, a);
    else
        cert_tc_kernel<false><<<L.grid / kEpiWarps, kThreads, kSmemBytes, st>>>(mxh, mxl, myh, myl, a);
    ADAGIO_CHECK_LAUNCH();
    return true;
}

}  // namespace adagio
