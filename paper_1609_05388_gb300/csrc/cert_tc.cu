// K8 (tensor-core path): all-pairs distortion tiles on tcgen05.
//
// One persistent CTA per SM walks 128 x 128 tiles (I, J), I <= J, of the
// pair matrix in the band order of the schedule table (bands of 8 tile rows,
// so the I-tiles of a band stay in L2 while the J-tiles stream).  For every
// tile it forms
//     Gy = Yc[I] Yc[J]^T   and   Gx = Xc[I] Xc[J]^T
// from 2-term split planes (hi + lo, FP16 or BF16, power-of-two scaled) with
// three products hi.hi + hi.lo + lo.hi per K chunk, accumulated in FP32 in
// tensor memory, and hands the two tiles to the epilogue (cert_common.cuh),
// which classifies every pair (Eq. 2), accumulates max / histogram / counts
// and queues the pairs that need the exact recompute.
//
// Roles (192 threads):
//   warp 0      TMA producer: 4 planes (A hi/lo, B hi/lo) of 64 K-elements per
//               stage, 3 stages of 64 KB, 128-byte swizzle
//   warp 1      TMEM owner (512 columns) and MMA issuer: tcgen05.mma kind::f16,
//               M = N = 128, K = 16, into two accumulator buffers of
//               256 columns (Gx | Gy), so the epilogue of tile t overlaps the
//               MMAs of tile t + 1
//   warps 2..5  epilogue: tcgen05.ld of their 32-lane quarter, 16 columns at
//               a time
// The producer decides the tile sequence and sends it down the pipeline (a
// tile index per first stage, -1 to stop), so early exit needs no CTA-wide
// barrier.  Every wait is bounded: on timeout the role records a status word
// and leaves, the producer drains its in-flight copies, the MMA warp waits
// for its last commit, and TMEM is freed.
#include <cuda.h>

#include "internal.cuh"
#include "cert.cuh"

#include <mutex>
#include <vector>

namespace adagio {

namespace {

constexpr int kThreads = 192;
constexpr int kStages = 3;
constexpr int kTile = 128;
constexpr int kKStep = 64;                                  // fp16 elements per stage row
constexpr uint32_t kPlaneBytes = kTile * kKStep * 2;        // 16 KB
constexpr uint32_t kStageBytes = 4 * kPlaneBytes;           // 64 KB
constexpr uint32_t kTmemCols = 512;
constexpr int kHistFlushTiles = 256;                        // u16 counters: <= 128 per tile
constexpr long long kSpinLimit = 4000000000ll;              // clock64 cycles (~2 s)

struct TcArgs {
    const RowStat *rsx, *rsy;
    const float *scale_x, *scale_y;
    const uint32_t *sched;     // (I << 16) | J per tile pair
    long long ntp;
    int n, kx_steps, ky_steps;
    uint32_t idesc;
    CertConst cc;
    CertPartial *partials;
    int2 *queue;
    unsigned long long *qcount, qcap;
    int *stop_flag;
    int *status;
    float4 *dump;              // optional: (dx2, dy2, ex, ey) of tile pairs t < dump_tiles
    long long dump_tiles;
};

struct SmemLayout {
    static constexpr uint32_t stages = 0;
    static constexpr uint32_t hist = kStages * kStageBytes;              // u16 [64][128]
    static constexpr uint32_t jstat = hist + kBins * 128 * 2;            // RowStat [2][128]
    static constexpr uint32_t red = jstat + 2 * 128 * sizeof(RowStat);   // reduction scratch
    static constexpr uint32_t bars = red + 4 * 1024;
    static constexpr uint32_t cmd = bars + 256;                           // int [kStages + 2]
    static constexpr uint32_t tmem_ptr = cmd + 64;
    static constexpr uint32_t total = tmem_ptr + 16;
};
constexpr size_t kSmemBytes = SmemLayout::total + 1024;   // + alignment slack

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

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(r[q]);
}

__device__ __forceinline__ void tmem_wait_ld() {
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void epi_bar() {  // the 4 epilogue warps only
    asm volatile("bar.sync 1, 128;" ::: "memory");
}

// ---------------------------------------------------------------- the kernel
__global__ void __launch_bounds__(kThreads, 1)
    cert_tc_kernel(const __grid_constant__ CUtensorMap map_xh, const __grid_constant__ CUtensorMap map_xl,
                   const __grid_constant__ CUtensorMap map_yh, const __grid_constant__ CUtensorMap map_yl,
                   TcArgs p) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                ~uintptr_t(1023));
    const uint32_t sbase = smem_u32(smem);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    uint16_t *s_hist = reinterpret_cast<uint16_t *>(smem + SmemLayout::hist);
    RowStat *s_jx = reinterpret_cast<RowStat *>(smem + SmemLayout::jstat);
    RowStat *s_jy = s_jx + 128;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + SmemLayout::bars);
    int *s_cmd = reinterpret_cast<int *>(smem + SmemLayout::cmd);      // [kStages] stage cmds, [kStages+b] tmem cmds
    uint32_t *s_tmem = reinterpret_cast<uint32_t *>(smem + SmemLayout::tmem_ptr);
    const uint32_t bar_full = smem_u32(bars);                 // [kStages]
    const uint32_t bar_empty = bar_full + 8 * kStages;        // [kStages]
    const uint32_t bar_tfull = bar_empty + 8 * kStages;       // [2]
    const uint32_t bar_tempty = bar_tfull + 16;               // [2]
    const uint32_t bar_done = bar_tempty + 16;                // MMA drain

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(bar_full + 8 * s, 1);
            mbar_init(bar_empty + 8 * s, 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(bar_tfull + 8 * b, 1);
            mbar_init(bar_tempty + 8 * b, 128);
        }
        mbar_init(bar_done, 1);
        for (int q = 0; q < kStages + 3; ++q) s_cmd[q] = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp >= 2) {
        const int et = threadIdx.x - 64;
        for (int b = 0; b < kBins; ++b) s_hist[b * 128 + et] = 0;
    }
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
        // lane 0 waits and issues; the outcome of every wait is broadcast so
        // the warp never diverges on a timeout
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
                int w = 0;
                if (lane == 0) {
                    w = mbar_wait(bar_empty + 8 * stage, phase ^ 1, p.status, 1);
                    if (w) {
                        s_cmd[stage] = -1;
                        mbar_arrive(bar_full + 8 * stage);
                    }
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
                int w = 0;
                if (lane == 0) w = mbar_wait(bar_empty + 8 * stage, phase ^ 1, p.status, 1);
                ok = __shfl_sync(0xffffffffu, w, 0) != 0;
                if (!ok) break;
                if (lane == 0) {
                    if (ks == 0) s_cmd[stage] = (int)t;
                    const uint32_t bar = bar_full + 8 * stage;
                    mbar_arrive_expect_tx(bar, kStageBytes);
                    const uint32_t dst = sbase + SmemLayout::stages + stage * kStageBytes;
                    const bool is_y = ks < p.ky_steps;
                    const int k0 = (is_y ? ks : ks - p.ky_steps) * kKStep;
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
        int stage = 0;
        uint32_t phase = 0;
        int buf = 0;
        uint32_t bphase = 0;
        bool any = false;
        while (true) {
            int w = 0, t = -1;
            if (lane == 0) {
                w = mbar_wait(bar_full + 8 * stage, phase, p.status, 2);
                if (w) t = s_cmd[stage];
            }
            if (!__shfl_sync(0xffffffffu, w, 0)) break;
            t = __shfl_sync(0xffffffffu, t, 0);
            if (t < 0) {
                // forward the stop to the epilogue once its buffer is free; a
                // plain arrive releases the store of the stop word
                if (lane == 0 && mbar_wait(bar_tempty + 8 * buf, bphase ^ 1, p.status, 2)) {
                    s_cmd[kStages + buf] = -1;
                    mbar_arrive(bar_tfull + 8 * buf);
                }
                __syncwarp();
                break;
            }
            if (lane == 0) w = mbar_wait(bar_tempty + 8 * buf, bphase ^ 1, p.status, 2);
            if (!__shfl_sync(0xffffffffu, w, 0)) break;
            tc_fence_after();
            bool ok = true;
            for (int ks = 0; ks < ksteps; ++ks) {
                if (ks > 0) {
                    if (lane == 0) w = mbar_wait(bar_full + 8 * stage, phase, p.status, 2);
                    ok = __shfl_sync(0xffffffffu, w, 0) != 0;
                    if (!ok) break;
                    tc_fence_after();
                }
                if (lane == 0) {
                    const bool is_y = ks < p.ky_steps;
                    const bool first = (ks == 0) || (ks == p.ky_steps);
                    const uint32_t d = tmem_base + (uint32_t)(buf * 256 + (is_y ? 128 : 0));
                    const uint32_t a0 = sbase + SmemLayout::stages + stage * kStageBytes;
                    const uint64_t ah = sw128_desc(a0), al = sw128_desc(a0 + kPlaneBytes);
                    const uint64_t bh = sw128_desc(a0 + 2 * kPlaneBytes);
                    const uint64_t bl = sw128_desc(a0 + 3 * kPlaneBytes);
#pragma unroll
                    for (int kk = 0; kk < kKStep / 16; ++kk) {
                        const uint64_t off = (uint64_t)(kk * 32) >> 4;  // 16 elements = 32 bytes
                        tc_mma(d, ah + off, bh + off, p.idesc, (first && kk == 0) ? 0u : 1u);
                        tc_mma(d, ah + off, bl + off, p.idesc, 1u);
                        tc_mma(d, al + off, bh + off, p.idesc, 1u);
                    }
                    tc_commit(bar_empty + 8 * stage);
                    any = true;
                }
                __syncwarp();
                if (++stage == kStages) {
                    stage = 0;
                    phase ^= 1;
                }
            }
            if (!ok) break;
            if (lane == 0) tc_commit(bar_tfull + 8 * buf);
            __syncwarp();
            buf ^= 1;
            if (buf == 0) bphase ^= 1;
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
        const int et = threadIdx.x - 64;   // 0..127
        const int quarter = warp & 3;      // TMEM lanes this warp may access
        const int r = quarter * 32 + lane; // row of the tile owned by this thread
        int buf = 0;
        uint32_t bphase = 0;
        unsigned long long npairs = 0, nviol = 0, nover = 0, nqueued = 0;
        double sum = 0.0, bsum = 0.0;
        float mx = -1.0f, mxb_all = 0.0f;
        int ai = 0x7fffffff, aj = 0x7fffffff;
        const float sx = *p.scale_x, sy = *p.scale_y;
        const float inv_sx2 = 1.0f / (sx * sx), inv_sy2 = 1.0f / (sy * sy);
        int tiles_since_flush = 0;
        int *s_state = s_cmd + kStages + 2;   // epilogue-wide decision word
        long long t = blockIdx.x;             // same static sequence the producer walks
        while (true) {
            // one thread waits; the decision reaches all 128 through the barrier
            if (et == 0) {
                const bool w = mbar_wait(bar_tfull + 8 * buf, bphase, p.status, 3);
                *s_state = !w ? 2 : (s_cmd[kStages + buf] < 0 ? 1 : 0);
            }
            epi_bar();
            if (*s_state != 0) break;
            tc_fence_after();
            const uint32_t packed = p.sched[t];
            const int I = (int)(packed >> 16), J = (int)(packed & 0xFFFF);
            s_jx[et] = p.rsx[J * kTile + et];
            s_jy[et] = p.rsy[J * kTile + et];
            const RowStat xi = p.rsx[I * kTile + r], yi = p.rsy[I * kTile + r];
            epi_bar();
            const int i = I * kTile + r;
            const uint32_t tx = tmem_base + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(buf * 256);
            float tsum = 0.0f, tbsum = 0.0f;
            bool stop = false;
            float4 *dump = (p.dump && t < p.dump_tiles) ? p.dump + (size_t)t * kTile * kTile : nullptr;
#pragma unroll 1
            for (int c0 = 0; c0 < kTile; c0 += 16) {
                float gx[16], gy[16];
                tmem_ld16(tx + c0, gx);
                tmem_ld16(tx + 128 + c0, gy);
                tmem_wait_ld();
#pragma unroll
                for (int jj = 0; jj < 16; ++jj) {
                    const int lj = c0 + jj;
                    const int j = J * kTile + lj;
                    FastPair fp;
                    int cls = PAIR_SKIP;
                    const float g_x = gx[jj] * inv_sx2, g_y = gy[jj] * inv_sy2;
                    if (i < j && j < p.n)
                        cls = classify_pair(g_x, g_y, xi, s_jx[lj], yi, s_jy[lj], p.cc, fp);
                    if (dump) {
                        const RowStat &xj = s_jx[lj], &yj = s_jy[lj];
                        float4 v;
                        v.x = (xi.n2 + xj.n2) - 2.0f * g_x;
                        v.y = (yi.n2 + yj.n2) - 2.0f * g_y;
                        v.z = fmaf(xi.q4, xj.q4, fmaf(xi.q1, xj.q1, p.cc.c_r * (xi.n2 + xj.n2)));
                        v.w = fmaf(yi.q4, yj.q4, fmaf(yi.q1, yj.q1, p.cc.c_r * (yi.n2 + yj.n2)));
                        dump[r * kTile + lj] = v;
                    }
                    queue_push(cls == PAIR_QUEUE, i, j, p.queue, p.qcount, p.qcap);
                    if (cls == PAIR_OK) {
                        ++npairs;
                        if (fp.bin >= 0) s_hist[fp.bin * 128 + et] += 1; else ++nover;
                        nviol += fp.violation;
                        tsum += fp.delta;
                        tbsum += fp.bound;
                        mxb_all = fmaxf(mxb_all, fp.bound);
                        if (better_max(fp.delta, i, j, mx, ai, aj)) { mx = fp.delta; ai = i; aj = j; }
                        stop |= fp.delta > p.cc.eps + fp.bound;
                    } else if (cls == PAIR_QUEUE) {
                        ++nqueued;
                    }
                }
            }
            tc_fence_before();
            mbar_arrive(bar_tempty + 8 * buf);
            t += gridDim.x;
            sum += (double)tsum;
            bsum += (double)tbsum;
            if (p.stop_flag && stop) atomicExch(p.stop_flag, 1);
            buf ^= 1;
            if (buf == 0) bphase ^= 1;
            epi_bar();  // every thread is done with s_jx / s_jy of this tile
            if (++tiles_since_flush == kHistFlushTiles) {
                tiles_since_flush = 0;
                // 2 threads per bin fold 64 u16 counters each into the CTA partial
                const int b = et >> 1, half = et & 1;
                unsigned acc = 0;
                for (int q = 0; q < 64; ++q) acc += s_hist[b * 128 + half * 64 + q];
                epi_bar();
                for (int q = 0; q < 64; ++q) s_hist[b * 128 + half * 64 + q] = 0;
                if (acc) atomicAdd(&p.partials[blockIdx.x].hist[b], (unsigned long long)acc);
                epi_bar();
            }
        }
        // final fold of the histogram and the scalar statistics
        epi_bar();
        {
            const int b = et >> 1, half = et & 1;
            unsigned acc = 0;
            for (int q = 0; q < 64; ++q) acc += s_hist[b * 128 + half * 64 + q];
            if (acc) atomicAdd(&p.partials[blockIdx.x].hist[b], (unsigned long long)acc);
        }
        unsigned long long u[4] = {npairs, nviol, nover, nqueued};
        for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
            for (int q = 0; q < 4; ++q) u[q] += __shfl_xor_sync(0xffffffffu, u[q], o);
            sum += __shfl_xor_sync(0xffffffffu, sum, o);
            bsum += __shfl_xor_sync(0xffffffffu, bsum, o);
            mxb_all = fmaxf(mxb_all, __shfl_xor_sync(0xffffffffu, mxb_all, o));
            const float om = __shfl_xor_sync(0xffffffffu, mx, o);
            const int oi = __shfl_xor_sync(0xffffffffu, ai, o);
            const int oj = __shfl_xor_sync(0xffffffffu, aj, o);
            if (better_max(om, oi, oj, mx, ai, aj)) { mx = om; ai = oi; aj = oj; }
        }
        unsigned long long *ru = reinterpret_cast<unsigned long long *>(smem + SmemLayout::red);
        double *rd = reinterpret_cast<double *>(ru + 4 * 4);
        float *rf = reinterpret_cast<float *>(rd + 2 * 4);
        int *ri = reinterpret_cast<int *>(rf + 2 * 4);
        const int ew = et >> 5;
        if (lane == 0) {
            for (int q = 0; q < 4; ++q) ru[q * 4 + ew] = u[q];
            rd[ew] = sum; rd[4 + ew] = bsum;
            rf[ew] = mx; rf[4 + ew] = mxb_all;
            ri[ew] = ai; ri[4 + ew] = aj;
        }
        epi_bar();
        if (et == 0) {
            CertPartial *dst = p.partials + blockIdx.x;
            unsigned long long t4[4] = {0, 0, 0, 0};
            double s0 = 0, s1 = 0;
            float m = -1.0f, mb = 0.0f;
            int bi = 0x7fffffff, bj = 0x7fffffff;
            for (int w = 0; w < 4; ++w) {
                for (int q = 0; q < 4; ++q) t4[q] += ru[q * 4 + w];
                s0 += rd[w]; s1 += rd[4 + w];
                mb = fmaxf(mb, rf[4 + w]);
                if (better_max(rf[w], ri[w], ri[4 + w], m, bi, bj)) { m = rf[w]; bi = ri[w]; bj = ri[4 + w]; }
            }
            dst->pairs = t4[0]; dst->violations = t4[1]; dst->overflow = t4[2]; dst->queued = t4[3];
            dst->degenerate = 0;
            dst->sum = s0; dst->bound_sum = s1;
            dst->max = m; dst->max_bound = mb; dst->argmax_i = bi; dst->argmax_j = bj;
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
struct SchedCache {
    int T = -1;
    uint32_t *dev = nullptr;
    size_t cap = 0;
};

static std::mutex g_sched_mu;

static const uint32_t *schedule_for(adagio_ctx *ctx, int T) {
    std::lock_guard<std::mutex> lk(g_sched_mu);
    static thread_local std::vector<std::pair<adagio_ctx *, SchedCache>> caches;
    SchedCache *c = nullptr;
    for (auto &e : caches)
        if (e.first == ctx) c = &e.second;
    if (!c) {
        caches.push_back({ctx, SchedCache{}});
        c = &caches.back().second;
    }
    if (c->T != T) {
        std::vector<uint32_t> s = band_schedule(T);
        if (s.size() > c->cap) {
            if (c->dev) cudaFree(c->dev);
            c->dev = nullptr;
            ADAGIO_CUDA(cudaMalloc(&c->dev, s.size() * sizeof(uint32_t)));
            c->cap = s.size();
        }
        ADAGIO_CUDA(cudaMemcpy(c->dev, s.data(), s.size() * sizeof(uint32_t), cudaMemcpyHostToDevice));
        c->T = T;
    }
    return c->dev;
}

int cert_tc_grid(adagio_ctx *ctx) { return ctx->num_sms; }

void tc_tile_coords(int T, long long t, int *I, int *J) {
    const std::vector<uint32_t> s = band_schedule(T);
    const uint32_t v = s.at((size_t)t);
    *I = (int)(v >> 16);
    *J = (int)(v & 0xFFFF);
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
    a.rsx = x.rs;
    a.rsy = y.rs;
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
    ADAGIO_CUDA(cudaFuncSetAttribute(cert_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kSmemBytes));
    cert_tc_kernel<<<L.grid, kThreads, kSmemBytes, st>>>(mxh, mxl, myh, myl, a);
    ADAGIO_CHECK_LAUNCH();
    return true;
}

}  // namespace adagio
