// Split-precision GEMM on tcgen05 (the products of the randomized PCA of
// Sec. 2 / Sec. 4.5 and the projection of Algorithm 1): C = A B^T from the
// 2-term 16-bit planes of A and B.
//
// Persistent: one CTA per SM walks the work items (128 x 128 output tile, K
// split), the barrier phases and TMEM slots running on from item to item, so
// that a CTA's setup is paid once and an item's epilogue overlaps the next
// item's loads and MMAs.  Roles (320 threads):
//   warp 0      TMA producer: A hi/lo and B hi/lo, 64 K-elements per stage,
//               3 stages of 64 KB, 128-byte swizzle
//   warp 1      TMEM owner (2 chunk slots of 128 columns) and MMA issuer:
//               every chunk of two 64-wide K steps goes to a fresh slot, the
//               cross products (hi.lo, lo.hi) first and the hi.hi products
//               last, as in the certificate tiles
//   warps 2..9  drain every slot into FP32 register sums (two warps per TMEM
//               lane quarter, 64 columns each) and write the tile, scaled
//               back by the planes' power-of-two scales
// Split-K partials are summed in FP64 by a second kernel, which also adds the
// bias and mirrors symmetric results.  Every wait is bounded (a status word
// records a timeout; the CTA drains its copies and MMAs and frees TMEM).
#include "internal.cuh"
#include "tc_ptx.cuh"
#include "tcgemm.cuh"

namespace adagio {

using namespace tc;

namespace {

constexpr int kTile = 128;
constexpr int kKStep = 64;
constexpr int kChunkSteps = 2;
constexpr int kStages = 3;
constexpr int kEpiWarps = 8;
constexpr int kThreads = 64 + 32 * kEpiWarps;
constexpr int kEpiCols = 64;
constexpr uint32_t kPlane = kTile * kKStep * 2;     // 16 KB
constexpr uint32_t kStageBytes = 4 * kPlane;        // 64 KB
constexpr uint32_t kTmemCols = 256;                 // two chunk slots
constexpr uint32_t kBars = kStages * kStageBytes;
constexpr uint32_t kTmemPtr = kBars + 128;
constexpr size_t kSmem = kTmemPtr + 16 + 1024;      // + alignment slack
static_assert(kSmem <= 232448, "GEMM tile exceeds the shared-memory limit");

struct GemmArgs {
    int M, N, tiles_n, tiles;  // tiles = tiles_m * tiles_n
    long long items;           // tiles x K splits
    int ksteps, ksplit;        // K steps in total / per split
    int sym;
    const float *sa, *sb;      // power-of-two scales
    int sa_stride, sb_stride;
    const float *bias;         // [N] or null (only with one split)
    float *out;                // [split][M][ldo]
    int64_t ldo, split_stride;
    uint32_t idesc;
    int *status;
};

__global__ void __launch_bounds__(kThreads, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap map_ah, const __grid_constant__ CUtensorMap map_al,
                   const __grid_constant__ CUtensorMap map_bh, const __grid_constant__ CUtensorMap map_bl,
                   GemmArgs p) {
    // work item w: tile w % tiles, K split w / tiles; the mirror of a
    // computed tile (sym, tn < tm) is skipped by every role alike
    struct Item {
        int tm, tn, split, k0, k1, nsteps, nchunks;
    };
    auto item = [&](long long w, Item &it) {
        const int tile = (int)(w % p.tiles);
        it.split = (int)(w / p.tiles);
        it.tm = tile / p.tiles_n;
        it.tn = tile % p.tiles_n;
        it.k0 = it.split * p.ksplit;
        it.k1 = min(p.ksteps, it.k0 + p.ksplit);
        it.nsteps = it.k1 - it.k0;
        it.nchunks = (it.nsteps + kChunkSteps - 1) / kChunkSteps;
        return !(p.sym && it.tn < it.tm);
    };

    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    const uint32_t sbase = smem_u32(smem);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint32_t *s_tmem = reinterpret_cast<uint32_t *>(smem + kTmemPtr);
    const uint32_t bar_full = sbase + kBars;            // [kStages]
    const uint32_t bar_empty = bar_full + 8 * kStages;  // [kStages]
    const uint32_t bar_sfull = bar_empty + 8 * kStages; // [2]
    const uint32_t bar_sempty = bar_sfull + 16;         // [2]
    const uint32_t bar_done = bar_sempty + 16;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(bar_full + 8 * s, 1);
            mbar_init(bar_empty + 8 * s, 1);
        }
        for (int s = 0; s < 2; ++s) {
            mbar_init(bar_sfull + 8 * s, 1);
            mbar_init(bar_sempty + 8 * s, kEpiWarps);
        }
        mbar_init(bar_done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
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

    if (warp == 0) {
        // ------------------------------------------------------ TMA producer
        int stage = 0;
        uint32_t phase = 0;
        bool issued[kStages];
        uint32_t issued_parity[kStages];
        for (int s = 0; s < kStages; ++s) issued[s] = false, issued_parity[s] = 0;
        bool ok = true;
        for (long long w = blockIdx.x; ok && w < p.items; w += gridDim.x) {
            Item it;
            if (!item(w, it)) continue;
            for (int ks = it.k0; ks < it.k1; ++ks) {
                if (!warp_wait(bar_empty + 8 * stage, phase ^ 1, p.status, 1)) {
                    ok = false;
                    break;
                }
                if (lane == 0) {
                    const uint32_t bar = bar_full + 8 * stage;
                    const uint32_t dst = sbase + stage * kStageBytes;
                    mbar_arrive_expect_tx(bar, kStageBytes);
                    tma_load_2d<false>(dst, &map_ah, ks * kKStep, it.tm * kTile, bar);
                    tma_load_2d<false>(dst + kPlane, &map_al, ks * kKStep, it.tm * kTile, bar);
                    tma_load_2d<false>(dst + 2 * kPlane, &map_bh, ks * kKStep, it.tn * kTile, bar);
                    tma_load_2d<false>(dst + 3 * kPlane, &map_bl, ks * kKStep, it.tn * kTile, bar);
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
        if (lane == 0)
            for (int s = 0; s < kStages; ++s)
                if (issued[s]) mbar_wait(bar_full + 8 * s, issued_parity[s], p.status, 1);
        __syncwarp();
    } else if (warp == 1) {
        // ------------------------------------------------------- MMA issuer
        int stage = 0, slot = 0;
        uint32_t phase = 0, sphase = 0;
        bool any = false;
        auto cross = [&](int st, uint32_t d, uint32_t acc_first) {
            const uint32_t a0 = sbase + st * kStageBytes;
            const uint64_t ah = sw128_desc(a0), al = sw128_desc(a0 + kPlane);
            const uint64_t bh = sw128_desc(a0 + 2 * kPlane), bl = sw128_desc(a0 + 3 * kPlane);
#pragma unroll
            for (int kk = 0; kk < kKStep / 16; ++kk) {
                const uint64_t off = (uint64_t)(kk * 32) >> 4;
                tc_mma<false>(d, ah + off, bl + off, p.idesc, kk == 0 ? acc_first : 1u);
                tc_mma<false>(d, al + off, bh + off, p.idesc, 1u);
            }
        };
        auto full_size = [&](int st, uint32_t d) {
            const uint32_t a0 = sbase + st * kStageBytes;
            const uint64_t ah = sw128_desc(a0), bh = sw128_desc(a0 + 2 * kPlane);
#pragma unroll
            for (int kk = 0; kk < kKStep / 16; ++kk) {
                const uint64_t off = (uint64_t)(kk * 32) >> 4;
                tc_mma<false>(d, ah + off, bh + off, p.idesc, 1u);
            }
        };
        bool ok = true;
        for (long long w = blockIdx.x; ok && w < p.items; w += gridDim.x) {
            Item it;
            if (!item(w, it)) continue;
            for (int c = 0; c < it.nchunks; ++c) {
                const int nst = min(kChunkSteps, it.nsteps - c * kChunkSteps);
                if (!warp_wait(bar_full + 8 * stage, phase, p.status, 2) ||
                    !warp_wait(bar_sempty + 8 * slot, sphase ^ 1, p.status, 2)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t d = tmem_base + (uint32_t)(slot * kTile);
                const int st0 = stage;
                int st1 = stage + 1;
                uint32_t ph1 = phase;
                if (st1 == kStages) {
                    st1 = 0;
                    ph1 ^= 1;
                }
                if (lane == 0) {
                    cross(st0, d, 0u);
                    any = true;
                }
                __syncwarp();
                if (nst == 2) {
                    if (!warp_wait(bar_full + 8 * st1, ph1, p.status, 2)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    if (lane == 0) cross(st1, d, 1u);
                    __syncwarp();
                }
                if (lane == 0) {
                    full_size(st0, d);
                    tc_commit<false>(bar_empty + 8 * st0);
                    if (nst == 2) {
                        full_size(st1, d);
                        tc_commit<false>(bar_empty + 8 * st1);
                    }
                    tc_commit<false>(bar_sfull + 8 * slot);
                }
                __syncwarp();
                for (int q = 0; q < nst; ++q)
                    if (++stage == kStages) {
                        stage = 0;
                        phase ^= 1;
                    }
                if (++slot == 2) {
                    slot = 0;
                    sphase ^= 1;
                }
            }
        }
        any = __shfl_sync(0xffffffffu, any ? 1 : 0, 0) != 0;
        if (lane == 0 && any) {
            tc_commit_local<false>(bar_done);
            mbar_wait(bar_done, 0, p.status, 2);
        }
        __syncwarp();
    } else {
        // --------------------------------------------------------- epilogue
        const int ew = warp - 2;
        const int quarter = warp & 3;
        const int h = ew >> 2;
        const uint32_t lane_addr = (uint32_t)(quarter * 32) << 16;
        int slot = 0;
        uint32_t sphase = 0;
        bool ok = true;
        for (long long w = blockIdx.x; ok && w < p.items; w += gridDim.x) {
            Item it;
            if (!item(w, it)) continue;
            float acc[kEpiCols];
#pragma unroll
            for (int c = 0; c < kEpiCols; ++c) acc[c] = 0.0f;
            for (int c = 0; c < it.nchunks; ++c) {
                ok = warp_wait(bar_sfull + 8 * slot, sphase, p.status, 3);
                if (!ok) break;
                tc_fence_after();
                uint32_t v[64];
                tmem_ld64_wait(tmem_base + lane_addr + (uint32_t)(slot * kTile + h * kEpiCols), v);
#pragma unroll
                for (int q = 0; q < kEpiCols; ++q) acc[q] += __uint_as_float(v[q]);
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(bar_sempty + 8 * slot);
                if (++slot == 2) {
                    slot = 0;
                    sphase ^= 1;
                }
            }
            // the item's tile, written while the next item's chunks run
            const int row = it.tm * kTile + quarter * 32 + lane;
            if (ok && row < p.M) {
                const float ia = 1.0f / p.sa[(int64_t)row * p.sa_stride];  // powers of two: exact
                float *dst = p.out + (int64_t)it.split * p.split_stride + (int64_t)row * p.ldo;
                const int c0 = it.tn * kTile + h * kEpiCols;
                // 16-byte stores where the row allows them: a lane writes its own
                // row, so each store instruction touches 32 rows
                const bool vec = c0 + kEpiCols <= p.N && ((reinterpret_cast<uintptr_t>(dst + c0) & 15u) == 0);
                if (vec) {
#pragma unroll
                    for (int q = 0; q < kEpiCols; q += 4) {
                        float v[4];
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const int col = c0 + q + e;
                            v[e] = acc[q + e] * ia * (1.0f / p.sb[(int64_t)col * p.sb_stride]);
                            if (p.bias) v[e] += p.bias[col];
                        }
                        *reinterpret_cast<float4 *>(dst + c0 + q) = make_float4(v[0], v[1], v[2], v[3]);
                    }
                } else {
#pragma unroll
                    for (int q = 0; q < kEpiCols; ++q) {
                        const int col = c0 + q;
                        if (col < p.N) {
                            float v = acc[q] * ia * (1.0f / p.sb[(int64_t)col * p.sb_stride]);
                            if (p.bias) v += p.bias[col];
                            dst[col] = v;
                        }
                    }
                }
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                     "r"(kTmemCols)
                     : "memory");
}

// C[r, c] = sum over splits (FP64) + bias[c]; sym: the lower tiles mirror the upper ones
__global__ void tc_gemm_reduce(const float *__restrict__ part, int splits, int64_t split_stride,
                               int M, int N, int64_t ldp, const float *__restrict__ bias, int sym,
                               float *__restrict__ C, int64_t ldc) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)M * N) return;
    const int r = (int)(e / N), c = (int)(e % N);
    int rr = r, cc = c;
    if (sym && c / kTile < r / kTile) rr = c, cc = r;
    double s = 0.0;
    for (int z = 0; z < splits; ++z) s += (double)part[(int64_t)z * split_stride + (int64_t)rr * ldp + cc];
    if (bias) s += (double)bias[c];
    C[(int64_t)r * ldc + c] = (float)s;
}

// One warp per row: power-of-two scale s with max |s x| <= 2^14, FP16 hi =
// round(s x), lo = round(s x - hi); zeros beyond the real columns.
__global__ void split_rows_kernel(const float *__restrict__ src, int64_t rows, int cols, int64_t ld,
                                  int Kp, uint16_t *__restrict__ hi, uint16_t *__restrict__ lo,
                                  float *__restrict__ scale) {
    const int lane = threadIdx.x & 31;
    const int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (r >= rows) return;
    float amax = 0.0f;
    for (int k = lane; k < cols; k += 32) amax = fmaxf(amax, fabsf(src[r * ld + k]));
    for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    float s = 1.0f;
    if (amax > 0.0f) {
        int e = (int)floorf(log2f(16384.0f / amax));
        e = max(-100, min(e, 100));
        s = ldexpf(1.0f, e);
        while (amax * s > 16384.0f) s *= 0.5f;
    }
    if (lane == 0) scale[r] = s;
    for (int k = lane; k < Kp; k += 32) {
        const float v = k < cols ? __fmul_rn(src[r * ld + k], s) : 0.0f;
        const __half hh = __float2half_rn(v);
        const __half ll = __float2half_rn(__fsub_rn(v, __half2float(hh)));
        hi[r * Kp + k] = __half_as_ushort(hh);
        lo[r * Kp + k] = __half_as_ushort(ll);
    }
}

// Transposed planes of s (X - mu): 32 x 32 tiles through shared memory.
__global__ void split_transpose_kernel(const float *__restrict__ X, int64_t n, int cols, int64_t ldx,
                                       const float *__restrict__ mu, const unsigned *__restrict__ amax_bits,
                                       int Kp, uint16_t *__restrict__ hi, uint16_t *__restrict__ lo,
                                       float *__restrict__ scale) {
    __shared__ float t[32][33];
    const float amax = __uint_as_float(*amax_bits);
    float s = 1.0f;
    if (amax > 0.0f) {
        int e = (int)floorf(log2f(16384.0f / amax));
        e = max(-100, min(e, 100));
        s = ldexpf(1.0f, e);
        while (amax * s > 16384.0f) s *= 0.5f;
    }
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0 && threadIdx.y == 0) *scale = s;
    const int c = blockIdx.x * 32 + threadIdx.x;
    const int64_t ktiles = (Kp + 31) / 32;
    for (int64_t kt = blockIdx.y; kt < ktiles; kt += gridDim.y) {
        for (int j = threadIdx.y; j < 32; j += 8) {
            const int64_t r = kt * 32 + j;
            t[j][threadIdx.x] = (r < n && c < cols) ? __fmul_rn(__fsub_rn(X[r * ldx + c], mu[c]), s) : 0.0f;
        }
        __syncthreads();
        const int64_t k = kt * 32 + threadIdx.x;
        for (int j = threadIdx.y; j < 32; j += 8) {
            const int cc = blockIdx.x * 32 + j;
            if (cc < cols && k < Kp) {
                const float v = t[threadIdx.x][j];
                const __half hh = __float2half_rn(v);
                const __half ll = __float2half_rn(__fsub_rn(v, __half2float(hh)));
                hi[(int64_t)cc * Kp + k] = __half_as_ushort(hh);
                lo[(int64_t)cc * Kp + k] = __half_as_ushort(ll);
            }
        }
        __syncthreads();
    }
}

// out[r] = A[r, :] . v, one warp per row
__global__ void rows_dot_kernel(const float *__restrict__ A, int rows, int cols, int64_t lda,
                                const float *__restrict__ v, float *__restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (r >= rows) return;
    float s = 0.0f;
    for (int k = lane; k < cols; k += 32) s = fmaf(A[(int64_t)r * lda + k], v[k], s);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) out[r] = s;
}

struct Plan {
    int tiles_m, tiles_n, tiles, ksteps, ksplit, splits;
};

Plan plan(adagio_ctx *ctx, int M, int N, int Kp, bool sym) {
    Plan q;
    q.tiles_m = (M + kTile - 1) / kTile;
    q.tiles_n = (N + kTile - 1) / kTile;
    q.tiles = sym ? q.tiles_m * (q.tiles_m + 1) / 2 : q.tiles_m * q.tiles_n;
    q.ksteps = Kp / kKStep;
    // split K until the work items fill the SMs once
    const int want = std::max(1, std::min(q.ksteps, (ctx->num_sms + q.tiles - 1) / q.tiles));
    q.ksplit = (q.ksteps + want - 1) / want;
    q.splits = (q.ksteps + q.ksplit - 1) / q.ksplit;
    return q;
}

}  // namespace

void tc_gemm_init() { set_max_dyn_smem((const void *)tc_gemm_kernel, (int)kSmem); }

int64_t tc_gemm_workspace(adagio_ctx *ctx, int M, int N, int Kp, bool sym) {
    // smaller shapes have fewer tiles and so more K splits: take the largest
    // partial buffer over every M' <= M, N' <= N (sym: M' = N' = M)
    const int tm = (M + kTile - 1) / kTile, tn = (N + kTile - 1) / kTile;
    int64_t best = 0;
    // shapes with at least one tile per SM take one split: only fewer matter
    for (int a = 1; a <= std::min(tm, ctx->num_sms); ++a)
        for (int b = 1; b <= tn && (sym || a * b < ctx->num_sms || (a == tm && b == tn)); ++b) {
            if (sym && a != b) continue;
            const int m = std::min(M, a * kTile), nn = std::min(N, b * kTile);
            const Plan q = plan(ctx, m, nn, Kp, sym);
            if (q.splits == 1 && !sym) continue;
            best = std::max(best, (int64_t)q.splits * m * nn);
        }
    return best;
}

void split_rows(const float *src, int64_t rows, int cols, int64_t ld, uint16_t *hi, uint16_t *lo,
                float *scale, cudaStream_t st) {
    if (rows <= 0) return;
    split_rows_kernel<<<(unsigned)ceil_div(rows, 8), 256, 0, st>>>(src, rows, cols, ld, pad64(cols), hi,
                                                                   lo, scale);
    ADAGIO_CHECK_LAUNCH();
}

void split_transpose_centred(const float *X, int64_t n, int cols, int64_t ldx, const float *mu,
                             const unsigned *amax_bits, uint16_t *hi, uint16_t *lo, float *scale,
                             cudaStream_t st) {
    const int Kp = pad64(n);
    dim3 grid((unsigned)ceil_div(cols, 32), (unsigned)std::min<int64_t>(ceil_div(Kp, 32), 65535));
    split_transpose_kernel<<<grid, dim3(32, 8), 0, st>>>(X, n, cols, ldx, mu, amax_bits, Kp, hi, lo, scale);
    ADAGIO_CHECK_LAUNCH();
}

void tc_gemm(adagio_ctx *ctx, const SplitPlanes &A, const SplitPlanes &B, int M, int N,
             const float *bias, float *C, int64_t ldc, bool sym, float *part, int *status,
             cudaStream_t st) {
    if (M <= 0 || N <= 0) return;
    if (A.Kp != B.Kp || A.Kp % kKStep != 0 || A.bf16 != B.bf16)
        fail(ADAGIO_E_CUDA, "internal: GEMM planes disagree (K %d / %d)", A.Kp, B.Kp);
    const Plan q = plan(ctx, M, N, A.Kp, sym);
    GemmArgs a;
    a.M = M;
    a.N = N;
    a.tiles_n = q.tiles_n;
    a.tiles = q.tiles_m * q.tiles_n;
    a.items = (long long)a.tiles * q.splits;
    a.ksteps = q.ksteps;
    a.ksplit = q.ksplit;
    a.sym = sym ? 1 : 0;
    a.sa = A.scale;
    a.sb = B.scale;
    a.sa_stride = A.scale_stride;
    a.sb_stride = B.scale_stride;
    const bool direct = q.splits == 1 && !sym;
    a.bias = direct ? bias : nullptr;
    a.out = direct ? C : part;
    a.ldo = direct ? ldc : N;
    a.split_stride = (int64_t)M * N;
    const uint32_t fmt = A.bf16 ? 1u : 0u;
    a.idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(kTile >> 3) << 17) |
              ((uint32_t)(kTile >> 4) << 24);
    a.status = status;
    const CUtensorMap mah = plane_map(A.hi, A.rows, A.Kp, kKStep, kTile, A.bf16);
    const CUtensorMap mal = plane_map(A.lo, A.rows, A.Kp, kKStep, kTile, A.bf16);
    const CUtensorMap mbh = plane_map(B.hi, B.rows, B.Kp, kKStep, kTile, B.bf16);
    const CUtensorMap mbl = plane_map(B.lo, B.rows, B.Kp, kKStep, kTile, B.bf16);
    tc_gemm_init();
    // persistent: at most one CTA per SM (the shared memory holds one)
    const unsigned grid = (unsigned)std::min<long long>(a.items, ctx->num_sms);
    tc_gemm_kernel<<<grid, kThreads, kSmem, st>>>(mah, mal, mbh, mbl, a);
    ADAGIO_CHECK_LAUNCH();
    if (!direct) {
        const int64_t total = (int64_t)M * N;
        tc_gemm_reduce<<<(unsigned)ceil_div(total, 256), 256, 0, st>>>(part, q.splits, a.split_stride, M, N,
                                                                      N, bias, a.sym, C, ldc);
        ADAGIO_CHECK_LAUNCH();
    }
}

size_t embed_tc_bytes(adagio_ctx *ctx, int64_t n, int m, int d) {
    const int Kd = pad64(d);
    size_t b = 2 * align_up((size_t)m * Kd * sizeof(uint16_t), 256);
    b += 2 * align_up((size_t)m * sizeof(float), 256);
    b += align_up((size_t)std::max<int64_t>(1, tc_gemm_workspace(ctx, (int)std::min<int64_t>(n, 1 << 30), m, Kd, false)) *
                      sizeof(float), 256);
    return b + 256;
}

void embed_tc(adagio_ctx *ctx, const SplitPlanes &Xp, int64_t n, const float *mu, const float *A, int m,
              int d, int64_t lda, float *Y, int64_t ldy, void *scratch, cudaStream_t st) {
    const int Kd = pad64(d);
    if (Xp.bf16 || Xp.Kp != Kd || n > (1ll << 30))
        fail(ADAGIO_E_CUDA, "internal: tensor embedding needs FP16 planes with K = %d", Kd);
    char *p = reinterpret_cast<char *>(scratch);
    auto carve = [&](size_t bytes) {
        char *q = p;
        p += align_up(bytes, 256);
        return q;
    };
    SplitPlanes Ap;
    uint16_t *ah = reinterpret_cast<uint16_t *>(carve((size_t)m * Kd * sizeof(uint16_t)));
    uint16_t *al = reinterpret_cast<uint16_t *>(carve((size_t)m * Kd * sizeof(uint16_t)));
    float *as = reinterpret_cast<float *>(carve((size_t)m * sizeof(float)));
    float *bias = reinterpret_cast<float *>(carve((size_t)m * sizeof(float)));
    float *part = reinterpret_cast<float *>(p);
    split_rows(A, m, d, lda, ah, al, as, st);
    Ap.hi = ah;
    Ap.lo = al;
    Ap.rows = m;
    Ap.Kp = Kd;
    Ap.scale = as;
    Ap.scale_stride = 1;
    if (mu) {
        rows_dot_kernel<<<(unsigned)ceil_div(m, 8), 256, 0, st>>>(A, m, d, lda, mu, bias);
        ADAGIO_CHECK_LAUNCH();
    }
    tc_gemm(ctx, Xp, Ap, (int)n, m, mu ? bias : nullptr, Y, ldy, false, part, ctx->dev_status, st);
}

}  // namespace adagio
