// K8 (plain FP32 path): all-pairs distortion tiles on CUDA cores.
//
// Each CTA walks 128 x 128 tiles (I, J), I <= J, of the upper triangle of the
// pair matrix (Eq. 3 is a max over unordered pairs) in a persistent,
// round-robin loop.  For every tile it forms the two Gram tiles
// Gy = Yc[I] Yc[J]^T and Gx = Xc[I] Xc[J]^T in FP32 (128x128x8 smem stages,
// an 8 x 8 register block per thread), then classifies each pair with the
// shared epilogue (cert_common.cuh).  The n x n matrix is never stored.
#include "internal.cuh"
#include "cert_common.cuh"
#include "cert.cuh"

namespace adagio {

namespace {

constexpr int BM = 128, BK = 8, NT = 256, PADS = 4;

struct SimtArgs {
    const float *Xc;
    const float *Yc;
    int ldx, ldy;      // = Kp32 of each side (multiple of 8)
    int Kx, Ky;        // padded contraction lengths
    const RowStat *rsx, *rsy;
    int n, T;
    long long t_begin, ntp;  // tile pairs [t_begin, ntp) of the row-major triangle
    CertConst cc;
    CertPartial *partials;
    int2 *queue;
    unsigned long long *qcount, qcap;
    int *stop_flag;    // non-null: early exit on a certain violation
    float4 *dump;      // optional per-pair (dx2, dy2, ex, ey) of tile pairs t < dump_tiles
    long long dump_tiles;
    long long dump_stride;  // tile pairs t = q * dump_stride, q < dump_tiles, into slot q
};

// Chunk of the FP32 accumulation: FMA chains of kChunk terms, each added into
// the running sum.  A chain's rounding error is at most kChunk u times its sum
// of |a_k b_k|, the additions of the K / kChunk chunk sums at most K / kChunk u
// times the total, so the Gram entry is off by at most
// (kChunk + K / kChunk + 1) u sum |a_k b_k| <= (kChunk + K / kChunk + 1) u |a| |b|
// (Cauchy-Schwarz): a worst-case bound (bound_model, FP32).
constexpr int kChunk = 32;

// acc[a][b] = rows(I) . rows(J) over K for the thread's 8 x 4 block of column
// half H (the thread's columns tx * 4 + b + 64 H), summed in chunks of kChunk
// terms.  Two halves per tile keep the chunk sums within the register budget.
template <int H>
__device__ __forceinline__ void gram_tile_half(const float *__restrict__ M, int ld, int K, int rowI,
                                               int rowJ, float (*As)[BK][BM + PADS],
                                               float (*Bs)[BK][BM + PADS], float acc[8][4]) {
    static_assert(kChunk % BK == 0, "chunks of whole stages");
    const int tid = threadIdx.x;
    const int ty = tid >> 4, tx = tid & 15;
    const int lr = tid >> 1, lk = (tid & 1) * 4;
    float tmp[8][4];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = tmp[a][b] = 0.0f;
    const float *pa = M + (int64_t)(rowI + lr) * ld + lk;
    const float *pb = M + (int64_t)(rowJ + lr) * ld + lk;
    float4 ra = *reinterpret_cast<const float4 *>(pa);
    float4 rb = *reinterpret_cast<const float4 *>(pb);
    int buf = 0;
    for (int k0 = 0; k0 < K; k0 += BK) {
        As[buf][lk + 0][lr] = ra.x; As[buf][lk + 1][lr] = ra.y;
        As[buf][lk + 2][lr] = ra.z; As[buf][lk + 3][lr] = ra.w;
        Bs[buf][lk + 0][lr] = rb.x; Bs[buf][lk + 1][lr] = rb.y;
        Bs[buf][lk + 2][lr] = rb.z; Bs[buf][lk + 3][lr] = rb.w;
        __syncthreads();
        if (k0 + BK < K) {
            ra = *reinterpret_cast<const float4 *>(pa + k0 + BK);
            rb = *reinterpret_cast<const float4 *>(pb + k0 + BK);
        }
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            float4 a0 = *reinterpret_cast<const float4 *>(&As[buf][kk][ty * 4]);
            float4 a1 = *reinterpret_cast<const float4 *>(&As[buf][kk][64 + ty * 4]);
            float4 b0 = *reinterpret_cast<const float4 *>(&Bs[buf][kk][64 * H + tx * 4]);
            float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            float bv[4] = {b0.x, b0.y, b0.z, b0.w};
#pragma unroll
            for (int a = 0; a < 8; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) tmp[a][b] = fmaf(av[a], bv[b], tmp[a][b]);
        }
        if ((k0 + BK) % kChunk == 0 || k0 + BK >= K) {
#pragma unroll
            for (int a = 0; a < 8; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    acc[a][b] += tmp[a][b];
                    tmp[a][b] = 0.0f;
                }
        }
        buf ^= 1;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(NT, 1) cert_simt_kernel(SimtArgs p) {
    __shared__ __align__(16) float As[2][BK][BM + PADS];
    __shared__ __align__(16) float Bs[2][BK][BM + PADS];
    __shared__ RowStat sIx[BM], sIy[BM], sJx[BM], sJy[BM];
    extern __shared__ unsigned s_hist[];  // [kBins][NT]

    const int tid = threadIdx.x;
    const int ty = tid >> 4, tx = tid & 15;
    for (int b = 0; b < kBins; ++b) s_hist[b * NT + tid] = 0;

    unsigned long long npairs = 0, nviol = 0, nover = 0, nqueued = 0;
    double sum = 0.0, bsum = 0.0;
    float mx = -1.0f, mxb_all = 0.0f;
    int ai = 0x7fffffff, aj = 0x7fffffff;
    float gx[8][4], gy[8][4];

    __shared__ int s_stop;
    for (long long t = p.t_begin + blockIdx.x; t < p.ntp; t += gridDim.x) {
        // block-uniform early-exit decision; also orders the previous tile's
        // epilogue reads of the row statistics before they are overwritten
        __syncthreads();
        if (tid == 0) s_stop = p.stop_flag ? *(volatile int *)p.stop_flag : 0;
        __syncthreads();
        if (s_stop) break;
        int I, J;
        tri_index(t, p.T, I, J);
        const int rowI = I * BM, rowJ = J * BM;
        if (tid < BM) {
            sIx[tid] = p.rsx[rowI + tid];
            sIy[tid] = p.rsy[rowI + tid];
            sJx[tid] = p.rsx[rowJ + tid];
            sJy[tid] = p.rsy[rowJ + tid];
        }
        float tsum = 0.0f, tbsum = 0.0f;
        bool stop = false;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            // the tile's Grams for the thread's column half h
            if (h == 0) {
                gram_tile_half<0>(p.Yc, p.ldy, p.Ky, rowI, rowJ, As, Bs, gy);
                gram_tile_half<0>(p.Xc, p.ldx, p.Kx, rowI, rowJ, As, Bs, gx);
            } else {
                gram_tile_half<1>(p.Yc, p.ldy, p.Ky, rowI, rowJ, As, Bs, gy);
                gram_tile_half<1>(p.Xc, p.ldx, p.Kx, rowI, rowJ, As, Bs, gx);
            }
#pragma unroll
            for (int a = 0; a < 8; ++a) {
                const int li = ty * 4 + (a & 3) + (a >> 2) * 64;
                const int i = rowI + li;
                const RowStat xi = sIx[li], yi = sIy[li];
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    const int lj = tx * 4 + b + h * 64;
                    const int j = rowJ + lj;
                    FastPair fp;
                    int cls = PAIR_SKIP;
                    if (i < j && j < p.n) cls = classify_pair(gx[a][b], gy[a][b], xi, sJx[lj], yi, sJy[lj], p.cc, fp);
                    if (p.dump && t % p.dump_stride == 0 && t / p.dump_stride < p.dump_tiles) {
                        const RowStat xj = sJx[lj], yj = sJy[lj];
                        float4 v;
                        v.x = (xi.n2 + xj.n2) - 2.0f * gx[a][b];
                        v.y = (yi.n2 + yj.n2) - 2.0f * gy[a][b];
                        v.z = fmaf(xi.q4, xj.q4, fmaf(xi.q1, xj.q1, p.cc.c_r * (xi.n2 + xj.n2)));
                        v.w = fmaf(yi.q4, yj.q4, fmaf(yi.q1, yj.q1, p.cc.c_r * (yi.n2 + yj.n2)));
                        p.dump[((t / p.dump_stride) * BM + li) * BM + lj] = v;
                    }
                    queue_push(cls == PAIR_QUEUE, i, j, p.queue, p.qcount, p.qcap);
                    if (cls == PAIR_OK) {
                        ++npairs;
                        if (fp.bin >= 0) s_hist[fp.bin * NT + tid] += 1u; else ++nover;
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
        }
        sum += (double)tsum;
        bsum += (double)tbsum;
        if (p.stop_flag && stop) atomicExch(p.stop_flag, 1);
    }
    write_partial<NT>(p.partials + blockIdx.x, s_hist, npairs, nviol, nover, nqueued, 0ull, sum,
                      bsum, mx, mxb_all, ai, aj);
}

}  // namespace

void launch_cert_simt(const CertLaunch &L, cudaStream_t st) {
    SimtArgs p;
    p.Xc = L.x->c32; p.Yc = L.y->c32;
    p.ldx = L.x->Kp32; p.ldy = L.y->Kp32;
    p.Kx = L.x->Kp32; p.Ky = L.y->Kp32;
    p.rsx = L.x->rs; p.rsy = L.y->rs;
    p.n = (int)L.x->n;
    p.T = (int)(L.x->n_pad / BM);
    p.ntp = L.t_end >= 0 ? L.t_end : (long long)p.T * (p.T + 1) / 2;
    p.t_begin = L.t_end >= 0 ? L.t_begin : 0;
    p.cc = L.cc;
    p.partials = L.partials;
    p.queue = L.queue; p.qcount = L.qcount; p.qcap = L.qcap;
    p.stop_flag = L.stop_flag;
    p.dump = reinterpret_cast<float4 *>(L.dump);
    p.dump_tiles = L.dump_tiles;
    p.dump_stride = L.dump_stride > 0 ? L.dump_stride : 1;
    const size_t smem = (size_t)kBins * NT * sizeof(unsigned);
    set_max_dyn_smem((const void *)cert_simt_kernel, (int)smem);
    cert_simt_kernel<<<L.grid, NT, smem, st>>>(p);
    ADAGIO_CHECK_LAUNCH();
}

int cert_simt_threads() { return NT; }

void cert_simt_init() {
    set_max_dyn_smem((const void *)cert_simt_kernel, (int)((size_t)kBins * NT * sizeof(unsigned)));
}

}  // namespace adagio
