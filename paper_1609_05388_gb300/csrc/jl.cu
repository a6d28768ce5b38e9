// JL matrix S of Algorithm 1 (entries +-1/sqrt(k), Lemma 2) and the random
// start block of the randomized subspace iteration.
//
// Random bits: SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) used as a
// counter-based generator.  Output number c of the stream seeded with `seed`
// mixes seed + (c + 1) * 0x9E3779B97F4A7C15 through two xor-shift-multiply
// rounds.  Entry (i, j) of S takes output c = i*2^32 + 2j (and c + 1 for the
// second uniform of the Gaussian option), so row i does not depend on k.
#include "internal.cuh"
#include "jl.cuh"
#include "rng.cuh"

namespace adagio {

namespace {

__global__ void jl_kernel(uint64_t seed, int k, int d, int dist, float scale, float *__restrict__ S,
                          int64_t lds) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)k * d) return;
    const uint64_t i = (uint64_t)(e / d), j = (uint64_t)(e % d);
    const uint64_t c = (i << 32) | (j << 1);
    const uint64_t z0 = splitmix64_out(seed, c);
    float v;
    if (dist == ADAGIO_JL_GAUSSIAN) {
        const uint64_t z1 = splitmix64_out(seed, c | 1ull);
        const double u1 = ((double)(z0 >> 11) + 0.5) * 0x1.0p-53;
        const double u2 = ((double)(z1 >> 11) + 0.5) * 0x1.0p-53;
        v = (float)(sqrt(-2.0 * log(u1)) * cospi(2.0 * u2)) * scale;
    } else {
        v = (z0 >> 63) ? -scale : scale;
    }
    S[(int64_t)i * lds + j] = v;
}

}  // namespace

void jl_matrix(uint64_t seed, int k, int d, int dist, float *S, int64_t lds, cudaStream_t st) {
    if (k <= 0) return;
    const float scale = (float)(1.0 / sqrt((double)k));
    const int64_t total = (int64_t)k * d;
    jl_kernel<<<(unsigned)ceil_div(total, 256), 256, 0, st>>>(seed, k, d, dist, scale, S, lds);
    ADAGIO_CHECK_LAUNCH();
}

void rademacher_block(uint64_t seed, int rows, int d, float *V, int64_t ldv, cudaStream_t st) {
    // +-1 entries (scale 1); a seed stream distinct from the JL matrix
    const uint64_t s2 = seed ^ 0x5DEECE66DA3B2C1Full;
    const int64_t total = (int64_t)rows * d;
    if (total <= 0) return;
    jl_kernel<<<(unsigned)ceil_div(total, 256), 256, 0, st>>>(s2, rows, d, ADAGIO_JL_RADEMACHER,
                                                              1.0f, V, ldv);
    ADAGIO_CHECK_LAUNCH();
}

}  // namespace adagio
