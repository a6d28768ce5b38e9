#pragma once

#include "internal.cuh"

namespace adagio {

// S (k x d, row-major, leading dimension lds): Algorithm 1's JL matrix.
void jl_matrix(uint64_t seed, int k, int d, int dist, float *S, int64_t lds, cudaStream_t st);
// rows x d block of +-1 entries (start block of the subspace iteration).
void rademacher_block(uint64_t seed, int rows, int d, float *V, int64_t ldv, cudaStream_t st);

}  // namespace adagio
