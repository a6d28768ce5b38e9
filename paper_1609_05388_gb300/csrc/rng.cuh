// SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) as a counter-based generator:
// output number c of the stream seeded with `seed` mixes seed + (c+1)*gamma
// through two xor-shift-multiply rounds.
#pragma once

#include <stdint.h>

namespace adagio {

__device__ __forceinline__ uint64_t splitmix64_out(uint64_t seed, uint64_t c) {
    uint64_t z = seed + (c + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

}  // namespace adagio
