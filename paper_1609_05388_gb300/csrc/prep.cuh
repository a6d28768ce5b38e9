// Prepared (centred, padded, split) point matrix shared by the certificate
// tile kernels.
#pragma once

#include "internal.cuh"
#include "cert_common.cuh"

namespace adagio {

constexpr int kTileRows = 128;  // tile height of the certificate kernels
constexpr int kRowPad = 256;    // row padding of every prepared matrix (two tile heights)

inline int64_t pad_rows(int64_t n) { return (n + kRowPad - 1) / kRowPad * kRowPad; }

struct PrepMat {
    int64_t n = 0, n_pad = 0;
    int K = 0, Kp32 = 0, Kp16 = 0;
    float *mu = nullptr;        // [K]
    RowStat *rs = nullptr;      // [n_pad]
    float *c32 = nullptr;       // [n_pad][Kp32] centred FP32
    uint16_t *hi = nullptr;     // [n_pad][Kp16] split plane, high part
    uint16_t *lo = nullptr;     // [n_pad][Kp16] split plane, low part
    float *scale = nullptr;     // device scalar: power-of-two split scale
    unsigned *amax = nullptr;   // device: max |x - mu| as float bits
    BoundModel bm{};
};

// Enqueues K0 for one matrix.  Allocates from the context workspace (the
// caller must have reserved enough).  `flags` (device) gets bit 0 on a
// non-finite input.
void prep_matrix(adagio_ctx *ctx, const float *X, int64_t n, int K, int64_t ld, int precision,
                 bool want_c32, bool want_split, PrepMat &pm, unsigned *flags, cudaStream_t st);

// Workspace bytes prep_matrix needs.
inline size_t prep_bytes(int64_t n, int K, bool want_c32, bool want_split) {
    int64_t n_pad = pad_rows(n);
    size_t Kp32 = align_up((size_t)K, 8), Kp16 = align_up((size_t)K, 64);
    size_t b = 0;
    b += align_up(K * sizeof(float), 256);
    b += align_up(n_pad * sizeof(RowStat), 256);
    if (want_c32) b += align_up(n_pad * Kp32 * sizeof(float), 256);
    if (want_split) b += 2 * align_up(n_pad * Kp16 * sizeof(uint16_t), 256);
    b += 2 * 256;
    b += align_up(((n + 2047) / 2048) * (size_t)K * sizeof(double), 256);
    return b + 1024;
}

}  // namespace adagio
