// Internal runtime of the ADAGIO library: context, workspace arena, status
// handling and the launch helpers shared by every translation unit.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <cstdarg>
#include <cstdio>
#include <map>
#include <string>
#include <vector>

#include "adagio.h"

namespace adagio {

constexpr int kBins = ADAGIO_HIST_BINS;

// Thrown only inside the library; every C entry point catches it and turns it
// into a status code, so nothing crosses the ABI.
struct Error {
    int code;
    std::string msg;
};

[[noreturn]] void fail(int code, const char *fmt, ...);

#define ADAGIO_CUDA(call)                                                          \
    do {                                                                           \
        cudaError_t e_ = (call);                                                   \
        if (e_ != cudaSuccess)                                                     \
            ::adagio::fail(ADAGIO_E_CUDA, "%s failed: %s (%s:%d)", #call,          \
                           cudaGetErrorString(e_), __FILE__, __LINE__);            \
    } while (0)

// Every kernel launch is followed by this check; it also counts launches.
void count_launch();
#define ADAGIO_CHECK_LAUNCH()                 \
    do {                                      \
        ::adagio::count_launch();             \
        ADAGIO_CUDA(cudaGetLastError());      \
    } while (0)

#define ADAGIO_REQUIRE(cond, ...)                                                  \
    do {                                                                           \
        if (!(cond)) ::adagio::fail(ADAGIO_E_INVALID_ARG, __VA_ARGS__);            \
    } while (0)

// Device workspace: one growable buffer, carved per call by a bump pointer.
// Growth frees the old buffer after synchronising the device, so a call must
// reserve its whole need before launching anything that uses it.
struct Workspace {
    char *base = nullptr;
    size_t cap = 0;
    size_t off = 0;
    size_t limit = 0;  // 0 = unlimited
};

struct Predictor;  // dimension predictor (mlp.cu)

// Tile configuration of the tensor-core certificate: the kernel (1 = one CTA
// per tile, 2 = CTA pairs) and the schedule's band height in tile rows.
struct TileConfig {
    int variant;
    int band;
};

// An autotuned configuration and the tile-kernel time it was measured at.
struct TunedTiles {
    int variant, band;
    double ms;
};

}  // namespace adagio

struct adagio_ctx {
    int device = 0;
    int num_sms = 0;
    adagio::Workspace ws;
    std::string last_error;
    // pinned host staging for small device->host results
    void *host_stage = nullptr;
    size_t host_stage_bytes = 0;
    // recompute queue of the certificate: context-owned, grown on demand
    // (qbuf_fixed: an external buffer that must not be replaced)
    int2 *qbuf = nullptr;
    unsigned long long qbuf_cap = 0;
    bool qbuf_fixed = false;
    adagio::Predictor *predictor = nullptr;
    // statistics of the most recent certificate (for diagnostics)
    adagio_cert_stats last_stats{-1.0, -1.0, -1.0, 0, 0, 0};
    adagio_fit_stats last_fit{0, 0, 0, 0, 0.0, 0.0, 0};
    int collect_timing = 0;
    // tile schedules of the tensor-core certificate, by tile-row count T
    // (built once, resident for the context's lifetime)
    std::map<int, uint32_t *> tc_sched;
    // tile kernel of the tensor-core certificate: 0 automatic, 1 one CTA per
    // tile, 2 CTA pairs; and how many CTA pairs fit at once (-1: not queried)
    int tc_variant = 0;
    int tc_band = 0;  // schedule band height in tile rows (0: tuned or default)
    int tc_pair_clusters = -1;
    // autotuned tile configurations by size class of n (adagio_autotune_tiles)
    std::map<int, adagio::TunedTiles> tc_tuned;
    std::string device_name;
    // device status word of the tensor-core GEMMs (nonzero: a bounded wait
    // gave up); checked and cleared by the calls that synchronise
    int *dev_status = nullptr;
    // a side stream and two events for work that overlaps the caller's
    // stream (created on first use)
    cudaStream_t side_stream = nullptr;
    cudaEvent_t side_ev[2] = {nullptr, nullptr};
    // streams and pinned host memory of batched fits (grown on demand)
    std::vector<cudaStream_t> batch_streams;
    void *batch_host = nullptr;
    size_t batch_host_bytes = 0;
    adagio_batch_stats last_batch{0, 0, 0, 0.0};
    // query rows of the last adagio_knn searched again over every base point
    int64_t last_knn_redo = 0;
};

namespace adagio {

// RAII device selection for the duration of an entry point.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) ADAGIO_CUDA(cudaSetDevice(dev));
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

// Workspace management -------------------------------------------------------
void ws_reset(adagio_ctx *ctx);
// raises a kernel's dynamic shared-memory limit to at least `bytes` on the
// current device (a no-op once done), so that launches need no attribute call
void set_max_dyn_smem(const void *fn, int bytes);
void ws_reserve(adagio_ctx *ctx, size_t bytes);           // capacity >= bytes
void *ws_alloc(adagio_ctx *ctx, size_t bytes, size_t align = 256);
template <typename T>
T *ws_array(adagio_ctx *ctx, size_t count) {
    return reinterpret_cast<T *>(ws_alloc(ctx, count * sizeof(T)));
}
void *host_stage(adagio_ctx *ctx, size_t bytes);

inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }
inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
// Row stride of an internal n x m embedding: a multiple of 4 floats, so the
// recompute reads its rows with 16-byte loads.
inline int emb_ld(int m) { return (int)align_up((size_t)(m < 1 ? 1 : m), 4); }

// Pointer kinds ----------------------------------------------------------------
bool is_device_ptr(const void *p, int device);

// Input staging: returns a device pointer to a row-major n x cols matrix with
// leading dimension *ld_out.  Host input is copied into the workspace.
const float *stage_input(adagio_ctx *ctx, const float *p, int64_t rows, int cols, int64_t ld,
                         int64_t *ld_out, cudaStream_t st);

// Error-bound constants of the pair distortion for one Gram arithmetic (see
// cert_common.cuh).
struct BoundModel {
    float c4;    // statistical product-error coefficient (times ||a||_4 ||b||_4)
    float cacc;  // accumulation coefficient (times ||a||_2 ||b||_2)
};
BoundModel bound_model(int precision, int K);

// Synchronises st and fails with ADAGIO_E_TIMEOUT (clearing the word) when a
// tensor-core GEMM enqueued on the context recorded a timeout.
void check_device_status(adagio_ctx *ctx, cudaStream_t st);
// The context's side stream (created on first use, with its two events).
cudaStream_t side_stream(adagio_ctx *ctx);
// A device copy of a rows x cols FP32 matrix whose rows start 16-byte aligned
// (base aligned, row stride a multiple of 4 floats), for kernels that read
// whole rows with 16-byte loads: aligned device data is used in place; host
// data is copied linearly and, when cols is not a multiple of 4, re-pitched
// on the device; unaligned device data is re-pitched.  *ld_out receives the
// stride; stage_aligned_bytes is the workspace it takes.
const float *stage_aligned(adagio_ctx *ctx, const float *p, int64_t rows, int cols, int64_t ld,
                           int64_t *ld_out, cudaStream_t st);
size_t stage_aligned_bytes(adagio_ctx *ctx, const float *p, int64_t rows, int cols, int64_t ld);

// Releases the dimension predictor held by a context (mlp.cu).
void free_predictor(adagio_ctx *ctx);

}  // namespace adagio
