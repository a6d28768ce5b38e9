// Allocation-free certificate entry point (the paper has no counterpart).
//
// Some callers cannot let a library allocate device memory during a call: a
// service that hands all device memory to its own pool at start-up (a
// cudaMalloc then fails or fragments the pool), or a latency-critical loop
// that cannot afford the implicit device synchronisation of cudaMalloc and
// cudaFree.  adagio_distortion_noalloc serves them for small problems: it runs
// the FP32 certificate (K0 prep, SIMT tiles, recompute, finaliser)
// entirely inside a fixed scratch area that is a file-scope __device__ array
// of this library, instead of the context workspace.
//
//  * Scratch: kScratchBytes (8 MiB) of static device memory.  Every GPU that
//    loads the library holds it until the process exits.
//  * Limits: n <= 1024 points, d <= 512, m <= 256.  Larger inputs are
//    rejected with ADAGIO_E_INVALID_ARG before any work is enqueued.  The
//    kernels run on at most kMaxCtaSms SMs' worth of CTAs (their per-CTA
//    partial records live in the scratch too), so the limits hold on a GPU
//    of any SM count.
//  * Set-up: the first call on a device looks up the array's device address
//    with cudaGetSymbolAddress (the host-side name of the array is only a
//    stand-in, not a device address) with that device current, and caches it.
//    Make that first call before capturing any stream on that device.
//  * Sharing: all calls share the one array and it keeps the previous call's
//    contents; every counter, flag and partial that must start at zero is
//    cleared on the stream at the start of each call.  Calls that overlapped
//    on the GPU would race on the array, so this entry point serialises its
//    callers with a host lock and synchronises the stream before returning,
//    also when it fails after enqueuing work.
//  * The certificate statistics of the call (adagio_last_cert_stats) are
//    those of the context passed in.
//  * It calls no cudaMalloc, cudaFree or allocating library routine: the
//    result is copied into a static host buffer and then into *out.
#include "internal.cuh"
#include "cert.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

namespace adagio {

namespace {

constexpr size_t kScratchBytes = 8u << 20;
constexpr int64_t kMaxN = 1024;
constexpr int kMaxD = 512;
constexpr int kMaxM = 256;
// the recompute queue can hold every pair of the largest allowed problem
constexpr unsigned long long kQueueEntries = (unsigned long long)kMaxN * (kMaxN - 1) / 2;
constexpr size_t kQueueBytes = kQueueEntries * sizeof(int2);
constexpr int kMaxDevices = 256;
// SMs whose CTAs the call uses at most: the FP32 tile kernel runs one CTA per
// SM and the recompute three, each with a partial record in the scratch
constexpr int kMaxCtaSms = 160;

__device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;
void *g_scratch_addr[kMaxDevices] = {};
alignas(256) unsigned char g_host_result[4096];

void *scratch_address(int device) {
    if (device < 0 || device >= kMaxDevices) fail(ADAGIO_E_INVALID_ARG, "device %d out of range", device);
    if (!g_scratch_addr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            fail(ADAGIO_E_CUDA, "cudaGetSymbolAddress of the scratch array failed: %s",
                 cudaGetErrorString(e));
        }
        g_scratch_addr[device] = p;
    }
    return g_scratch_addr[device];
}

}  // namespace

}  // namespace adagio

using namespace adagio;

extern "C" int adagio_distortion_noalloc(adagio_ctx *ctx, const float *X, int64_t n, int d,
                                         int64_t ldx, const float *Y, int m, int64_t ldy, double eps,
                                         double hist_lo, double hist_hi, adagio_cert *out,
                                         void *stream) {
    if (!ctx) return ADAGIO_E_INVALID_ARG;
    ctx->last_error.clear();
    try {
        DeviceGuard guard(ctx->device);
        ADAGIO_REQUIRE(X && Y && out, "null pointer argument");
        ADAGIO_REQUIRE(n >= 2 && n <= kMaxN, "n = %lld outside [2, %lld] (allocation-free limit)",
                       (long long)n, (long long)kMaxN);
        ADAGIO_REQUIRE(d >= 1 && d <= kMaxD && m >= 1 && m <= kMaxM,
                       "d = %d, m = %d outside the allocation-free limits d <= %d, m <= %d", d, m,
                       kMaxD, kMaxM);
        ADAGIO_REQUIRE(ldx >= d && ldy >= m, "leading dimensions too small");
        ADAGIO_REQUIRE(is_device_ptr(X, ctx->device) && is_device_ptr(Y, ctx->device),
                       "X and Y must be device pointers on the context's device");
        ADAGIO_REQUIRE(std::isfinite(eps) && eps > 0.0 && eps < 1.0, "eps must lie in (0, 1), got %g", eps);
        if (!(hist_hi > hist_lo)) {
            hist_lo = 0.0;
            hist_hi = 2.0 * eps;
        }
        ADAGIO_REQUIRE(std::isfinite(hist_lo) && std::isfinite(hist_hi) && hist_lo >= 0.0,
                       "bad histogram range");
        std::lock_guard<std::mutex> lock(g_mu);
        char *base = static_cast<char *>(scratch_address(ctx->device));
        // a context view: workspace and recompute queue are slices of the
        // static scratch, result staging is a static host buffer
        adagio_ctx view;
        view.device = ctx->device;
        view.num_sms = std::min(ctx->num_sms, kMaxCtaSms);
        view.qbuf = reinterpret_cast<int2 *>(base);
        view.qbuf_cap = kQueueEntries;
        view.qbuf_fixed = true;
        view.ws.base = base + align_up(kQueueBytes, 256);
        view.ws.cap = kScratchBytes - align_up(kQueueBytes, 256);
        view.ws.off = 0;
        view.ws.limit = 0;
        view.host_stage = g_host_result;
        view.host_stage_bytes = sizeof(g_host_result);
        const size_t need = certify_bytes(&view, n, d, m, ADAGIO_PREC_FP32);
        ADAGIO_REQUIRE(need <= view.ws.cap, "problem needs %zu scratch bytes, %zu available", need,
                       view.ws.cap);
        CertOptions co;
        co.eps = eps;
        co.lo = hist_lo;
        co.hi = hist_hi;
        co.precision = ADAGIO_PREC_FP32;
        int rc = ADAGIO_OK;
        try {
            rc = certify(&view, X, ldx, Y, ldy, n, d, m, co, out, (cudaStream_t)stream);
        } catch (...) {
            // work may still be queued on the stream: the scratch stays
            // locked until the GPU is done with it
            cudaStreamSynchronize((cudaStream_t)stream);
            cudaGetLastError();
            view.qbuf = nullptr;
            view.host_stage = nullptr;
            view.ws.base = nullptr;
            throw;
        }
        ctx->last_stats = view.last_stats;
        // the view owns none of these buffers
        view.qbuf = nullptr;
        view.host_stage = nullptr;
        view.ws.base = nullptr;
        return rc;
    } catch (const Error &e) {
        ctx->last_error = e.msg;
        return e.code;
    } catch (...) {
        ctx->last_error = "unknown failure";
        return ADAGIO_E_CUDA;
    }
}
