// Context, workspace arena, status handling and host/device pointer staging.
#include "internal.cuh"
#include "linalg.cuh"

#include <atomic>
#include <cstring>
#include <map>
#include <mutex>

namespace adagio {

static std::atomic<uint64_t> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

void fail(int code, const char *fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    throw Error{code, std::string(buf)};
}

void ws_reset(adagio_ctx *ctx) { ctx->ws.off = 0; }

void set_max_dyn_smem(const void *fn, int bytes) {
    static std::mutex mu;
    static std::map<std::pair<const void *, int>, int> done;
    int dev = 0;
    ADAGIO_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(mu);
    int &have = done[{fn, dev}];
    if (have >= bytes) return;
    ADAGIO_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    have = bytes;
}

void ws_reserve(adagio_ctx *ctx, size_t bytes) {
    Workspace &w = ctx->ws;
    bytes = align_up(bytes, 1 << 20);
    if (w.limit && bytes > w.limit)
        fail(ADAGIO_E_WORKSPACE, "workspace of %zu bytes needed, limit is %zu", bytes, w.limit);
    if (bytes <= w.cap) return;
    if (w.base) {
        // the old buffer may still be in use by enqueued work
        ADAGIO_CUDA(cudaDeviceSynchronize());
        ADAGIO_CUDA(cudaFree(w.base));
        w.base = nullptr;
        w.cap = 0;
    }
    cudaError_t e = cudaMalloc(&w.base, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        w.base = nullptr;
        fail(ADAGIO_E_WORKSPACE, "cudaMalloc of %zu workspace bytes failed: %s", bytes,
             cudaGetErrorString(e));
    }
    w.cap = bytes;
}

void *ws_alloc(adagio_ctx *ctx, size_t bytes, size_t align) {
    Workspace &w = ctx->ws;
    size_t off = align_up(w.off, align);
    if (off + bytes > w.cap)
        fail(ADAGIO_E_WORKSPACE, "internal: workspace carve of %zu bytes exceeds reservation (%zu of %zu used)",
             bytes, off, w.cap);
    w.off = off + bytes;
    return w.base + off;
}

void *host_stage(adagio_ctx *ctx, size_t bytes) {
    if (bytes > ctx->host_stage_bytes) {
        if (ctx->host_stage) cudaFreeHost(ctx->host_stage);
        ctx->host_stage = nullptr;
        ctx->host_stage_bytes = 0;
        ADAGIO_CUDA(cudaMallocHost(&ctx->host_stage, bytes));
        ctx->host_stage_bytes = bytes;
    }
    return ctx->host_stage;
}

bool is_device_ptr(const void *p, int device) {
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) {
        if (a.type == cudaMemoryTypeDevice && a.device != device)
            fail(ADAGIO_E_INVALID_ARG, "device pointer %p lives on device %d, context is on %d", p,
                 a.device, device);
        return true;
    }
    return false;
}

void check_device_status(adagio_ctx *ctx, cudaStream_t st) {
    ADAGIO_CUDA(cudaStreamSynchronize(st));
    int h = 0;
    ADAGIO_CUDA(cudaMemcpy(&h, ctx->dev_status, sizeof(int), cudaMemcpyDeviceToHost));
    if (h != 0) {
        ADAGIO_CUDA(cudaMemset(ctx->dev_status, 0, sizeof(int)));
        fail(ADAGIO_E_TIMEOUT, "tensor-core GEMM gave up a bounded wait (status %d)", h);
    }
}

static bool rows_aligned(const float *p, int64_t ld) {
    return reinterpret_cast<uintptr_t>(p) % 16 == 0 && ld % 4 == 0;
}

size_t stage_aligned_bytes(adagio_ctx *ctx, const float *p, int64_t rows, int cols, int64_t ld) {
    const size_t padded = align_up((size_t)rows * emb_ld(cols) * sizeof(float), 256);
    if (is_device_ptr(p, ctx->device)) return rows_aligned(p, ld) ? 0 : padded;
    const size_t linear = align_up((size_t)rows * cols * sizeof(float), 256);
    return linear + (cols % 4 == 0 ? 0 : padded);
}

const float *stage_aligned(adagio_ctx *ctx, const float *p, int64_t rows, int cols, int64_t ld,
                           int64_t *ld_out, cudaStream_t st) {
    const float *src = p;
    int64_t lds = ld;
    if (!is_device_ptr(p, ctx->device)) {
        src = stage_input(ctx, p, rows, cols, ld, &lds, st);  // linear, stride cols
    } else if (rows_aligned(p, ld)) {
        *ld_out = ld;
        return p;
    }
    if (rows_aligned(src, lds)) {
        *ld_out = lds;
        return src;
    }
    const int ldp = emb_ld(cols);
    float *d = ws_array<float>(ctx, (size_t)rows * ldp);
    copy_rows(src, lds, d, ldp, (int)rows, cols, st);
    *ld_out = ldp;
    return d;
}

cudaStream_t side_stream(adagio_ctx *ctx) {
    if (!ctx->side_stream) {
        ADAGIO_CUDA(cudaStreamCreateWithFlags(&ctx->side_stream, cudaStreamNonBlocking));
        for (cudaEvent_t &e : ctx->side_ev) ADAGIO_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    }
    return ctx->side_stream;
}

const float *stage_input(adagio_ctx *ctx, const float *p, int64_t rows, int cols, int64_t ld,
                         int64_t *ld_out, cudaStream_t st) {
    if (is_device_ptr(p, ctx->device)) {
        *ld_out = ld;
        return p;
    }
    float *d = ws_array<float>(ctx, (size_t)rows * cols);
    // contiguous rows: one linear copy (a pitched copy of many short rows
    // moves far slower over the host link)
    if (ld == cols)
        ADAGIO_CUDA(cudaMemcpyAsync(d, p, (size_t)rows * cols * sizeof(float), cudaMemcpyHostToDevice, st));
    else
        ADAGIO_CUDA(cudaMemcpy2DAsync(d, (size_t)cols * sizeof(float), p, (size_t)ld * sizeof(float),
                                      (size_t)cols * sizeof(float), (size_t)rows,
                                      cudaMemcpyHostToDevice, st));
    *ld_out = cols;
    return d;
}

}  // namespace adagio

using namespace adagio;

static thread_local std::string g_create_error;

extern "C" {

void adagio_default_fit_opts(adagio_fit_opts *o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->eps = 0.1;
    o->m = 0;
    o->s = -1;
    o->seed = 0;
    o->jl_dist = ADAGIO_JL_RADEMACHER;
    o->precision = ADAGIO_PREC_FP16X3;
    o->use_predictor = 0;
    o->hist_lo = 0.0;
    o->hist_hi = 0.0;
    o->max_iter = 100;
    o->tol = 1e-6;
    o->oversample = 32;
}

int adagio_ctx_create(int device, size_t workspace_limit, adagio_ctx **out) {
    if (!out) return ADAGIO_E_INVALID_ARG;
    *out = nullptr;
    try {
        int count = 0;
        ADAGIO_CUDA(cudaGetDeviceCount(&count));
        if (device < 0 || device >= count)
            fail(ADAGIO_E_INVALID_ARG, "device %d out of range (%d devices)", device, count);
        cudaDeviceProp prop;
        ADAGIO_CUDA(cudaGetDeviceProperties(&prop, device));
        if (!(prop.major == 10 && prop.minor == 3))
            fail(ADAGIO_E_UNSUPPORTED, "device %d is sm_%d%d; this library is built for sm_103a",
                 device, prop.major, prop.minor);
        DeviceGuard g(device);
        ADAGIO_CUDA(cudaFree(nullptr));  // make sure the primary context exists
        int *status = nullptr;
        ADAGIO_CUDA(cudaMalloc(&status, 256));
        cudaError_t e = cudaMemset(status, 0, 256);
        if (e != cudaSuccess) {
            cudaFree(status);
            ADAGIO_CUDA(e);
        }
        adagio_ctx *ctx = new adagio_ctx();
        ctx->device = device;
        ctx->num_sms = prop.multiProcessorCount;
        ctx->ws.limit = workspace_limit;
        ctx->dev_status = status;
        ctx->device_name = prop.name;
        *out = ctx;
        return ADAGIO_OK;
    } catch (const Error &e) {
        g_create_error = e.msg;
        return e.code;
    } catch (...) {
        g_create_error = "unknown failure";
        return ADAGIO_E_CUDA;
    }
}


int adagio_ctx_destroy(adagio_ctx *ctx) {
    if (!ctx) return ADAGIO_OK;
    {
        int prev = -1;
        cudaGetDevice(&prev);
        cudaSetDevice(ctx->device);
        cudaDeviceSynchronize();
        free_predictor(ctx);
        if (ctx->ws.base) cudaFree(ctx->ws.base);
        if (ctx->qbuf && !ctx->qbuf_fixed) cudaFree(ctx->qbuf);
        if (ctx->host_stage) cudaFreeHost(ctx->host_stage);
        for (auto &e : ctx->tc_sched) cudaFree(e.second);
        for (cudaStream_t s : ctx->batch_streams) cudaStreamDestroy(s);
        if (ctx->side_stream) cudaStreamDestroy(ctx->side_stream);
        for (cudaEvent_t e : ctx->side_ev)
            if (e) cudaEventDestroy(e);
        if (ctx->batch_host) cudaFreeHost(ctx->batch_host);
        if (ctx->dev_status) cudaFree(ctx->dev_status);
        if (prev >= 0) cudaSetDevice(prev);
    }
    delete ctx;
    return ADAGIO_OK;
}

const char *adagio_last_error(const adagio_ctx *ctx) {
    if (!ctx) return g_create_error.c_str();
    return ctx->last_error.c_str();
}

size_t adagio_workspace_bytes(const adagio_ctx *ctx) { return ctx ? ctx->ws.cap : 0; }

int adagio_set_timing(adagio_ctx *ctx, int enable) {
    if (!ctx) return ADAGIO_E_INVALID_ARG;
    ctx->collect_timing = enable ? 1 : 0;
    return ADAGIO_OK;
}

int adagio_set_tile_kernel(adagio_ctx *ctx, int variant, int band) {
    if (!ctx || variant < ADAGIO_TILES_AUTO || variant > ADAGIO_TILES_PAIR || band < 0 || band > 64)
        return ADAGIO_E_INVALID_ARG;
    ctx->tc_variant = variant;
    ctx->tc_band = band;
    return ADAGIO_OK;
}

int adagio_last_cert_stats(const adagio_ctx *ctx, adagio_cert_stats *out) {
    if (!ctx || !out) return ADAGIO_E_INVALID_ARG;
    *out = ctx->last_stats;
    return ADAGIO_OK;
}

int adagio_last_batch_stats(const adagio_ctx *ctx, adagio_batch_stats *out) {
    if (!ctx || !out) return ADAGIO_E_INVALID_ARG;
    *out = ctx->last_batch;
    return ADAGIO_OK;
}

int adagio_last_fit_stats(const adagio_ctx *ctx, adagio_fit_stats *out) {
    if (!ctx || !out) return ADAGIO_E_INVALID_ARG;
    *out = ctx->last_fit;
    return ADAGIO_OK;
}

uint64_t adagio_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

}  // extern "C"
