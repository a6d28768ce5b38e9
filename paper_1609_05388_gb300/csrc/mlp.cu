// Dimension predictor: a small network that maps spectrum features of a data
// set to the target dimension the certified search returns (the paper has no
// learned component; this is a serving-side accelerator of the search).
//
//   features  f[0..63] = 0.5 log(theta_i / tr C) for the 64 leading
//             eigenvalues of the covariance (log singular values relative to
//             the total), f[64] = log n, f[65] = log d, f[66] = eps, f[67] = 1
//   network   68 -> 256 -> 256 -> 1, GELU (exact erf form), output y = log m
//   weights   FP32 master copy + BF16 copies used by the products; FP32
//             accumulation and FP32 activations
//   training  mean squared error on y, Adam with bias correction
//   serving   m = ceil(1.05 exp(y)); adagio_fit with use_predictor verifies m
//             with the exhaustive certificate and continues the search above
//             it when the guess fails
//
// Parameter vector layout: W1 [256][68], b1 [256], W2 [256][256], b2 [256],
// w3 [256], b3 [1].
#include "internal.cuh"
#include "fit.cuh"
#include "linalg.cuh"
#include "pca.cuh"
#include "rng.cuh"

#include <algorithm>

#include <cmath>
#include <cstdio>
#include <cstring>

namespace adagio {

constexpr int kIn = 68, kH1 = 256, kH2 = 256;
constexpr int64_t kOffW1 = 0, kOffB1 = kOffW1 + (int64_t)kH1 * kIn, kOffW2 = kOffB1 + kH1,
                  kOffB2 = kOffW2 + (int64_t)kH2 * kH1, kOffW3 = kOffB2 + kH2, kOffB3 = kOffW3 + kH2,
                  kNParam = kOffB3 + 1;

struct Predictor {
    float *master = nullptr;                 // [kNParam]
    float *m = nullptr, *v = nullptr;        // Adam moments
    __nv_bfloat16 *wb = nullptr;             // BF16 copy of the whole vector (biases unused)
    int64_t step = 0;
    float *scratch = nullptr;                // batch activations and gradients
    int batch_cap = 0;
    double *loss = nullptr;                  // device scalar
};

namespace {

__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float x) {
    return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) + x * 0.39894228040143268f * expf(-0.5f * x * x);
}

__global__ void init_kernel(uint64_t seed, float *w) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= kNParam) return;
    float a = 0.0f;
    if (e < kOffB1) a = sqrtf(6.0f / (kIn + kH1));
    else if (e >= kOffW2 && e < kOffB2) a = sqrtf(6.0f / (kH1 + kH2));
    else if (e >= kOffW3 && e < kOffB3) a = sqrtf(6.0f / (kH2 + 1));
    if (a > 0.0f) {
        const uint64_t z = splitmix64_out(seed ^ 0xA5A5A5A5ull, (uint64_t)e);
        const float u = ((float)(z >> 40) + 0.5f) * (1.0f / 16777216.0f);  // (0, 1)
        w[e] = (2.0f * u - 1.0f) * a;
    } else {
        w[e] = (e == kOffB3) ? 5.0f : 0.0f;   // output bias starts near log(150)
    }
}

__global__ void to_bf16_kernel(const float *w, __nv_bfloat16 *wb) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < kNParam) wb[e] = __float2bfloat16_rn(w[e]);
}

// z <- z + bias (per column); h <- GELU(z)
__global__ void bias_gelu_kernel(float *z, float *h, const float *bias, int B, int N) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)B * N) return;
    const float v = z[e] + bias[e % N];
    z[e] = v;
    h[e] = gelu(v);
}

__global__ void output_kernel(float *y, const float *b3, const float *t, int B, float *dy,
                              double *loss) {
    __shared__ double red[256];
    double acc = 0.0;
    for (int b = threadIdx.x; b < B; b += blockDim.x) {
        const float v = y[b] + b3[0];
        y[b] = v;
        if (t) {
            const float r = v - t[b];
            dy[b] = 2.0f * r / (float)B;
            acc += (double)r * (double)r;
        }
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0 && t) *loss = red[0] / (double)B;
}

// dz[b][j] = dy[b] * w3[j] * GELU'(z2[b][j])
__global__ void out_back_kernel(const float *dy, const __nv_bfloat16 *w3, const float *z2, float *dz,
                                int B, int N) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)B * N) return;
    const int j = (int)(e % N);
    dz[e] = dy[e / N] * __bfloat162float(w3[j]) * gelu_grad(z2[e]);
}

// dz <- dh * GELU'(z)
__global__ void gelu_back_kernel(float *dz, const float *z, int64_t count) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < count) dz[e] *= gelu_grad(z[e]);
}

// g[j] = sum_b dz[b][j]
__global__ void colsum_kernel(const float *dz, int B, int N, float *g) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    float acc = 0.0f;
    for (int b = 0; b < B; ++b) acc += dz[(int64_t)b * N + j];
    g[j] = acc;
}

__global__ void adam_kernel(float *w, const float *g, float *m, float *v, float lr, float c1,
                            float c2) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= kNParam) return;
    const float ge = g[e];
    const float me = 0.9f * m[e] + 0.1f * ge;
    const float ve = 0.999f * v[e] + 0.001f * ge * ge;
    m[e] = me;
    v[e] = ve;
    w[e] -= lr * (me / c1) / (sqrtf(ve / c2) + 1e-8f);
}

__global__ void predict_kernel(const float *y, int count, int *m_out) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= count) return;
    const double r = ceil(1.05 * exp((double)fminf(fmaxf(y[b], -20.0f), 20.0f)));
    m_out[b] = (int)fmin(fmax(r, 1.0), 1073741824.0);
}

__global__ void features_kernel(const double *theta, int have, const float *C, int d, int64_t n,
                                float eps, float *f) {
    __shared__ double tr;
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < d; ++i) s += (double)C[(int64_t)i * d + i];
        tr = s > 0.0 ? s : 1.0;
    }
    __syncthreads();
    const int i = threadIdx.x;
    if (i < 64) {
        const double th = i < have ? theta[i] : 0.0;
        f[i] = (float)(0.5 * log(fmax(th / tr, 1e-12)));
    } else if (i == 64) {
        f[i] = (float)log((double)n);
    } else if (i == 65) {
        f[i] = (float)log((double)d);
    } else if (i == 66) {
        f[i] = eps;
    } else if (i == 67) {
        f[i] = 1.0f;
    }
}

constexpr int kT = 256;
inline unsigned blocks(int64_t n) { return (unsigned)ceil_div(n, kT); }

Predictor *predictor(adagio_ctx *ctx, bool create) {
    if (!ctx->predictor && create) {
        Predictor *p = new Predictor();
        cudaError_t e = cudaMalloc(&p->master, kNParam * sizeof(float) * 3 + kNParam * sizeof(__nv_bfloat16) +
                                                   sizeof(double) + 1024);
        if (e != cudaSuccess) {
            cudaGetLastError();
            delete p;
            fail(ADAGIO_E_WORKSPACE, "cudaMalloc of the predictor failed: %s", cudaGetErrorString(e));
        }
        p->m = p->master + kNParam;
        p->v = p->m + kNParam;
        p->wb = reinterpret_cast<__nv_bfloat16 *>(align_up((uintptr_t)(p->v + kNParam), 256));
        p->loss = reinterpret_cast<double *>(align_up((uintptr_t)(p->wb + kNParam), 256));
        ctx->predictor = p;
    }
    if (!ctx->predictor) fail(ADAGIO_E_INVALID_ARG, "no predictor on this context (init or load one first)");
    return ctx->predictor;
}

void ensure_batch(Predictor *p, int B) {
    if (B <= p->batch_cap) return;
    if (p->scratch) {
        ADAGIO_CUDA(cudaDeviceSynchronize());
        ADAGIO_CUDA(cudaFree(p->scratch));
        p->scratch = nullptr;
        p->batch_cap = 0;
    }
    // z1, h1, z2, h2, dz2, dh1: B x 256 each; y, dy: B; gradient vector
    const size_t floats = (size_t)B * kH1 * 6 + (size_t)B * 2 + kNParam + 64;
    ADAGIO_CUDA(cudaMalloc(&p->scratch, floats * sizeof(float)));
    p->batch_cap = B;
}

struct Batch {
    float *z1, *h1, *z2, *h2, *dz2, *dh1, *y, *dy, *grad;
};

Batch carve(Predictor *p) {
    const size_t S = (size_t)p->batch_cap * kH1;
    Batch b;
    b.z1 = p->scratch;
    b.h1 = b.z1 + S;
    b.z2 = b.h1 + S;
    b.h2 = b.z2 + S;
    b.dz2 = b.h2 + S;
    b.dh1 = b.dz2 + S;
    b.y = b.dh1 + S;
    b.dy = b.y + p->batch_cap;
    b.grad = b.dy + p->batch_cap;
    return b;
}

void forward(Predictor *p, const float *X, int B, Batch &bt, cudaStream_t st) {
    using bf = __nv_bfloat16;
    gemm<float, bf, float, float>(B, kH1, kIn, 1.0f, MatView<float>{X, kIn, 1},
                                  MatView<bf>{p->wb + kOffW1, 1, kIn}, 0.0f, bt.z1, kH1, st);
    bias_gelu_kernel<<<blocks((int64_t)B * kH1), kT, 0, st>>>(bt.z1, bt.h1, p->master + kOffB1, B, kH1);
    ADAGIO_CHECK_LAUNCH();
    gemm<float, bf, float, float>(B, kH2, kH1, 1.0f, MatView<float>{bt.h1, kH1, 1},
                                  MatView<bf>{p->wb + kOffW2, 1, kH1}, 0.0f, bt.z2, kH2, st);
    bias_gelu_kernel<<<blocks((int64_t)B * kH2), kT, 0, st>>>(bt.z2, bt.h2, p->master + kOffB2, B, kH2);
    ADAGIO_CHECK_LAUNCH();
    gemm<float, bf, float, float>(B, 1, kH2, 1.0f, MatView<float>{bt.h2, kH2, 1},
                                  MatView<bf>{p->wb + kOffW3, 1, kH2}, 0.0f, bt.y, 1, st);
}

// forward + loss + gradient into bt.grad (layout of the parameter vector)
void grad_pass(Predictor *p, const float *X, const float *t, int B, Batch &bt, cudaStream_t st) {
    using bf = __nv_bfloat16;
    forward(p, X, B, bt, st);
    output_kernel<<<1, 256, 0, st>>>(bt.y, p->master + kOffB3, t, B, bt.dy, p->loss);
    ADAGIO_CHECK_LAUNCH();
    float *g = bt.grad;
    // output layer: g_w3 = h2^T dy, g_b3 = sum dy
    gemm<float, float, float, float>(1, kH2, B, 1.0f, MatView<float>{bt.dy, 0, 1},
                                     MatView<float>{bt.h2, kH2, 1}, 0.0f, g + kOffW3, kH2, st);
    colsum_kernel<<<1, 32, 0, st>>>(bt.dy, B, 1, g + kOffB3);
    ADAGIO_CHECK_LAUNCH();
    // dz2 = (dy w3^T) * GELU'(z2)
    out_back_kernel<<<blocks((int64_t)B * kH2), kT, 0, st>>>(bt.dy, p->wb + kOffW3, bt.z2, bt.dz2, B, kH2);
    ADAGIO_CHECK_LAUNCH();
    // g_W2 = dz2^T h1, g_b2 = colsum dz2
    gemm<float, float, float, float>(kH2, kH1, B, 1.0f, MatView<float>{bt.dz2, 1, kH2},
                                     MatView<float>{bt.h1, kH1, 1}, 0.0f, g + kOffW2, kH1, st);
    colsum_kernel<<<blocks(kH2), kT, 0, st>>>(bt.dz2, B, kH2, g + kOffB2);
    ADAGIO_CHECK_LAUNCH();
    // dz1 = (dz2 W2) * GELU'(z1)
    gemm<float, bf, float, float>(B, kH1, kH2, 1.0f, MatView<float>{bt.dz2, kH2, 1},
                                  MatView<bf>{p->wb + kOffW2, kH1, 1}, 0.0f, bt.dh1, kH1, st);
    gelu_back_kernel<<<blocks((int64_t)B * kH1), kT, 0, st>>>(bt.dh1, bt.z1, (int64_t)B * kH1);
    ADAGIO_CHECK_LAUNCH();
    // g_W1 = dz1^T X, g_b1 = colsum dz1
    gemm<float, float, float, float>(kH1, kIn, B, 1.0f, MatView<float>{bt.dh1, 1, kH1},
                                     MatView<float>{X, kIn, 1}, 0.0f, g + kOffW1, kIn, st);
    colsum_kernel<<<blocks(kH1), kT, 0, st>>>(bt.dh1, B, kH1, g + kOffB1);
    ADAGIO_CHECK_LAUNCH();
}

void refresh_bf16(Predictor *p, cudaStream_t st) {
    to_bf16_kernel<<<blocks(kNParam), kT, 0, st>>>(p->master, p->wb);
    ADAGIO_CHECK_LAUNCH();
}

const float *stage_rows(adagio_ctx *ctx, const float *p, int64_t rows, int cols, cudaStream_t st) {
    int64_t ld;
    return stage_input(ctx, p, rows, cols, cols, &ld, st);
}

}  // namespace

void free_predictor(adagio_ctx *ctx) {
    if (!ctx || !ctx->predictor) return;
    Predictor *p = ctx->predictor;
    if (p->master) cudaFree(p->master);
    if (p->scratch) cudaFree(p->scratch);
    delete p;
    ctx->predictor = nullptr;
}

// Predicted dimension from 68 device features (synchronises).
int predict_one(adagio_ctx *ctx, const float *feats, cudaStream_t st) {
    Predictor *p = predictor(ctx, false);
    ensure_batch(p, 1);
    Batch bt = carve(p);
    forward(p, feats, 1, bt, st);
    output_kernel<<<1, 256, 0, st>>>(bt.y, p->master + kOffB3, nullptr, 1, nullptr, nullptr);
    ADAGIO_CHECK_LAUNCH();
    int *dm = reinterpret_cast<int *>(bt.dy);
    predict_kernel<<<1, 32, 0, st>>>(bt.y, 1, dm);
    ADAGIO_CHECK_LAUNCH();
    int m = 0;
    ADAGIO_CUDA(cudaMemcpyAsync(&m, dm, sizeof(int), cudaMemcpyDeviceToHost, st));
    ADAGIO_CUDA(cudaStreamSynchronize(st));
    return m;
}

void predict_many(adagio_ctx *ctx, const float *feats, int B, int *dm, int *m_host, cudaStream_t st) {
    Predictor *p = predictor(ctx, false);
    ensure_batch(p, B);
    Batch bt = carve(p);
    forward(p, feats, B, bt, st);
    output_kernel<<<1, 256, 0, st>>>(bt.y, p->master + kOffB3, nullptr, B, nullptr, nullptr);
    ADAGIO_CHECK_LAUNCH();
    predict_kernel<<<(unsigned)ceil_div(B, 256), 256, 0, st>>>(bt.y, B, dm);
    ADAGIO_CHECK_LAUNCH();
    ADAGIO_CUDA(cudaMemcpyAsync(m_host, dm, B * sizeof(int), cudaMemcpyDeviceToHost, st));
}

void spectrum_features(const double *theta, int have, const float *C, int d, int64_t n, double eps,
                       float *feats, cudaStream_t st) {
    features_kernel<<<1, 128, 0, st>>>(theta, have, C, d, n, (float)eps, feats);
    ADAGIO_CHECK_LAUNCH();
}

bool has_predictor(const adagio_ctx *ctx) { return ctx && ctx->predictor; }

}  // namespace adagio

using namespace adagio;

#define MLP_BEGIN(ctx)                         \
    if (!(ctx)) return ADAGIO_E_INVALID_ARG;   \
    (ctx)->last_error.clear();                 \
    try {                                      \
        DeviceGuard guard_((ctx)->device);     \
        ws_reset(ctx);

#define MLP_END(ctx)                           \
    }                                          \
    catch (const Error &e) {                   \
        (ctx)->last_error = e.msg;             \
        return e.code;                         \
    }                                          \
    catch (...) {                              \
        (ctx)->last_error = "unknown failure"; \
        return ADAGIO_E_CUDA;                  \
    }

extern "C" {

int64_t adagio_mlp_num_params(void) { return kNParam; }

int adagio_mlp_init(adagio_ctx *ctx, uint64_t seed) {
    MLP_BEGIN(ctx)
    Predictor *p = predictor(ctx, true);
    init_kernel<<<blocks(kNParam), kT>>>(seed, p->master);
    ADAGIO_CHECK_LAUNCH();
    ADAGIO_CUDA(cudaMemset(p->m, 0, 2 * kNParam * sizeof(float)));
    refresh_bf16(p, 0);
    p->step = 0;
    ADAGIO_CUDA(cudaDeviceSynchronize());
    return ADAGIO_OK;
    MLP_END(ctx)
}

int adagio_mlp_set_params(adagio_ctx *ctx, const float *params, int64_t count) {
    MLP_BEGIN(ctx)
    ADAGIO_REQUIRE(params && count == kNParam, "expected %lld parameters", (long long)kNParam);
    Predictor *p = predictor(ctx, true);
    ADAGIO_CUDA(cudaMemcpy(p->master, params, kNParam * sizeof(float), cudaMemcpyDefault));
    ADAGIO_CUDA(cudaMemset(p->m, 0, 2 * kNParam * sizeof(float)));
    p->step = 0;
    refresh_bf16(p, 0);
    ADAGIO_CUDA(cudaDeviceSynchronize());
    return ADAGIO_OK;
    MLP_END(ctx)
}

int adagio_mlp_get_params(adagio_ctx *ctx, float *params, int64_t count) {
    MLP_BEGIN(ctx)
    ADAGIO_REQUIRE(params && count == kNParam, "expected %lld parameters", (long long)kNParam);
    Predictor *p = predictor(ctx, false);
    ADAGIO_CUDA(cudaMemcpy(params, p->master, kNParam * sizeof(float), cudaMemcpyDefault));
    return ADAGIO_OK;
    MLP_END(ctx)
}

int adagio_mlp_forward(adagio_ctx *ctx, const float *feats, int count, float *y, void *stream) {
    MLP_BEGIN(ctx)
    ADAGIO_REQUIRE(feats && y && count >= 1, "bad arguments");
    cudaStream_t st = (cudaStream_t)stream;
    Predictor *p = predictor(ctx, false);
    ensure_batch(p, count);
    ws_reserve(ctx, (size_t)count * kIn * sizeof(float) + 4096);
    const float *X = stage_rows(ctx, feats, count, kIn, st);
    Batch bt = carve(p);
    forward(p, X, count, bt, st);
    output_kernel<<<1, 256, 0, st>>>(bt.y, p->master + kOffB3, nullptr, count, nullptr, nullptr);
    ADAGIO_CHECK_LAUNCH();
    ADAGIO_CUDA(cudaMemcpyAsync(y, bt.y, count * sizeof(float), cudaMemcpyDefault, st));
    ADAGIO_CUDA(cudaStreamSynchronize(st));
    return ADAGIO_OK;
    MLP_END(ctx)
}

int adagio_mlp_grad(adagio_ctx *ctx, const float *feats, const float *target, int count,
                    double *loss, float *grads, void *stream) {
    MLP_BEGIN(ctx)
    ADAGIO_REQUIRE(feats && target && grads && count >= 1, "bad arguments");
    cudaStream_t st = (cudaStream_t)stream;
    Predictor *p = predictor(ctx, false);
    ensure_batch(p, count);
    ws_reserve(ctx, (size_t)count * (kIn + 1) * sizeof(float) + 8192);
    const float *X = stage_rows(ctx, feats, count, kIn, st);
    const float *t = stage_rows(ctx, target, count, 1, st);
    Batch bt = carve(p);
    grad_pass(p, X, t, count, bt, st);
    ADAGIO_CUDA(cudaMemcpyAsync(grads, bt.grad, kNParam * sizeof(float), cudaMemcpyDefault, st));
    if (loss) ADAGIO_CUDA(cudaMemcpyAsync(loss, p->loss, sizeof(double), cudaMemcpyDefault, st));
    ADAGIO_CUDA(cudaStreamSynchronize(st));
    return ADAGIO_OK;
    MLP_END(ctx)
}

int adagio_mlp_train_step(adagio_ctx *ctx, const float *feats, const float *target, int count,
                          float lr, double *loss, void *stream) {
    MLP_BEGIN(ctx)
    ADAGIO_REQUIRE(feats && target && count >= 1 && lr > 0.0f, "bad arguments");
    cudaStream_t st = (cudaStream_t)stream;
    Predictor *p = predictor(ctx, false);
    ensure_batch(p, count);
    ws_reserve(ctx, (size_t)count * (kIn + 1) * sizeof(float) + 8192);
    const float *X = stage_rows(ctx, feats, count, kIn, st);
    const float *t = stage_rows(ctx, target, count, 1, st);
    Batch bt = carve(p);
    grad_pass(p, X, t, count, bt, st);
    p->step += 1;
    const float c1 = (float)(1.0 - pow(0.9, (double)p->step));
    const float c2 = (float)(1.0 - pow(0.999, (double)p->step));
    adam_kernel<<<blocks(kNParam), kT, 0, st>>>(p->master, bt.grad, p->m, p->v, lr, c1, c2);
    ADAGIO_CHECK_LAUNCH();
    refresh_bf16(p, st);
    if (loss) {
        ADAGIO_CUDA(cudaMemcpyAsync(loss, p->loss, sizeof(double), cudaMemcpyDefault, st));
        ADAGIO_CUDA(cudaStreamSynchronize(st));
    }
    return ADAGIO_OK;
    MLP_END(ctx)
}

int adagio_predict_m(adagio_ctx *ctx, const float *feats, int count, int *m_out, void *stream) {
    MLP_BEGIN(ctx)
    ADAGIO_REQUIRE(feats && m_out && count >= 1, "bad arguments");
    cudaStream_t st = (cudaStream_t)stream;
    Predictor *p = predictor(ctx, false);
    ensure_batch(p, count);
    ws_reserve(ctx, (size_t)count * kIn * sizeof(float) + (size_t)count * sizeof(int) + 8192);
    const float *X = stage_rows(ctx, feats, count, kIn, st);
    Batch bt = carve(p);
    forward(p, X, count, bt, st);
    output_kernel<<<1, 256, 0, st>>>(bt.y, p->master + kOffB3, nullptr, count, nullptr, nullptr);
    ADAGIO_CHECK_LAUNCH();
    int *dm = ws_array<int>(ctx, count);
    predict_kernel<<<(unsigned)ceil_div(count, 256), 256, 0, st>>>(bt.y, count, dm);
    ADAGIO_CHECK_LAUNCH();
    ADAGIO_CUDA(cudaMemcpyAsync(m_out, dm, count * sizeof(int), cudaMemcpyDefault, st));
    ADAGIO_CUDA(cudaStreamSynchronize(st));
    return ADAGIO_OK;
    MLP_END(ctx)
}

int adagio_features(adagio_ctx *ctx, const float *X, int64_t n, int d, int64_t ldx, double eps,
                    const adagio_fit_opts *opts, float *feats, void *stream) {
    MLP_BEGIN(ctx)
    ADAGIO_REQUIRE(X && feats && n >= 2 && d >= 1 && ldx >= d, "bad arguments");
    adagio_fit_opts o;
    if (opts) o = *opts; else adagio_default_fit_opts(&o);
    cudaStream_t st = (cudaStream_t)stream;
    const int s = std::min(64, d);
    const bool x_dev = is_device_ptr(X, ctx->device);
    ws_reserve(ctx, (x_dev ? 0 : align_up((size_t)n * d * sizeof(float), 256)) +
                        pca_bytes(ctx, n, d, s, o.oversample, o.precision != ADAGIO_PREC_FP32) + 8192);
    int64_t lx;
    const float *dX = stage_input(ctx, X, n, d, ldx, &lx, st);
    PCA pca;
    pca.init(ctx, dX, n, d, lx, s, o.seed, o.max_iter, o.tol, o.oversample,
             o.precision != ADAGIO_PREC_FP32, st);
    pca.extend(s, st);
    float *df = ws_array<float>(ctx, kIn);
    spectrum_features(pca.theta, pca.s_done, pca.C, d, n, eps, df, st);
    ADAGIO_CUDA(cudaMemcpyAsync(feats, df, kIn * sizeof(float), cudaMemcpyDefault, st));
    ADAGIO_CUDA(cudaStreamSynchronize(st));
    return ADAGIO_OK;
    MLP_END(ctx)
}

int adagio_mlp_save(adagio_ctx *ctx, const char *path) {
    MLP_BEGIN(ctx)
    ADAGIO_REQUIRE(path, "null path");
    Predictor *p = predictor(ctx, false);
    std::vector<float> buf((size_t)kNParam * 3);
    ADAGIO_CUDA(cudaMemcpy(buf.data(), p->master, buf.size() * sizeof(float), cudaMemcpyDeviceToHost));
    FILE *f = std::fopen(path, "wb");
    ADAGIO_REQUIRE(f, "cannot open %s for writing", path);
    const char magic[8] = {'A', 'D', 'A', 'G', 'M', 'L', 'P', '1'};
    const int64_t hdr[2] = {kNParam, p->step};
    bool ok = std::fwrite(magic, 1, 8, f) == 8 && std::fwrite(hdr, sizeof(hdr), 1, f) == 1 &&
              std::fwrite(buf.data(), sizeof(float), buf.size(), f) == buf.size();
    ok = (std::fclose(f) == 0) && ok;
    ADAGIO_REQUIRE(ok, "write to %s failed", path);
    return ADAGIO_OK;
    MLP_END(ctx)
}

int adagio_mlp_load(adagio_ctx *ctx, const char *path) {
    MLP_BEGIN(ctx)
    ADAGIO_REQUIRE(path, "null path");
    FILE *f = std::fopen(path, "rb");
    ADAGIO_REQUIRE(f, "cannot open %s", path);
    char magic[8];
    int64_t hdr[2] = {0, 0};
    std::vector<float> buf((size_t)kNParam * 3);
    bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, "ADAGMLP1", 8) == 0 &&
              std::fread(hdr, sizeof(hdr), 1, f) == 1 && hdr[0] == kNParam &&
              std::fread(buf.data(), sizeof(float), buf.size(), f) == buf.size();
    std::fclose(f);
    ADAGIO_REQUIRE(ok, "%s is not a predictor file of this library", path);
    Predictor *p = predictor(ctx, true);
    ADAGIO_CUDA(cudaMemcpy(p->master, buf.data(), buf.size() * sizeof(float), cudaMemcpyHostToDevice));
    p->step = hdr[1];
    refresh_bf16(p, 0);
    ADAGIO_CUDA(cudaDeviceSynchronize());
    return ADAGIO_OK;
    MLP_END(ctx)
}

}  // extern "C"
