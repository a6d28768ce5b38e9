#pragma once

#include <vector>

#include "internal.cuh"
#include "tcgemm.cuh"

namespace adagio {

struct FitProbe {
    int r;
    int ok;
    double max;
};

// Optional trace of a fit: the probes of the search, the PCA effort, and a
// predicted starting dimension (verified first; the search continues above
// it on failure).
struct FitTrace {
    int start_r = 0;
    bool verify_only = false;  // with start_r: accept start_r if it passes
    std::vector<FitProbe> probes;
    int pca_iterations = 0;
    int s_computed = 0;
};

// A = [P ; S (I - P^T P)] (Algorithm 1); T is k x s scratch.
void assemble(const float *P, int s, int64_t ldp, const float *S, int k, int64_t lds, int d,
              float *A, int64_t lda, float *T, cudaStream_t st);

size_t fit_bytes(adagio_ctx *ctx, int64_t n, int d, int s_cap, int k_cap, int m_cap, int precision,
                 int oversample);

// The projection Y = X A^T (Algorithm 1) as adagio_embed computes it: per-row
// FP16 split planes of the raw rows of X, made once and reused for every map
// A (up to m_cap rows), and the tensor-core GEMM.  Every fit embeds this way,
// so a returned certificate is the one of adagio_embed's Y, bit for bit.
struct EmbedPlanes {
    SplitPlanes Xp;
    int64_t n = 0;
    int d = 0;
    void *scratch = nullptr;
};
size_t embed_planes_bytes(adagio_ctx *ctx, int64_t n, int d, int m_cap);
void embed_planes_init(adagio_ctx *ctx, const float *X, int64_t n, int d, int64_t ldx, int m_cap,
                       EmbedPlanes &ep, cudaStream_t st);
void embed_planes_run(adagio_ctx *ctx, const EmbedPlanes &ep, const float *A, int m, int64_t lda,
                      float *Y, int64_t ldy, cudaStream_t st);

// Fit on device data; A_out (device) gets m x d rows with leading dimension d.
int fit_device(adagio_ctx *ctx, const float *X, int64_t n, int d, int64_t ldx,
               const adagio_fit_opts *o, float *A_out, int m_cap, int *m_out, int *s_out,
               adagio_cert *cert, cudaStream_t st, FitTrace *trace);

// Public-argument fit (checks, staging) with an optional trace.
int fit_entry(adagio_ctx *ctx, const float *X, int64_t n, int d, int64_t ldx,
              const adagio_fit_opts *opts, float *A, int m_cap, int *m_out, int *s_out,
              adagio_cert *cert, void *stream, FitTrace *trace);

// Dimension predictor (mlp.cu).
bool has_predictor(const adagio_ctx *ctx);
int predict_one(adagio_ctx *ctx, const float *feats, cudaStream_t st);
// predictions for B feature rows (device, B x 68) into dm (device) and m_host
// (pinned host); enqueued only, the caller synchronises
void predict_many(adagio_ctx *ctx, const float *feats, int B, int *dm, int *m_host, cudaStream_t st);
void spectrum_features(const double *theta, int have, const float *C, int d, int64_t n, double eps,
                       float *feats, cudaStream_t st);

}  // namespace adagio
