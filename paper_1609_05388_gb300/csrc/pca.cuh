#pragma once

#include "internal.cuh"
#include "tcgemm.cuh"

#include <algorithm>

namespace adagio {

// Incremental randomized PCA of one data set (see pca.cu).  All buffers come
// from the context workspace; reserve pca_bytes() first.
struct PCA {
    adagio_ctx *ctx = nullptr;
    int64_t n = 0;
    int d = 0, s_cap = 0, p = 32, max_iter = 100;
    uint64_t seed = 0;
    double tol = 1e-6, theta1 = 0.0;
    int s_done = 0, iterations = 0;
    float *C = nullptr;        // d x d covariance
    float *P = nullptr;        // s_cap x d principal rows (first s_done valid)
    double *theta = nullptr;   // eigenvalue estimates of those rows
    float *V = nullptr, *W = nullptr, *T = nullptr, *U = nullptr, *coef = nullptr, *res = nullptr;
    double *G = nullptr, *H = nullptr, *theta_blk = nullptr, *f64part = nullptr;
    float *G32 = nullptr, *R32 = nullptr, *part = nullptr;  // FP32 Gram, Cholesky factor, split-K
    float *Dinv = nullptr;     // b x 32: inverses of the factor's diagonal blocks
    int64_t part_floats = 0;
    unsigned *flags = nullptr;
    // tensor: the covariance and the products V C on tcgen05 from split
    // planes (the split-precision fits); otherwise FP32 SIMT (the plain path)
    bool tensor = false;
    SplitPlanes Cp, Vp;        // tensor: planes of C and of the current block
    float *gpart = nullptr;    // tensor: split-K partials of V C
    double *elapsed_ms = nullptr;  // optional: extend() adds its wall time here
    // pinned host buffer of at least pca_host_bytes() for the convergence
    // checks; null: the context's staging buffer at each use
    void *hbuf = nullptr;

    void init(adagio_ctx *ctx, const float *X, int64_t n, int d, int64_t ldx, int s_cap,
              uint64_t seed, int max_iter, double tol, int oversample, bool tensor, cudaStream_t st);
    // make sure the first s_needed rows of P are computed (synchronises)
    void extend(int s_needed, cudaStream_t st);

    // The same computation as a resumable sequence, for lock-step batches:
    //   init_enqueue ; sync ; init_check
    //   while (needs(s)) { advance(s) ; sync ; resolve() }
    // advance enqueues work up to the next convergence test (with its copy to
    // the host); resolve reads it after the caller synchronised the stream and
    // enqueues the next iteration or the acceptance of the block.
    void init_enqueue(adagio_ctx *ctx, const float *X, int64_t n, int d, int64_t ldx, int s_cap,
                      uint64_t seed, int max_iter, double tol, int oversample, bool tensor,
                      cudaStream_t st);
    void init_check();
    bool needs(int s_needed) const { return s_done < std::min(s_needed, s_cap); }
    void advance(int s_needed, cudaStream_t st);
    void resolve(cudaStream_t st);

   private:
    struct Block {
        bool active = false;
        int it = 0, s_blk = 0, b = 0, remaining = 0;
        int next_rr = 0;  // iteration of the next Rayleigh-Ritz step
        int rr = 0;       // Rayleigh-Ritz steps taken in this block
        bool last = false;
    } blk;
    void *stage(size_t bytes);
    void begin_block(int s_needed, cudaStream_t st);
    void accept_block(cudaStream_t st);
    void deflate(float *M, int r, cudaStream_t st);
    // passes: 3 (orthonormal to FP32 precision from any FP32-representable
    // conditioning) or 1 (the first pass alone: with shift0 > 0 a
    // well-conditioned basis of the same span; with shift0 = 0 the
    // re-orthonormalisation of an almost orthonormal M); shift0 is relative
    // to the largest Gram entry
    void orth(float *M, int b, cudaStream_t st, int passes = 3, float shift0 = 1e-5f);
    bool rr_follows(int it) const;
    void times_C(const float *M, int b, float *out, cudaStream_t st);  // out = M C
    void copy_status(cudaStream_t st);
    void check_status();
};

// tensor: the split-precision PCA (see PCA::tensor)
size_t pca_bytes(adagio_ctx *ctx, int64_t n, int d, int s_cap, int oversample, bool tensor);
size_t pca_host_bytes();

}  // namespace adagio
