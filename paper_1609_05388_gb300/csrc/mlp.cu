// Dimension predictor (not built yet): every entry fails loudly.
#include "internal.cuh"
#include "fit.cuh"

namespace adagio {

int fit_predicted(adagio_ctx *ctx, const float *, int64_t, int, int64_t, const adagio_fit_opts *,
                  float *, int, int *, int *, adagio_cert *, void *) {
    if (ctx) ctx->last_error = "the dimension predictor is not available in this build";
    return ADAGIO_E_UNSUPPORTED;
}

void free_predictor(adagio_ctx *) {}

}  // namespace adagio
