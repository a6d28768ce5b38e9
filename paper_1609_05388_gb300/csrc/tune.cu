// Autotuner of the certificate's tile configuration (tile kernel and schedule
// band), its per-context table by size class of n, and the table's JSON file.
#include "internal.cuh"
#include "cert.cuh"
#include "api_guard.cuh"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

using namespace adagio;

namespace {

// the fastest of one warm-up and three timed certificates, tile kernel only
double time_config(adagio_ctx *ctx, const float *X, int64_t ldx, const float *Y, int64_t ldy,
                   int64_t n, int d, int m, const CertOptions &co, cudaStream_t st) {
    adagio_cert c;
    certify(ctx, X, ldx, Y, ldy, n, d, m, co, &c, st);
    double best = 1e300;
    for (int r = 0; r < 3; ++r) {
        certify(ctx, X, ldx, Y, ldy, n, d, m, co, &c, st);
        best = std::min(best, ctx->last_stats.tile_ms);
    }
    return best;
}

// A tiny reader for the table format adagio_tune_save writes.
bool read_string_field(const std::string &s, const char *key, std::string *out) {
    const std::string k = std::string("\"") + key + "\"";
    size_t p = s.find(k);
    if (p == std::string::npos) return false;
    p = s.find(':', p + k.size());
    if (p == std::string::npos) return false;
    p = s.find('"', p);
    if (p == std::string::npos) return false;
    const size_t e = s.find('"', p + 1);
    if (e == std::string::npos) return false;
    *out = s.substr(p + 1, e - p - 1);
    return true;
}

bool read_number_field(const std::string &obj, const char *key, double *out) {
    const std::string k = std::string("\"") + key + "\"";
    size_t p = obj.find(k);
    if (p == std::string::npos) return false;
    p = obj.find(':', p + k.size());
    if (p == std::string::npos) return false;
    char *end = nullptr;
    const double v = std::strtod(obj.c_str() + p + 1, &end);
    if (end == obj.c_str() + p + 1) return false;
    *out = v;
    return true;
}

}  // namespace

extern "C" {

int adagio_autotune_tiles(adagio_ctx *ctx, const float *X, int64_t n, int d, int64_t ldx,
                          const float *Y, int m, int64_t ldy, double eps, int precision,
                          adagio_tile_config *best, void *stream) {
    API_BEGIN(ctx)
    ADAGIO_REQUIRE(X && Y && best, "null pointer argument");
    ADAGIO_REQUIRE(n >= 2 && n < (1ll << 31) - 256 && d >= 1 && m >= 1 && ldx >= d && ldy >= m,
                   "bad sizes n=%lld d=%d m=%d", (long long)n, d, m);
    ADAGIO_REQUIRE(std::isfinite(eps) && eps > 0.0 && eps < 1.0, "eps must lie in (0, 1), got %g", eps);
    ADAGIO_REQUIRE(precision == ADAGIO_PREC_FP16X3 || precision == ADAGIO_PREC_BF16X3,
                   "the tile configuration applies to the split precisions, not %d", precision);
    cudaStream_t st = (cudaStream_t)stream;
    ws_reserve(ctx, stage_aligned_bytes(ctx, X, n, d, ldx) + stage_aligned_bytes(ctx, Y, n, m, ldy) +
                        certify_bytes(ctx, n, d, m, precision) + 4096);
    int64_t lx, ly;
    const float *dX = stage_aligned(ctx, X, n, d, ldx, &lx, st);
    const float *dY = stage_aligned(ctx, Y, n, m, ldy, &ly, st);
    CertOptions co;
    co.eps = eps;
    co.lo = 0.0;
    co.hi = 2.0 * eps;
    co.precision = precision;
    const int saved_variant = ctx->tc_variant, saved_band = ctx->tc_band, saved_timing = ctx->collect_timing;
    std::vector<int> variants{ADAGIO_TILES_SINGLE};
    if (pad_rows(n) % 256 == 0 && tc_pair_supported(ctx)) variants.push_back(ADAGIO_TILES_PAIR);
    adagio_tile_config b{ADAGIO_TILES_SINGLE, 8, 1e300, tc_size_class(n)};
    struct Restore {
        adagio_ctx *c;
        int v, bd, t;
        ~Restore() {
            c->tc_variant = v;
            c->tc_band = bd;
            c->collect_timing = t;
        }
    } restore{ctx, saved_variant, saved_band, saved_timing};
    ctx->collect_timing = 1;
    for (int v : variants)
        for (int band : {4, 8, 16, 32, 64}) {
            ctx->tc_variant = v;
            ctx->tc_band = band;
            const double ms = time_config(ctx, dX, lx, dY, ly, n, d, m, co, st);
            if (ms < b.tile_ms) b = adagio_tile_config{v, band, ms, b.size_class};
        }
    ctx->tc_tuned[b.size_class] = TunedTiles{b.variant, b.band, b.tile_ms};
    *best = b;
    return ADAGIO_OK;
    API_END(ctx)
}

int adagio_tune_save(const adagio_ctx *ctx, const char *path) {
    if (!ctx || !path) return ADAGIO_E_INVALID_ARG;
    FILE *f = std::fopen(path, "w");
    if (!f) return ADAGIO_E_INVALID_ARG;
    std::string name = ctx->device_name;
    for (char &ch : name)
        if (ch == '"' || ch == '\\') ch = '_';
    std::fprintf(f, "{\"device\": \"%s\", \"entries\": [", name.c_str());
    bool first = true;
    for (const auto &e : ctx->tc_tuned) {
        std::fprintf(f, "%s\n  {\"size_class\": %d, \"variant\": %d, \"band\": %d, \"tile_ms\": %.6f}",
                     first ? "" : ",", e.first, e.second.variant, e.second.band, e.second.ms);
        first = false;
    }
    std::fprintf(f, "\n]}\n");
    const bool ok = std::fclose(f) == 0;
    return ok ? ADAGIO_OK : ADAGIO_E_INVALID_ARG;
}

int adagio_tune_load(adagio_ctx *ctx, const char *path) {
    if (!ctx || !path) return ADAGIO_E_INVALID_ARG;
    FILE *f = std::fopen(path, "r");
    if (!f) {
        ctx->last_error = std::string("cannot open ") + path;
        return ADAGIO_E_INVALID_ARG;
    }
    std::string s;
    char buf[4096];
    size_t k;
    while ((k = std::fread(buf, 1, sizeof(buf), f)) > 0) s.append(buf, k);
    std::fclose(f);
    std::string dev;
    if (!read_string_field(s, "device", &dev)) {
        ctx->last_error = "malformed tile table: no device";
        return ADAGIO_E_INVALID_ARG;
    }
    std::string mine = ctx->device_name;
    for (char &ch : mine)
        if (ch == '"' || ch == '\\') ch = '_';
    if (dev != mine) {
        ctx->last_error = "tile table of device '" + dev + "', this context runs on '" + mine + "'";
        return ADAGIO_E_INVALID_ARG;
    }
    std::map<int, TunedTiles> table;
    size_t p = s.find('[');
    if (p == std::string::npos) {
        ctx->last_error = "malformed tile table: no entries";
        return ADAGIO_E_INVALID_ARG;
    }
    while (true) {
        const size_t o = s.find('{', p + 1);
        if (o == std::string::npos) break;
        const size_t c = s.find('}', o);
        if (c == std::string::npos) {
            ctx->last_error = "malformed tile table: unterminated entry";
            return ADAGIO_E_INVALID_ARG;
        }
        const std::string obj = s.substr(o, c - o + 1);
        double sc, v, bd, ms;
        if (!read_number_field(obj, "size_class", &sc) || !read_number_field(obj, "variant", &v) ||
            !read_number_field(obj, "band", &bd) || !read_number_field(obj, "tile_ms", &ms) ||
            !(v == 1 || v == 2) || !(bd >= 1 && bd <= 64) || sc < 0 || sc > 30) {
            ctx->last_error = "malformed tile table entry: " + obj;
            return ADAGIO_E_INVALID_ARG;
        }
        table[(int)sc] = TunedTiles{(int)v, (int)bd, ms};
        p = c;
    }
    for (const auto &e : table) ctx->tc_tuned[e.first] = e.second;
    return ADAGIO_OK;
}

}  // extern "C"
