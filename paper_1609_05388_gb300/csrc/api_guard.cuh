// Entry-point guard of the C ABI: selects the context's device, resets the
// workspace arena and turns internal failures into status codes (no C++
// exception crosses the ABI).
#pragma once

#include <exception>

#include "internal.cuh"

#define API_BEGIN(ctx)                                  \
    if (!(ctx)) return ADAGIO_E_INVALID_ARG;            \
    (ctx)->last_error.clear();                          \
    try {                                               \
        adagio::DeviceGuard guard_((ctx)->device);      \
        adagio::ws_reset(ctx);

#define API_END(ctx)                                    \
    }                                                   \
    catch (const adagio::Error &e) {                    \
        (ctx)->last_error = e.msg;                      \
        return e.code;                                  \
    }                                                   \
    catch (const std::exception &e) {                   \
        (ctx)->last_error = e.what();                   \
        return ADAGIO_E_CUDA;                           \
    }                                                   \
    catch (...) {                                       \
        (ctx)->last_error = "unknown failure";          \
        return ADAGIO_E_CUDA;                           \
    }
