// Exception-to-status translation used by every extern "C" entry point.
#pragma once

#include <new>

#include "tnh_internal.h"

namespace tnh {

void set_error(Ctx* ctx, const std::string& m);

template <class F>
tnh_status guard(Ctx* ctx, F&& f) {
    try {
        if (ctx) {
            AllocScope scope(ctx->stream);
            f();
        } else {
            f();
        }
        return TNH_OK;
    } catch (const Error& e) {
        set_error(ctx, e.msg);
        return e.code;
    } catch (const std::bad_alloc&) {
        set_error(ctx, "host allocation failed");
        return TNH_ERR_OOM;
    } catch (const std::exception& e) {
        set_error(ctx, e.what());
        return TNH_ERR_ARG;
    }
}

}  // namespace tnh
