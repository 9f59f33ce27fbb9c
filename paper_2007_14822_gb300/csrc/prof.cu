// Kernel-launch profiler (see prof.h) and its two entry points.
#include <cstring>
#include <map>

#include "prof.h"
#include "tnh_guard.h"

namespace tnh {

namespace {
thread_local Profiler* g_active = nullptr;
}

Profiler* active_profiler() { return g_active; }
void set_active_profiler(Profiler* p) { g_active = p; }

cudaEvent_t Profiler::get() {
    if (!pool.empty()) {
        cudaEvent_t e = pool.back();
        pool.pop_back();
        return e;
    }
    cudaEvent_t e;
    CUDA_CHECK(cudaEventCreate(&e));
    return e;
}

void Profiler::clear() {
    for (auto& r : recs) {
        pool.push_back(r.a);
        pool.push_back(r.b);
    }
    recs.clear();
}

Profiler::~Profiler() {
    clear();
    for (auto e : pool) cudaEventDestroy(e);
}

}  // namespace tnh

using namespace tnh;

extern "C" {

tnh_status tnh_profile_begin(tnh_ctx* ctx) {
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    return guard(c, [&] {
        TNH_REQUIRE(c, TNH_ERR_ARG, "tnh_profile_begin: ctx NULL");
        if (!c->prof) c->prof = std::make_unique<Profiler>();
        c->prof->clear();
        c->prof->on = true;
        set_active_profiler(c->prof.get());
    });
}

tnh_status tnh_profile_end(tnh_ctx* ctx, int32_t max_kinds, int32_t* nkinds, char* names, int64_t* launches,
                           double* ms) {
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    return guard(c, [&] {
        TNH_REQUIRE(c && nkinds, TNH_ERR_ARG, "tnh_profile_end: NULL argument");
        TNH_REQUIRE(c->prof && c->prof->on, TNH_ERR_ARG, "tnh_profile_end: profiling was not started");
        CUDA_CHECK(cudaStreamSynchronize(c->stream));
        std::map<std::string, std::pair<int64_t, double>> agg;
        for (auto& r : c->prof->recs) {
            float t = 0.f;
            CUDA_CHECK(cudaEventElapsedTime(&t, r.a, r.b));
            auto& e = agg[r.name];
            e.first += 1;
            e.second += t;
        }
        c->prof->on = false;
        c->prof->clear();
        if (active_profiler() == c->prof.get()) set_active_profiler(nullptr);
        int k = 0;
        for (auto& kv : agg) {
            if (k < max_kinds) {
                if (names) {
                    std::strncpy(names + (size_t)k * 64, kv.first.c_str(), 63);
                    names[(size_t)k * 64 + 63] = 0;
                }
                if (launches) launches[k] = kv.second.first;
                if (ms) ms[k] = kv.second.second;
            }
            ++k;
        }
        *nkinds = k;
    });
}

}  // extern "C"
