// Kernel-launch profiler: when enabled on a context, every kernel launch of
// the library is bracketed by CUDA events on the launch stream, so the caller
// can read per-kernel device time and launch counts for a region of work.
#pragma once

#include "tnh_internal.h"

namespace tnh {

struct Profiler {
    struct Rec {
        const char* name;
        cudaEvent_t a, b;
    };
    bool on = false;
    std::vector<Rec> recs;
    std::vector<cudaEvent_t> pool;
    cudaEvent_t get();
    void clear();
    ~Profiler();
};

Profiler* active_profiler();
void set_active_profiler(Profiler* p);

// RAII scope around one kernel launch.
struct KScope {
    Profiler* p;
    cudaStream_t s;
    size_t idx;
    KScope(const char* name, cudaStream_t st) : p(active_profiler()), s(st), idx(0) {
        if (p && p->on) {
            Profiler::Rec r{name, p->get(), p->get()};
            cudaEventRecord(r.a, s);
            p->recs.push_back(r);
            idx = p->recs.size();
        }
    }
    ~KScope() {
        if (p && p->on && idx) cudaEventRecord(p->recs[idx - 1].b, s);
    }
};

}  // namespace tnh
