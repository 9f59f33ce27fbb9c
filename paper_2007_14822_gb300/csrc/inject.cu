// Failure injection for tests (no counterpart in the paper).
//
// The library reports failures as status codes and keeps the context usable
// after them. These entry points make the failures happen on purpose, in the
// two forms that need no GPU fault:
//   - a device allocation that fails on the host side (the k-th one from
//     now), which must give TNH_ERR_OOM and leave no memory held;
//   - a bounded device wait that nothing ever completes: the kernel gives
//     up after a short limit, records the site in the context's error flag
//     and returns, and the host turns the flag into TNH_ERR_TIMEOUT.
// Nothing here traps, faults or hangs a device.
#include <atomic>

#include "ptx.cuh"
#include "tnh_guard.h"
#include "tnh_internal.h"

namespace tnh {

namespace {

// > 0: the allocation that brings the count to zero fails
std::atomic<int64_t> g_alloc_countdown{0};

// One thread waits on an mbarrier on which no thread ever arrives, with the
// same bounded wait the GEMM pipelines use; it gives up after limit_ns.
__global__ void wait_nothing_kernel(int* err, uint64_t limit_ns) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        ptx::mbar_init(&bar, 1);
        ptx::fence_mbar_init();
        ptx::mbar_wait(&bar, 0, err, /*site=*/100, /*watch_flag=*/false, limit_ns);
    }
}

}  // namespace

bool alloc_fault_injected() {
    int64_t c = g_alloc_countdown.load();
    while (c > 0) {
        if (g_alloc_countdown.compare_exchange_weak(c, c - 1)) return c == 1;
    }
    return false;
}

}  // namespace tnh

using namespace tnh;

extern "C" {

tnh_status tnh_debug_fail_alloc(int64_t k) {
    return guard(nullptr, [&] {
        TNH_REQUIRE(k >= 0, TNH_ERR_ARG, "tnh_debug_fail_alloc: k must be >= 0 (got %lld)", (long long)k);
        g_alloc_countdown.store(k);
    });
}

tnh_status tnh_debug_pool_used(tnh_ctx* ctx, uint64_t* bytes) {
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    return guard(c, [&] {
        TNH_REQUIRE(c && bytes, TNH_ERR_ARG, "tnh_debug_pool_used: NULL argument");
        CUDA_CHECK(cudaSetDevice(c->device));
        CUDA_CHECK(cudaStreamSynchronize(c->stream));
        *bytes = pool_used_bytes();
    });
}

tnh_status tnh_debug_wait_timeout(tnh_ctx* ctx, uint64_t limit_ns) {
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    return guard(c, [&] {
        TNH_REQUIRE(c, TNH_ERR_ARG, "tnh_debug_wait_timeout: ctx is NULL");
        TNH_REQUIRE(limit_ns >= 1000 && limit_ns <= 1000000000ull, TNH_ERR_ARG,
                    "tnh_debug_wait_timeout: limit %llu ns outside [1 us, 1 s]", (unsigned long long)limit_ns);
        CUDA_CHECK(cudaSetDevice(c->device));
        wait_nothing_kernel<<<1, 32, 0, c->stream>>>(c->d_flag.as<int>(), limit_ns);
        CUDA_CHECK(cudaGetLastError());
        check_device_flag(c);
    });
}

}  // extern "C"
