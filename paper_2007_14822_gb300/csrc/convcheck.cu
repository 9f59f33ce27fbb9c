// Self-check of the float32 <-> float64 conversions written with integer
// operations (split.cuh), against the GPU's own conversion instructions.
//
// The packers round float64 inputs to float32 with f64_to_f32_rn and the
// epilogues widen float32 results with f32_to_f64; both must give the bits of
// the hardware conversion (round to nearest, ties to even; widening exact).
// The check draws bit patterns from a counter-based generator (SplitMix64,
// Steele, Lea and Flood 2014): a quarter uniform over all 64-bit patterns, a
// quarter with exponents around the float32 range and its edges, a quarter of
// exact rounding ties and a quarter near the float32 overflow boundary. For
// the widening the low 32 bits serve as the float32 input. NaN results count
// as equal when both sides are NaN.
#include <algorithm>

#include "split.cuh"
#include "tnh_guard.h"
#include "tnh_internal.h"

namespace tnh {

namespace {

__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
    x += 0x9e3779b97f4a7c15ull;
    x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ull;
    x = (x ^ (x >> 27)) * 0x94d049bb133111ebull;
    return x ^ (x >> 31);
}

__device__ __forceinline__ uint64_t pattern(uint64_t seed, uint64_t i) {
    const uint64_t r = splitmix64(seed ^ splitmix64(i));
    const uint64_t r2 = splitmix64(r);
    const uint64_t sign = r & 0x8000000000000000ull;
    const uint64_t frac = r2 & 0xfffffffffffffull;
    switch (i & 3) {
        case 0: return r;
        case 1: {
            // exponents 896 - 40 .. 896 + 255 + 40: subnormal float32 results,
            // the whole normal range and overflow
            const uint64_t e = 856 + (r >> 40) % 335;
            return sign | (e << 52) | frac;
        }
        case 2: {
            // a tie: the 29 bits below the float32 fraction are 1 followed by zeros
            const uint64_t e = 897 + (r >> 40) % 253;
            return sign | (e << 52) | (frac & ~0x1fffffffull) | 0x10000000ull;
        }
        default: {
            // the largest float32 binade, fraction near all ones
            const uint64_t e = 896 + 254;
            return sign | (e << 52) | (0xfffffull << 32) | (frac & 0xffffffffull);
        }
    }
}

__device__ __forceinline__ bool same(float a, float b) {
    return (a != a && b != b) || __float_as_uint(a) == __float_as_uint(b);
}
__device__ __forceinline__ bool same(double a, double b) {
    return (a != a && b != b) || __double_as_longlong(a) == __double_as_longlong(b);
}

__global__ void convert_check_kernel(uint64_t n, uint64_t seed, unsigned long long* bad) {
    unsigned long long local = 0;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t bits = pattern(seed, i);
        const double x = __longlong_as_double((long long)bits);
        if (!same(f64_to_f32_rn(x), (float)x)) ++local;
        const float y = __uint_as_float((uint32_t)bits);
        if (!same(f32_to_f64(y), (double)y)) ++local;
    }
    if (local) atomicAdd(bad, local);
}

}  // namespace

}  // namespace tnh

using namespace tnh;

extern "C" {

tnh_status tnh_debug_convert_check(tnh_ctx* ctx, uint64_t n, uint64_t seed, uint64_t* mismatches) {
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    return guard(c, [&] {
        TNH_REQUIRE(c && mismatches, TNH_ERR_ARG, "tnh_debug_convert_check: NULL argument");
        CUDA_CHECK(cudaSetDevice(c->device));
        AllocScope scope(c->stream);
        DevBuf bad(sizeof(unsigned long long));
        CUDA_CHECK(cudaMemsetAsync(bad.p, 0, sizeof(unsigned long long), c->stream));
        if (n > 0) {
            const int grid = (int)std::min<uint64_t>((n + 255) / 256, 4096);
            convert_check_kernel<<<grid, 256, 0, c->stream>>>(n, seed, bad.as<unsigned long long>());
            CUDA_CHECK(cudaGetLastError());
        }
        unsigned long long h = 0;
        CUDA_CHECK(cudaMemcpyAsync(&h, bad.p, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
        CUDA_CHECK(cudaStreamSynchronize(c->stream));
        *mismatches = h;
    });
}

}  // extern "C"
