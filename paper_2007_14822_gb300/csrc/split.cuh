// Split-bfloat16 operand format shared by the packers and the GEMM: the
// 128-byte-swizzled K-major tile layout and the hi / mid / lo parts, and the
// float32 <-> float64 conversions of the packers and epilogues.
#pragma once

#include <cuda_bf16.h>

#include <cstdint>

namespace tnh {

// Offset of element (row, k) inside a 128 x 64 bfloat16 operand tile in the
// 128-byte-swizzled K-major layout of the tcgen05 shared-memory descriptor:
// the 16-byte chunk j of row r holds k-group j ^ (r & 7).
__device__ __forceinline__ int swz(int row, int k) {
    return row * 64 + ((((k >> 3) ^ (row & 7))) << 3) + (k & 7);
}

// hi / mid / lo bfloat16 parts (round to nearest each) of two float32
// values, packed in pairs: plane p holds (part p of a) | (part p of b) << 16
template <int P>
__device__ __forceinline__ void split2(float a, float b, uint32_t* w) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    w[0] = *reinterpret_cast<uint32_t*>(&h);
    if (P > 1) {
        const float2 hf = __bfloat1622float2(h);
        const float ra = a - hf.x, rb = b - hf.y;
        __nv_bfloat162 m = __floats2bfloat162_rn(ra, rb);
        w[1] = *reinterpret_cast<uint32_t*>(&m);
        if (P > 2) {
            const float2 mf = __bfloat1622float2(m);
            __nv_bfloat162 l = __floats2bfloat162_rn(ra - mf.x, rb - mf.y);
            w[2] = *reinterpret_cast<uint32_t*>(&l);
        }
    }
}

// Conversions between the IEEE 754 binary32 and binary64 formats written with
// integer operations: GB300 issues float64 conversions on its float64 pipe,
// which has a small fraction of the float32 rate, and the packers and
// epilogues convert every element once. Values outside the fast cases take the
// hardware conversion.

// float32 -> float64 (exact): exponent rebiased from 127 to 1023, the 23-bit
// fraction widened to 52 bits. Subnormal float32 inputs take the hardware path.
__device__ __forceinline__ void f32_to_f64_words(float x, uint32_t& hi, uint32_t& lo) {
    const uint32_t u = __float_as_uint(x);
    const uint32_t e = (u >> 23) & 0xffu, f = u & 0x7fffffu, sign = u & 0x80000000u;
    if (e == 0u) {
        if (f == 0u) { hi = sign; lo = 0u; return; }
        const double d = (double)x;
        hi = (uint32_t)__double2hiint(d);
        lo = (uint32_t)__double2loint(d);
        return;
    }
    const uint32_t e64 = e == 0xffu ? 0x7ffu : e + 896u;
    hi = sign | (e64 << 20) | (f >> 3);
    lo = f << 29;
}

__device__ __forceinline__ double f32_to_f64(float x) {
    uint32_t hi, lo;
    f32_to_f64_words(x, hi, lo);
    return __hiloint2double((int)hi, (int)lo);
}

// float64 -> float32, rounded to nearest (ties to even), for inputs whose
// result is zero or a normal float32; the 52-bit fraction keeps its top 23
// bits and the 29 bits below decide the rounding (a carry into the exponent,
// up to infinity, is the correct rounded result). Subnormal results and
// infinities or NaNs on input take the hardware path.
__device__ __forceinline__ float f64_to_f32_rn(double x) {
    const uint32_t hi = (uint32_t)__double2hiint(x), lo = (uint32_t)__double2loint(x);
    const uint32_t sign = hi & 0x80000000u;
    if (((hi & 0x7fffffffu) | lo) == 0u) return __uint_as_float(sign);
    const int e32 = (int)((hi >> 20) & 0x7ffu) - 896;
    if (e32 <= 0 || e32 >= 255) return (float)x;
    const uint32_t f = ((hi & 0xfffffu) << 3) | (lo >> 29);
    const uint32_t r = lo & 0x1fffffffu;
    uint32_t mag = ((uint32_t)e32 << 23) | f;
    if (r > 0x10000000u || (r == 0x10000000u && (f & 1u))) mag += 1u;
    return __uint_as_float(sign | mag);
}

}  // namespace tnh
