// Split-bfloat16 operand format shared by the packers and the GEMM: the
// 128-byte-swizzled K-major tile layout and the hi / mid / lo parts.
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

}  // namespace tnh
