// Operand packing: strided block -> GEMM operand (float64 plain or split
// bfloat16 tiles), and GEMM result -> strided block.
//
// The permutation of the contraction ("permute then GEMM", Sec. 9.4) happens
// here, in the same pass that converts float64 into the operand format, so
// the GEMM reads only contiguous tiles.
#include <cuda_bf16.h>

#include "prof.h"
#include "tnh_internal.h"

namespace tnh {

namespace {

__device__ __forceinline__ int64_t strided_offset(const Piece& p, int r, int c) {
    int64_t o = 0;
    for (int q = p.nr - 1; q >= 0; --q) {
        int d = p.dims[q];
        o += (int64_t)(r % d) * p.strides[q];
        r /= d;
    }
    for (int q = p.nc - 1; q >= 0; --q) {
        int d = p.dims[p.nr + q];
        o += (int64_t)(c % d) * p.strides[p.nr + q];
        c /= d;
    }
    return o;
}

__global__ void pack_f64_kernel(const Piece* __restrict__ pieces, const Chunk* __restrict__ chunks,
                                const OpGeom* __restrict__ geom, const double* __restrict__ src,
                                double* __restrict__ dst) {
    __shared__ Piece sp;
    const Chunk ch = chunks[blockIdx.x];
    if (threadIdx.x == 0) sp = pieces[ch.piece];
    __syncthreads();
    const OpGeom g = geom[sp.task];
    for (int e = threadIdx.x; e < ch.count; e += blockDim.x) {
        int idx = ch.start + e;
        int r = idx / sp.cols, c = idx - r * sp.cols;
        double x = src[sp.src_off + strided_offset(sp, r, c)];
        dst[g.base + (int64_t)(sp.row0 + r) * g.ld + sp.col0 + c] = x;
    }
}

// Offset of element (row, k) inside a 128 x 64 bf16 tile stored in the
// 128-byte-swizzled K-major layout the tcgen05 smem descriptor expects:
// 128-byte rows, 16-byte chunk index XOR (row mod 8).
__device__ __forceinline__ int swz(int row, int k) {
    return row * 64 + ((((k >> 3) ^ (row & 7))) << 3) + (k & 7);
}

template <int P>
__global__ void pack_bf16_kernel(const Piece* __restrict__ pieces, const Chunk* __restrict__ chunks,
                                 const OpGeom* __restrict__ geom, const double* __restrict__ src,
                                 uint16_t* __restrict__ dst) {
    __shared__ Piece sp;
    const Chunk ch = chunks[blockIdx.x];
    if (threadIdx.x == 0) sp = pieces[ch.piece];
    __syncthreads();
    const OpGeom g = geom[sp.task];
    for (int e = threadIdx.x; e < ch.count; e += blockDim.x) {
        int idx = ch.start + e;
        int r = idx / sp.cols, c = idx - r * sp.cols;
        double x = src[sp.src_off + strided_offset(sp, r, c)];
        int R = sp.row0 + r, K = sp.col0 + c;
        int64_t tile = g.base + (int64_t)(R >> 7) * g.ld + (K >> 6);
        uint16_t* t = dst + tile * (int64_t)(P * kTcTileElems);
        int w = swz(R & 127, K & 63);
        // x = hi + mid + lo, each part rounded to nearest bfloat16
        __nv_bfloat16 hi = __double2bfloat16(x);
        t[w] = __bfloat16_as_ushort(hi);
        if (P > 1) {
            double r1 = x - (double)__bfloat162float(hi);
            __nv_bfloat16 mid = __double2bfloat16(r1);
            t[kTcTileElems + w] = __bfloat16_as_ushort(mid);
            if (P > 2) {
                double r2 = r1 - (double)__bfloat162float(mid);
                t[2 * kTcTileElems + w] = __bfloat16_as_ushort(__double2bfloat16(r2));
            }
        }
    }
}

__global__ void unpack_kernel(const Piece* __restrict__ pieces, const Chunk* __restrict__ chunks,
                              const int64_t* __restrict__ cbase, const int* __restrict__ ldc,
                              const double* __restrict__ Ct, double* __restrict__ dst) {
    __shared__ Piece sp;
    const Chunk ch = chunks[blockIdx.x];
    if (threadIdx.x == 0) sp = pieces[ch.piece];
    __syncthreads();
    const int64_t base = cbase[sp.task];
    const int ld = ldc[sp.task];
    for (int e = threadIdx.x; e < ch.count; e += blockDim.x) {
        int idx = ch.start + e;
        int r = idx / sp.cols, c = idx - r * sp.cols;
        dst[sp.src_off + strided_offset(sp, r, c)] = Ct[base + (int64_t)r * ld + c];
    }
}

}  // namespace

void launch_pack_f64(const Piece* d_pieces, const Chunk* d_chunks, int nchunks, const OpGeom* d_geom,
                     const double* src, double* dst, cudaStream_t s) {
    if (nchunks == 0) return;
    KScope ks("pack_f64", s);
    pack_f64_kernel<<<nchunks, 256, 0, s>>>(d_pieces, d_chunks, d_geom, src, dst);
}

void launch_pack_bf16(const Piece* d_pieces, const Chunk* d_chunks, int nchunks, const OpGeom* d_geom,
                      const double* src, uint16_t* dst, int planes, cudaStream_t s) {
    if (nchunks == 0) return;
    KScope ks("pack_split_bf16", s);
    if (planes == 3)
        pack_bf16_kernel<3><<<nchunks, 256, 0, s>>>(d_pieces, d_chunks, d_geom, src, dst);
    else if (planes == 2)
        pack_bf16_kernel<2><<<nchunks, 256, 0, s>>>(d_pieces, d_chunks, d_geom, src, dst);
    else
        pack_bf16_kernel<1><<<nchunks, 256, 0, s>>>(d_pieces, d_chunks, d_geom, src, dst);
}

void launch_unpack(const Piece* d_pieces, const Chunk* d_chunks, int nchunks, const int64_t* d_cbase,
                   const int* d_ldc, const double* Ct, double* dst, cudaStream_t s) {
    if (nchunks == 0) return;
    KScope ks("unpack", s);
    unpack_kernel<<<nchunks, 256, 0, s>>>(d_pieces, d_chunks, d_cbase, d_ldc, Ct, dst);
}

}  // namespace tnh
