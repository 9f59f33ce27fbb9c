// Grouped float64 GEMM on the CUDA cores: the plain FP64 path of the
// matrix-multiply step of a contraction (Sec. 9.4).
//
// C_t[M][ldc] = A_t[M][K] * B_t[N][K]^T for every task t, both operands
// K-major and zero-padded to 64-row / 16-column multiples by the packer
// (row pitches lda, ldb >= 16 * kt).
// One CTA computes one 64 x 64 output tile; tiles of all tasks form one grid.
#include "prof.h"
#include "tnh_internal.h"

namespace tnh {

namespace {

__device__ __forceinline__ int find_task(const GemmTask* __restrict__ tasks, int ntasks, int tile) {
    int lo = 0, hi = ntasks - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (tasks[mid].tile0 <= tile) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__global__ void __launch_bounds__(256) gemm_f64_kernel(const GemmTask* __restrict__ tasks, int ntasks,
                                                       const double* __restrict__ A,
                                                       const double* __restrict__ B,
                                                       double* __restrict__ C,
                                                       const int64_t* __restrict__ row_off) {
    __shared__ double As[kF64TileK][kF64TileM + 1];
    __shared__ double Bs[kF64TileK][kF64TileN + 1];
    const int tile = blockIdx.x;
    const GemmTask t = tasks[find_task(tasks, ntasks, tile)];
    const int local = tile - t.tile0;
    const int mi = local / t.nt, ni = local - mi * t.nt;
    const double* Ab = A + t.a_base + (int64_t)mi * kF64TileM * t.lda;
    const double* Bb = B + t.b_base + (int64_t)ni * kF64TileN * t.ldb;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
    for (int k0 = 0; k0 < t.kt * kF64TileK; k0 += kF64TileK) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            int e = tid + i * 256, row = e >> 4, k = e & 15;
            As[k][row] = Ab[(int64_t)row * t.lda + k0 + k];
            Bs[k][row] = Bb[(int64_t)row * t.ldb + k0 + k];
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kF64TileK; ++k) {
            double a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[k][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[k][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        int m = mi * kF64TileM + ty + 16 * i;
        if (m >= t.M) continue;
        const int64_t rb = t.use_roff ? row_off[t.roff + m] : t.c_base + (int64_t)m * t.ldc;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int n = ni * kF64TileN + tx + 16 * j;
            if (n < t.N) C[rb + n] = acc[i][j];
        }
    }
}

}  // namespace

void launch_gemm_f64(const GemmTask* d_tasks, int ntasks, int total_tiles, const double* A, const double* B,
                     double* C, cudaStream_t s, const int64_t* row_off) {
    if (total_tiles == 0) return;
    KScope ks("gemm_f64", s);
    gemm_f64_kernel<<<total_tiles, 256, 0, s>>>(d_tasks, ntasks, A, B, C, row_off);
}

}  // namespace tnh
