// Grouped split-bfloat16 GEMM on the 5th-generation tensor cores (tcgen05):
// the matrix-multiply step of a permute-then-multiply contraction (Sec. 9.4),
// one task per output block of a block-sparse product (Sec. 8.3, Sec. 9.2).
//
// C_t[M][ldc] (float64, or float32 per task) = sum over products (p, q) of A_t^(p) * B_t^(q)^T,
// where A^(0..P-1) / B^(0..P-1) are the bfloat16 parts of the float64
// operands (x = hi + mid + lo). P = 3 keeps the six products
// hh, hm, mh, hl, lh, mm; P = 2 keeps hh, hm, mh; P = 1 keeps hh.
//
// Persistent warp-specialised kernel, one CTA per SM, 128 x 128 output tiles:
//   warp 0      producer: bulk-copies the P A-tiles and P B-tiles of one
//               64-wide K block into a shared-memory stage (TMA engine,
//               mbarrier complete_tx); operands arrive pre-tiled and
//               pre-swizzled from the packer, one 16 KB copy per tile.
//   warp 1      MMA issuer: one thread issues tcgen05.mma (M=128, N=128,
//               K=16) into tensor memory; hh goes to its own accumulator,
//               the cross products to a second one, so the large partial
//               sums are not rounded once per small cross term.
//   warps 2..9  epilogue (two warps per TMEM lane quarter, 64 columns each;
//               rows leave through a small shared-memory stage so that
//               every store is one contiguous row segment). The tensor core accumulates one K chunk (128
//               for the three-part split) at a time; the epilogue adds every
//               chunk's two accumulators into float32 registers (round to
//               nearest) and stores float64 at the end of the tile. The
//               tensor-core accumulation error grows linearly with the
//               number of MMAs accumulated, so short chunks bound it.
//               Two accumulator pairs (512 TMEM columns) let the epilogue of
//               one chunk overlap the MMAs of the next.
// Every wait is bounded (ptx::mbar_wait); a timeout sets the device error flag.
#include <cuda_bf16.h>

#include <type_traits>

#include "gather.h"
#include "prof.h"
#include "ptx.cuh"
#include "split.cuh"
#include "tnh_internal.h"

namespace tnh {

namespace {

constexpr int kTileBytes = kTcTileM * kTcTileK * 2;   // 16384, A and B tiles alike
constexpr int kThreads = 320;   // producer, MMA, 8 epilogue warps
constexpr int kEpiWarps = 8;
// with the A operand formed in the kernel: 4 more warps (warps 10-13) that
// build each A stage from its gather segments
constexpr int kAWarps = 4;
constexpr int kThreadsFused = kThreads + 32 * kAWarps;

// epilogue staging: per epilogue warp 32 rows x 33 words (a 32 x 32 float or
// 32 x 16 double block, one padding word per row against bank conflicts)
constexpr int kStageWords = 32 * 33;
constexpr int kEpiStageBytes = kEpiWarps * kStageWords * 4;

template <int P>
struct TcCfg {
    static constexpr int kStages = P == 3 ? 2 : (P == 2 ? 3 : 6);
    static constexpr int kNumProd = P == 3 ? 6 : (P == 2 ? 3 : 1);
    static constexpr int kStageBytes = 2 * P * kTileBytes;
    static constexpr int kSmem = kStages * kStageBytes + 1024 /*align*/ + 256 /*barriers*/ + kEpiStageBytes;
    static_assert(kSmem <= 232448, "shared memory of one CTA");
    // k-blocks (of 64) accumulated on the tensor core before the epilogue
    // folds the partial sum into registers
    static constexpr int kChunk = P == 3 ? 2 : (P == 2 ? 4 : 8);
};

// products (a-part, b-part); the first one is hh
__constant__ int kProdA[6] = {0, 0, 1, 0, 2, 1};
__constant__ int kProdB[6] = {0, 1, 0, 2, 0, 1};

__device__ __forceinline__ int find_task(const GemmTask* __restrict__ tasks, int ntasks, int tile) {
    int lo = 0, hi = ntasks - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (tasks[mid].tile0 <= tile) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// kFusedA: operand A is not read pre-packed but formed in the kernel, tile
// by tile, from float32 source rows: A tile (task, mi, kb) is the gather tile
// a_base + mi * kstride + kb of (atiles, asegs, aterms), every segment of it
// a rectangle whose elements are sums of coef * asrc[off + r rs + c] (the
// W1.W2 step of the effective Hamiltonian feeding S4 directly). Segments
// cover every row below M and every column of the tile; four warps write the
// split-bfloat16 planes into the stage and arrive on its barrier.
template <int P, bool kFusedA>
__global__ void __launch_bounds__(kFusedA ? kThreadsFused : kThreads, 1)
    gemm_tc_kernel(const GemmTask* __restrict__ tasks, int ntasks, int total_tiles,
                   const uint16_t* __restrict__ A, const uint16_t* __restrict__ B, double* __restrict__ C,
                   int* err, const int64_t* __restrict__ row_off, const GatherTile* __restrict__ atiles,
                   const GatherSeg* __restrict__ asegs, const GatherTerm* __restrict__ aterms,
                   const float* __restrict__ asrc) {
    using Cfg = TcCfg<P>;
    constexpr int S = Cfg::kStages;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    uint8_t* sA = smem;                               // [S][P] tiles
    uint8_t* sB = smem + S * P * kTileBytes;          // [S][P] tiles
    uint64_t* full = reinterpret_cast<uint64_t*>(sB + S * P * kTileBytes);
    uint64_t* empty = full + S;
    uint64_t* tfull = empty + S;
    uint64_t* tempty = tfull + 2;
    uint64_t* fin = tempty + 2;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(fin + 1);
    uint32_t* stage_all = reinterpret_cast<uint32_t*>(smem + 2 * S * P * kTileBytes + 256);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            ptx::mbar_init(&full[s], kFusedA ? 1 + kAWarps : 1);
            ptx::mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            ptx::mbar_init(&tfull[b], 1);
            ptx::mbar_init(&tempty[b], kEpiWarps);
        }
        ptx::mbar_init(fin, 1);
        ptx::fence_mbar_init();
    }
    if (warp == 0) {
        ptx::tmem_alloc(tmem_slot, 512);
        ptx::tmem_relinquish();
    }
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- producer
            int stage = 0;
            uint32_t phase = 0;
            bool ok = true;
            for (int tile = blockIdx.x; ok && tile < total_tiles; tile += gridDim.x) {
                const GemmTask& t = tasks[find_task(tasks, ntasks, tile)];
                const int local = tile - t.tile0;
                const int mi = local / t.nt, ni = local - mi * t.nt;
                const int ks = t.kstride ? t.kstride : t.kt;
                const int tn = t.tn ? t.tn : kTcTileN;
                // an N tile of tn rows of B is rows [ni*tn, ni*tn + tn) of the
                // 128-row packed tiles: a contiguous slice of one of them (the
                // 128-byte swizzle repeats every 8 rows)
                const int bt = (ni * tn) >> 7, boff = ((ni * tn) & 127) * 64;
                const uint32_t bbytes = (uint32_t)tn * 128u;
                const uint16_t* a = A + (t.a_base + (int64_t)mi * ks) * P * kTcTileElems;
                const uint16_t* b = B + (t.b_base + (int64_t)bt * ks) * P * kTcTileElems + boff;
                for (int kb = 0; kb < t.kt; ++kb) {
                    if (!ptx::mbar_wait(&empty[stage], phase ^ 1u, err, 1)) { ok = false; break; }
                    ptx::mbar_expect_tx(&full[stage], P * ((kFusedA ? 0u : (uint32_t)kTileBytes) + bbytes));
                    if (!kFusedA) {
#pragma unroll
                        for (int p = 0; p < P; ++p)
                            ptx::bulk_g2s(sA + (stage * P + p) * kTileBytes,
                                          a + ((int64_t)kb * P + p) * kTcTileElems, kTileBytes, &full[stage]);
                    }
#pragma unroll
                    for (int p = 0; p < P; ++p)
                        ptx::bulk_g2s(sB + (stage * P + p) * kTileBytes,
                                      b + ((int64_t)kb * P + p) * kTcTileElems, bbytes, &full[stage]);
                    if (++stage == S) { stage = 0; phase ^= 1u; }
                }
            }
            if (!ok) __nanosleep(20000);   // let copies already in flight land
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------- MMA issuer
            int stage = 0;
            uint32_t phase = 0;
            bool ok = true;
            int it = 0;
            for (int tile = blockIdx.x; ok && tile < total_tiles; tile += gridDim.x) {
                const GemmTask& t = tasks[find_task(tasks, ntasks, tile)];
                const int tn = t.tn ? t.tn : kTcTileN;
                const uint32_t idesc = tn == 128 ? ptx::idesc_bf16_f32(kTcTileM, 128)
                                                 : (tn == 64 ? ptx::idesc_bf16_f32(kTcTileM, 64)
                                                             : ptx::idesc_bf16_f32(kTcTileM, 32));
                for (int k0 = 0; ok && k0 < t.kt; k0 += Cfg::kChunk, ++it) {
                    const int k1 = min(t.kt, k0 + Cfg::kChunk);
                    const int buf = it & 1;
                    const uint32_t tph = (uint32_t)(it >> 1) & 1u;
                    if (!ptx::mbar_wait(&tempty[buf], tph ^ 1u, err, 2)) { ok = false; break; }
                    ptx::tc_fence_after();
                    const uint32_t d_hh = tmem + buf * 256, d_x = tmem + buf * 256 + 128;
                    for (int kb = k0; kb < k1; ++kb) {
                        if (!ptx::mbar_wait(&full[stage], phase, err, 3)) { ok = false; break; }
                        ptx::tc_fence_after();
                        const uint32_t a0 = ptx::smem_u32(sA + stage * P * kTileBytes);
                        const uint32_t b0 = ptx::smem_u32(sB + stage * P * kTileBytes);
#pragma unroll
                        for (int kk = 0; kk < kTcTileK / 16; ++kk) {
#pragma unroll
                            for (int j = 0; j < Cfg::kNumProd; ++j) {
                                const uint64_t ad =
                                    ptx::sw128_kmajor_desc(a0 + kProdA[j] * kTileBytes + kk * 32);
                                const uint64_t bd =
                                    ptx::sw128_kmajor_desc(b0 + kProdB[j] * kTileBytes + kk * 32);
                                const bool first = (kb == k0 && kk == 0);
                                const uint32_t acc = j == 0 ? !first : (!first || j > 1);
                                ptx::mma_bf16(j == 0 ? d_hh : d_x, ad, bd, idesc, acc);
                            }
                        }
                        ptx::mma_commit(&empty[stage]);
                        if (++stage == S) { stage = 0; phase ^= 1u; }
                    }
                    if (!ok) break;
                    ptx::mma_commit(&tfull[buf]);
                }
            }
            // every MMA issued above completes before the tensor memory is freed
            ptx::mma_commit(fin);
            ptx::mbar_wait(fin, 0, err, 4, /*watch_flag=*/false);
        }
    } else if (kFusedA && warp >= 2 + kEpiWarps) {
        // ---------------- A producers: form each A stage from its segments
        const int ptid = threadIdx.x - 32 * (2 + kEpiWarps);
        int stage = 0;
        uint32_t phase = 0;
        bool ok = true;
        for (int tile = blockIdx.x; ok && tile < total_tiles; tile += gridDim.x) {
            const GemmTask& t = tasks[find_task(tasks, ntasks, tile)];
            const int mi = (tile - t.tile0) / t.nt;
            const int ks = t.kstride ? t.kstride : t.kt;
            for (int kb = 0; kb < t.kt; ++kb) {
                if (!ptx::mbar_wait(&empty[stage], phase ^ 1u, err, 6)) { ok = false; break; }
                const GatherTile g = atiles[t.a_base + (int64_t)mi * ks + kb];
                uint8_t* sa = sA + stage * P * kTileBytes;
                for (int si = g.seg0; si < g.seg1; ++si) {
                    const GatherSeg sg = asegs[si];
                    const int ncq = sg.nc >> 2, nq = sg.nr * ncq;
                    for (int e = ptid; e < nq; e += 32 * kAWarps) {
                        const int r = e / ncq, cq = e - r * ncq;
                        float v[4] = {0.f, 0.f, 0.f, 0.f};
                        for (int j = sg.t0; j < sg.t1; ++j) {
                            const GatherTerm gt = aterms[j];
                            const float4 x =
                                __ldg(reinterpret_cast<const float4*>(asrc + gt.off + (int64_t)r * gt.rs + 4 * cq));
                            v[0] = fmaf(gt.coef32, x.x, v[0]);
                            v[1] = fmaf(gt.coef32, x.y, v[1]);
                            v[2] = fmaf(gt.coef32, x.z, v[2]);
                            v[3] = fmaf(gt.coef32, x.w, v[3]);
                        }
                        uint32_t w0[3], w1[3];
                        split2<P>(v[0], v[1], w0);
                        split2<P>(v[2], v[3], w1);
                        const int off = swz(sg.r0 + r, sg.c0 + 4 * cq);
#pragma unroll
                        for (int p = 0; p < P; ++p)
                            *reinterpret_cast<uint2*>(sa + p * kTileBytes + off * 2) = make_uint2(w0[p], w1[p]);
                    }
                }
                // the tensor core (async proxy) reads what these threads wrote
                ptx::fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) ptx::mbar_arrive(&full[stage]);
                if (++stage == S) { stage = 0; phase ^= 1u; }
            }
        }
    } else {
        // ---------------- epilogue: warp w owns TMEM lane quarter (w % 4) and
        // the column half (w - 2) / 4 of the tile
        const int q = warp & 3;
        const int half = (warp - 2) >> 2;
        constexpr int kCols = kTcTileN / 2;
        int it = 0;
        bool ok = true;
        for (int tile = blockIdx.x; ok && tile < total_tiles; tile += gridDim.x) {
            const GemmTask& t = tasks[find_task(tasks, ntasks, tile)];
            const int local = tile - t.tile0;
            const int mi = local / t.nt, ni = local - mi * t.nt;
            const int tn = t.tn ? t.tn : kTcTileN;
            // columns of this warp: 128-wide tiles give each half 64; a 64- or
            // 32-wide tile is read by the half-0 warps alone
            const int cbase = tn == 128 ? half * kCols : 0;
            const int ncols = tn == 128 ? kCols : (half == 0 ? tn : 0);
            const int nend = min(t.N, ni * tn + tn);   // last column of this tile + 1
            float acc[kCols];
#pragma unroll
            for (int j = 0; j < kCols; ++j) acc[j] = 0.0f;
            for (int k0 = 0; k0 < t.kt; k0 += Cfg::kChunk, ++it) {
                const int buf = it & 1;
                const uint32_t tph = (uint32_t)(it >> 1) & 1u;
                if (!ptx::mbar_wait(&tfull[buf], tph, err, 5)) { ok = false; break; }
                ptx::tc_fence_after();
                const uint32_t row_addr = tmem + ((uint32_t)(q * 32) << 16) + buf * 256 + cbase;
#pragma unroll
                for (int c0 = 0; c0 < kCols; c0 += 32) {
                    if (c0 >= ncols) break;
                    if constexpr (kFusedA) {
                        // one 32-column buffer at a time (the 14-warp launch
                        // leaves fewer registers per thread): the chunk's hh
                        // and cross sums are added to the running sum in turn
                        uint32_t r[32];
                        ptx::tmem_ld32(row_addr + c0, r);
                        ptx::tmem_wait_ld();
#pragma unroll
                        for (int j = 0; j < 32; ++j) acc[c0 + j] += __uint_as_float(r[j]);
                        if (P > 1) {
                            ptx::tmem_ld32(row_addr + 128 + c0, r);
                            ptx::tmem_wait_ld();
#pragma unroll
                            for (int j = 0; j < 32; ++j) acc[c0 + j] += __uint_as_float(r[j]);
                        }
                    } else {
                        uint32_t rh[32], rx[32];
                        ptx::tmem_ld32(row_addr + c0, rh);
                        if (P > 1) ptx::tmem_ld32(row_addr + 128 + c0, rx);
                        ptx::tmem_wait_ld();
#pragma unroll
                        for (int j = 0; j < 32; ++j) {
                            float v = __uint_as_float(rh[j]);
                            if (P > 1) v += __uint_as_float(rx[j]);
                            acc[c0 + j] += v;
                        }
                    }
                }
                ptx::tc_fence_before();
                __syncwarp();
                if (lane == 0) ptx::mbar_arrive(&tempty[buf]);
            }
            if (!ok) break;
            // ---- store: each warp stages 32 x 32 (float) or 32 x 16 (double)
            // blocks in shared memory and writes every row as one contiguous
            // segment (row starts come from row m's owner lane)
            const int m = mi * kTcTileM + q * 32 + lane;
            const int mrow = m < t.M;
            const int64_t rb = mrow ? (t.use_roff ? row_off[t.roff + m] : t.c_base + (int64_t)m * t.ldc) : 0;
            const int n0 = ni * tn + cbase;
            uint32_t* buf = stage_all + (warp - 2) * kStageWords;
            // float32 rows that start on 16-byte boundaries and end on them
            // (every row of a float32 result without scatter whose base,
            // pitch and width are multiples of 4, in a 16-byte-aligned
            // output) leave by 16-byte stores
            const bool vec4 = t.c_f32 && !t.use_roff && ((t.c_base | (int64_t)t.ldc | (int64_t)t.N) & 3) == 0 &&
                              (reinterpret_cast<uintptr_t>(C) & 15) == 0;
            if (ncols == 0) {
                // nothing to store for this warp
            } else if (vec4) {
                // aligned float32 rows: the 32 x 32 block goes through the
                // stage (a row per lane), then every lane stores 16 bytes of
                // one of four rows per step: eight 128-byte row segments per
                // store instruction, and no wait on a copy engine
                float* Cf = reinterpret_cast<float*>(C);
                const int cq = (lane & 7) * 4, rsub = lane >> 3;
#pragma unroll
                for (int pass = 0; pass < kCols / 32; ++pass) {
                    const int c0 = n0 + pass * 32, nv = nend - c0;
                    if (nv <= 0) break;
#pragma unroll
                    for (int j = 0; j < 32; ++j) buf[lane * 33 + j] = __float_as_uint(acc[pass * 32 + j]);
                    __syncwarp();
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        const int row = 4 * k + rsub;
                        const int64_t rbr = __shfl_sync(0xffffffffu, rb, row);
                        const int ok = __shfl_sync(0xffffffffu, mrow, row);
                        if (ok && cq < nv) {
                            const uint32_t* b = buf + row * 33 + cq;
                            *reinterpret_cast<float4*>(Cf + rbr + c0 + cq) =
                                make_float4(__uint_as_float(b[0]), __uint_as_float(b[1]), __uint_as_float(b[2]),
                                            __uint_as_float(b[3]));
                        }
                    }
                    __syncwarp();
                }
            } else if (t.c_f32) {
                float* Cf = reinterpret_cast<float*>(C);
#pragma unroll
                for (int pass = 0; pass < kCols / 32; ++pass) {
                    const int c0 = n0 + pass * 32, nv = nend - c0;
                    if (nv <= 0) break;
#pragma unroll
                    for (int j = 0; j < 32; ++j) buf[lane * 33 + j] = __float_as_uint(acc[pass * 32 + j]);
                    __syncwarp();
                    for (int r = 0; r < 32; ++r) {
                        const int64_t rbr = __shfl_sync(0xffffffffu, rb, r);
                        const int ok = __shfl_sync(0xffffffffu, mrow, r);
                        if (ok && lane < nv) Cf[rbr + c0 + lane] = __uint_as_float(buf[r * 33 + lane]);
                    }
                    __syncwarp();
                }
            } else {
#pragma unroll
                for (int pass = 0; pass < kCols / 16; ++pass) {
                    const int c0 = n0 + pass * 16, nv = nend - c0;
                    if (nv <= 0) break;
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        f32_to_f64_words(acc[pass * 16 + j], buf[lane * 33 + 2 * j + 1], buf[lane * 33 + 2 * j]);
                    }
                    __syncwarp();
                    // four rows per step, a lane two consecutive doubles of one
                    // row: one 16-byte store where the pair's address is on a
                    // 16-byte boundary (scattered rows start anywhere, and the
                    // output itself may start on any 8-byte boundary), else two
                    const int j0 = 2 * (lane & 7);
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        const int row = 4 * k + (lane >> 3);
                        const int64_t rbr = __shfl_sync(0xffffffffu, rb, row);
                        const int ok = __shfl_sync(0xffffffffu, mrow, row);
                        if (ok && j0 < nv) {
                            const uint32_t* b = buf + row * 33 + 2 * j0;
                            const double d0 = __hiloint2double((int)b[1], (int)b[0]);
                            const double d1 = __hiloint2double((int)b[3], (int)b[2]);
                            double* p = C + rbr + c0 + j0;
                            if (j0 + 1 < nv && (reinterpret_cast<uintptr_t>(p) & 15) == 0) {
                                *reinterpret_cast<double2*>(p) = make_double2(d0, d1);
                            } else {
                                p[0] = d0;
                                if (j0 + 1 < nv) p[1] = d1;
                            }
                        }
                    }
                    __syncwarp();
                }
            }
        }
    }
    __syncthreads();
    if (warp == 0) {
        ptx::tc_fence_after();
        ptx::tmem_dealloc(tmem, 512);
    }
}

template <int P, bool kFusedA>
void launch_p(const GemmTask* d_tasks, int ntasks, int total_tiles, const uint16_t* A, const uint16_t* B,
              double* C, int num_sms, int* err, cudaStream_t s, const int64_t* row_off, const GatherTile* atiles,
              const GatherSeg* asegs, const GatherTerm* aterms, const float* asrc) {
    static bool configured = false;
    if (!configured) {
        CUDA_CHECK(cudaFuncSetAttribute(gemm_tc_kernel<P, kFusedA>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        TcCfg<P>::kSmem));
        configured = true;
    }
    int grid = std::min(total_tiles, num_sms > 0 ? num_sms : 148);
    KScope ks(kFusedA ? "gemm_tc_bf16x6_w12" : (P == 3 ? "gemm_tc_bf16x6" : (P == 2 ? "gemm_tc_bf16x3" : "gemm_tc_bf16")),
              s);
    gemm_tc_kernel<P, kFusedA><<<grid, kFusedA ? kThreadsFused : kThreads, TcCfg<P>::kSmem, s>>>(
        d_tasks, ntasks, total_tiles, A, B, C, err, row_off, atiles, asegs, aterms, asrc);
}

// K-split reduction: block b sums rows [m0, m1) of one reduction R over its
// S partial slabs [S][M][N], in slab order, and writes them to the output rows
// (scattered by row_off, or at c_base + m ldc). float32 partials (the
// split-bfloat16 GEMM, itself accumulating in float32) are summed in float32
// and widened to float64 on the integer pipes; float64 partials in float64. A
// thread takes kE elements and issues their loads of one slab together, so a
// block waits S load latencies, not S times its element count.
template <class PartT>
__global__ void __launch_bounds__(256, 6) splitk_reduce(const SplitRed* __restrict__ reds,
                                                        const RedBlock* __restrict__ blocks,
                                                        const PartT* __restrict__ part, void* __restrict__ out,
                                                        const int64_t* __restrict__ row_off) {
    constexpr int kE = 8;
    const RedBlock b = blocks[blockIdx.x];
    const SplitRed R = reds[b.red];
    const int64_t mn = (int64_t)R.M * R.N;
    const int nel = (b.m1 - b.m0) * R.N;
    if (nel <= 0) return;
    const PartT* p0 = part + R.part + (int64_t)b.m0 * R.N;
    // (row, column) of this thread's first element and the step between its
    // elements (256 apart), without a division per element
    const int dm = 256 / R.N, dn = 256 - dm * R.N;
    for (int base = 0; base < nel; base += kE * 256) {
        PartT acc[kE];
#pragma unroll
        for (int i = 0; i < kE; ++i) acc[i] = PartT(0);
        for (int j = 0; j < R.S; ++j) {
            PartT v[kE];
#pragma unroll
            for (int i = 0; i < kE; ++i) {
                const int e = base + i * 256 + threadIdx.x;
                v[i] = e < nel ? __ldg(p0 + j * mn + e) : PartT(0);
            }
#pragma unroll
            for (int i = 0; i < kE; ++i) acc[i] += v[i];
        }
        // destinations are formed after the sums, so that they hold no
        // registers while the slices load (six blocks of 256 threads fit an SM)
        int ml = (base + (int)threadIdx.x) / R.N, n = base + (int)threadIdx.x - ml * R.N;
#pragma unroll
        for (int i = 0; i < kE; ++i) {
            const int e = base + i * 256 + threadIdx.x;
            if (e < nel) {
                const int m = b.m0 + ml;
                const int64_t d = R.use_roff ? __ldg(row_off + R.roff + m) + n : R.c_base + (int64_t)m * R.ldc + n;
                if (R.out_f32) static_cast<float*>(out)[d] = (float)acc[i];
                else if constexpr (std::is_same<PartT, float>::value) static_cast<double*>(out)[d] = f32_to_f64(acc[i]);
                else static_cast<double*>(out)[d] = acc[i];
            }
            ml += dm;
            n += dn;
            if (n >= R.N) { n -= R.N; ++ml; }
        }
    }
}

}  // namespace

void launch_gemm_tc(const GemmTask* d_tasks, int ntasks, int total_tiles, const uint16_t* A, const uint16_t* B,
                    double* C, int planes, int num_sms, int* err, cudaStream_t s, const int64_t* row_off) {
    if (total_tiles == 0) return;
    if (planes == 3)
        launch_p<3, false>(d_tasks, ntasks, total_tiles, A, B, C, num_sms, err, s, row_off, nullptr, nullptr, nullptr,
                           nullptr);
    else if (planes == 2)
        launch_p<2, false>(d_tasks, ntasks, total_tiles, A, B, C, num_sms, err, s, row_off, nullptr, nullptr, nullptr,
                           nullptr);
    else
        launch_p<1, false>(d_tasks, ntasks, total_tiles, A, B, C, num_sms, err, s, row_off, nullptr, nullptr, nullptr,
                           nullptr);
}

void launch_gemm_tc_fused(const GemmTask* d_tasks, int ntasks, int total_tiles, const GatherTile* atiles,
                          const GatherSeg* asegs, const GatherTerm* aterms, const float* asrc, const uint16_t* B,
                          double* C, int num_sms, int* err, cudaStream_t s, const int64_t* row_off) {
    if (total_tiles == 0) return;
    launch_p<3, true>(d_tasks, ntasks, total_tiles, nullptr, B, C, num_sms, err, s, row_off, atiles, asegs, aterms,
                      asrc);
}

}  // namespace tnh

namespace tnh {

std::vector<RedBlock> reduction_blocks(const std::vector<SplitRed>& reds) {
    std::vector<RedBlock> out;
    for (int r = 0; r < (int)reds.size(); ++r) {
        const int rpb = std::max(1, 2048 / std::max(1, reds[r].N));
        for (int m0 = 0; m0 < reds[r].M; m0 += rpb) out.push_back({r, m0, std::min(reds[r].M, m0 + rpb)});
    }
    return out;
}

void launch_splitk_reduce(const SplitRed* d_reds, const RedBlock* d_blocks, int nblocks, const float* part,
                          void* out, const int64_t* row_off, cudaStream_t s) {
    if (nblocks == 0) return;
    KScope ks("splitk_reduce", s);
    splitk_reduce<float><<<nblocks, 256, 0, s>>>(d_reds, d_blocks, part, out, row_off);
}

void launch_splitk_reduce(const SplitRed* d_reds, const RedBlock* d_blocks, int nblocks, const double* part,
                          void* out, const int64_t* row_off, cudaStream_t s) {
    if (nblocks == 0) return;
    KScope ks("splitk_reduce_f64", s);
    splitk_reduce<double><<<nblocks, 256, 0, s>>>(d_reds, d_blocks, part, out, row_off);
}

}  // namespace tnh
