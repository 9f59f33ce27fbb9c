// Tile gather: build GEMM operand tiles from weighted sums of strided
// sub-blocks.
//
// Two CTAs own one 128-row x 64-column tile of a GEMM operand (K-major),
// 64 rows each. The tile is assembled in shared memory from its segments; a segment is a
// rectangle of the tile whose every element is
//     sum_j coef_j * src[off_j + r * rs_j + c * cs_j]
// (r, c relative to the segment). Elements covered by no segment are zero,
// so the tile is written whole and no operand buffer needs clearing.
//
// Uses in the effective-Hamiltonian plan: packing L and R (once per plan)
// and psi (every application) into GEMM operands, one term per segment: a
// transposing, format-converting copy whose reads run along the unit-stride
// direction.
//
// In the split formats all arithmetic is float32 (the operands end up as
// three bfloat16 parts, 24 significant bits); the float64 format keeps
// float64 arithmetic.
//
// The fused S2+S3 step (w12_kernel below) works per cell instead: every
// output sub-block of one (a'-sector, b-sector) pair is a weighted sum of
// the cell's T1 sub-blocks, weights = nonzero entries of the two-site MPO
// product W1*W2 (Sec. 7.2); a thread forms four consecutive columns of one
// row for every output, reading its inputs with 16-byte loads (a cell's
// inputs are reused through L1 across its outputs).
//
// Output formats: float64 rows (pitch ld) for the FP64 GEMM, or the split
// bfloat16 swizzled tiles (x = hi + mid + lo) of the tcgen05 GEMM.
#include <cuda_bf16.h>

#include <algorithm>
#include <type_traits>

#include "gather.h"
#include "prof.h"
#include "split.cuh"

namespace tnh {

namespace {

constexpr int kPitch = kGatherCols + 1;   // padded smem row (doubles)
// one CTA builds a quarter (32 rows) of a tile: four times the CTAs of one
// per tile, so that the few tiles of a ψ pack still fill the SMs
constexpr int kTileParts = 4;
constexpr int kPartRows = kGatherRows / kTileParts;
constexpr int kSmemBytes = kPartRows * kPitch * 8;

// x = hi + mid + lo, each part rounded to nearest bfloat16; float32
// arithmetic (exact residuals), the float64 units of this GPU being scarce
template <int P>
__device__ __forceinline__ void split_bf16(float x, uint16_t* part) {
    const __nv_bfloat16 hi = __float2bfloat16_rn(x);
    part[0] = __bfloat16_as_ushort(hi);
    if (P > 1) {
        const float r1 = x - __bfloat162float(hi);
        const __nv_bfloat16 mid = __float2bfloat16_rn(r1);
        part[1] = __bfloat16_as_ushort(mid);
        if (P > 2) part[2] = __bfloat16_as_ushort(__float2bfloat16_rn(r1 - __bfloat162float(mid)));
    }
}

// float64 rows: float64 arithmetic; split-bfloat16 tiles: float32
template <bool kF64>
struct Acc { using T = float; };
template <>
struct Acc<true> { using T = double; };

template <bool kF64>
__device__ __forceinline__ typename Acc<kF64>::T coef_of(const GatherTerm& g) {
    if constexpr (kF64) return g.coef; else return g.coef32;
}

// source element -> accumulation type; float64 sources are rounded to float32
// on the integer pipes
template <class AccT, class SrcT>
__device__ __forceinline__ AccT to_acc(SrcT x) {
    if constexpr (std::is_same<AccT, float>::value && std::is_same<SrcT, double>::value) return f64_to_f32_rn(x);
    else return (AccT)x;
}

// CTA kTileParts t + h builds rows [kPartRows h, kPartRows (h + 1)) of tile t.
// The split formats run seven CTAs per SM (32 registers; no spills for the
// float64 sources that the effective-Hamiltonian plan packs): more loads in
// flight for packs of many small tiles (the U(1)xU(1) Hubbard ψ, m = 4096:
// 43 -> 38 us).
template <class SrcT, bool kF64, int P>
__global__ void __launch_bounds__(256, kF64 ? 6 : 7) gather_kernel(const GatherTile* __restrict__ tiles,
                                                                   const GatherSeg* __restrict__ segs,
                                                                   const GatherTerm* __restrict__ terms,
                                                                   const OpGeom* __restrict__ geom,
                                                                   const SrcT* __restrict__ src,
                                                                   void* __restrict__ dst) {
    using AccT = typename Acc<kF64>::T;
    extern __shared__ double tile_raw[];
    AccT* tile_s = reinterpret_cast<AccT*>(tile_raw);   // [kPartRows][kPitch]
    const GatherTile T = tiles[blockIdx.x / kTileParts];
    const int h0 = (blockIdx.x % kTileParts) * kPartRows;   // first tile row of this CTA
    for (int e = threadIdx.x; e < kPartRows * kPitch; e += blockDim.x) tile_s[e] = AccT(0);
    __syncthreads();
    for (int si = T.seg0; si < T.seg1; ++si) {
        const GatherSeg S = segs[si];
        // rows of the segment inside this half
        const int rb = max(0, h0 - S.r0), re = min(S.nr, h0 + kPartRows - S.r0);
        if (rb >= re) continue;
        const int nr = re - rb;
        const int n = nr * S.nc;
        const bool cfast = terms[S.t0].cs == 1;
        // element e of the segment part is (row, column) = (e / nc, e % nc)
        // when the source runs along columns, else (e % nr, e / nr): with
        // minor = nc or nr, e = major * minor + minor index. A thread's
        // elements are blockDim.x apart, so it steps (major, minor) instead
        // of dividing per element.
        const int minor = cfast ? S.nc : nr;
        const int dmaj = (int)blockDim.x / minor, dmin = (int)blockDim.x - dmaj * minor;
        if (S.t1 - S.t0 == 1) {
            // one term (a copy): eight independent loads in flight per thread
            const GatherTerm g = terms[S.t0];
            const AccT cf = coef_of<kF64>(g);
            for (int e0 = threadIdx.x; e0 < n; e0 += 8 * blockDim.x) {
                int maj = e0 / minor, mnr = e0 - maj * minor;
                AccT v[8];
                int pos[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int e = e0 + u * blockDim.x;
                    const int r = (cfast ? maj : mnr) + rb, c = cfast ? mnr : maj;
                    pos[u] = e < n ? (S.r0 + r - h0) * kPitch + S.c0 + c : -1;
                    v[u] = e < n ? cf * to_acc<AccT>(src[g.off + (int64_t)r * g.rs + (int64_t)c * g.cs]) : AccT(0);
                    maj += dmaj;
                    mnr += dmin;
                    if (mnr >= minor) { mnr -= minor; ++maj; }
                }
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    if (pos[u] >= 0) tile_s[pos[u]] = v[u];
            }
            continue;
        }
        int maj = (int)threadIdx.x / minor, mnr = (int)threadIdx.x - maj * minor;
        for (int e = threadIdx.x; e < n; e += blockDim.x) {
            const int r = (cfast ? maj : mnr) + rb, c = cfast ? mnr : maj;
            AccT v = AccT(0);
            for (int j = S.t0; j < S.t1; ++j) {
                const GatherTerm& g = terms[j];
                v += coef_of<kF64>(g) * to_acc<AccT>(src[g.off + (int64_t)r * g.rs + (int64_t)c * g.cs]);
            }
            tile_s[(S.r0 + r - h0) * kPitch + S.c0 + c] = v;
            maj += dmaj;
            mnr += dmin;
            if (mnr >= minor) { mnr -= minor; ++maj; }
        }
    }
    __syncthreads();
    const OpGeom G = geom[T.task];
    if constexpr (kF64) {
        double* d = static_cast<double*>(dst) + G.base + ((int64_t)T.mi * kGatherRows + h0) * G.ld +
                    (int64_t)T.ki * kGatherCols;
        for (int e = threadIdx.x; e < kPartRows * kGatherCols; e += blockDim.x) {
            const int r = e / kGatherCols, c = e - r * kGatherCols;
            d[(int64_t)r * G.ld + c] = tile_s[r * kPitch + c];
        }
    } else {
        // tile (mi, ki) of a [mt][kt] grid of P-plane 128 x 64 tiles; the
        // 16-byte chunk j of row r holds k-group j ^ (r & 7) (128-byte swizzle)
        uint16_t* d = static_cast<uint16_t*>(dst) +
                      (G.base + (int64_t)T.mi * G.ld + T.ki) * (int64_t)(P * kTcTileElems);
        for (int ci = threadIdx.x; ci < kPartRows * 8; ci += blockDim.x) {
            const int rl = ci >> 3, j = ci & 7, r = h0 + rl;
            const int kg = j ^ (r & 7);
            const float* v = tile_s + rl * kPitch + kg * 8;
            uint32_t w[3][4];
#pragma unroll
            for (int hh = 0; hh < 4; ++hh) {
                uint16_t a[3], b[3];
                split_bf16<P>(v[2 * hh], a);
                split_bf16<P>(v[2 * hh + 1], b);
#pragma unroll
                for (int p = 0; p < P; ++p) w[p][hh] = (uint32_t)a[p] | ((uint32_t)b[p] << 16);
            }
#pragma unroll
            for (int p = 0; p < P; ++p)
                *reinterpret_cast<uint4*>(d + p * kTcTileElems + (r * 8 + j) * 8) =
                    make_uint4(w[p][0], w[p][1], w[p][2], w[p][3]);
        }
    }
}


// four consecutive source elements (16-byte aligned for float, 32 for double)
__device__ __forceinline__ void load4(const float* p, float* v) {
    const float4 x = __ldg(reinterpret_cast<const float4*>(p));
    v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
}
__device__ __forceinline__ void load4(const double* p, double* v) {
    const double2 x = __ldg(reinterpret_cast<const double2*>(p));
    const double2 y = __ldg(reinterpret_cast<const double2*>(p) + 1);
    v[0] = x.x; v[1] = x.y; v[2] = y.x; v[3] = y.y;
}

// outputs and terms of one cell staged in shared memory (cells with more read
// them from global memory)
constexpr int kW12StageOuts = 96;
constexpr int kW12StageTerms = 384;

template <class SrcT, bool kF64, int P>
__global__ void __launch_bounds__(kW12Threads) w12_kernel(const W12Cta* __restrict__ ctas,
                                                          const W12Cell* __restrict__ cells,
                                                          const W12In* __restrict__ ins,
                                                          const W12Out* __restrict__ outs,
                                                          const W12Term* __restrict__ terms,
                                                          const OpGeom* __restrict__ geom,
                                                          const SrcT* __restrict__ src, void* __restrict__ dst) {
    using AccT = typename Acc<kF64>::T;
    __shared__ W12Out s_out[kW12StageOuts];
    __shared__ W12Term s_term[kW12StageTerms];
    const W12Cta T = ctas[blockIdx.x];
    const W12Cell C = cells[T.cell];
    // the terms of a cell's outputs are contiguous, in output order
    const int tb = C.nout > 0 ? outs[C.out0].t0 : 0;
    const int nterm = C.nout > 0 ? outs[C.out0 + C.nout - 1].t1 - tb : 0;
    const bool staged = C.nout <= kW12StageOuts && nterm <= kW12StageTerms;
    if (staged) {
        for (int k = threadIdx.x; k < C.nout; k += blockDim.x) s_out[k] = outs[C.out0 + k];
        for (int k = threadIdx.x; k < nterm; k += blockDim.x) s_term[k] = terms[tb + k];
    }
    __syncthreads();
    const W12Out* po = staged ? s_out : outs + C.out0;
    const W12Term* pt = staged ? s_term : terms + tb;
    const int dbq = (C.Db + 3) >> 2;
    const int q = T.q0 + (int)threadIdx.x;
    if (q >= C.Da * dbq) return;
    const int r = q / dbq, c = (q - r * dbq) * 4;
    // one output: its four columns lie inside one K piece of the S4 operand
    // (padded to 4 columns): columns past Db are padding, written as zero
    auto store = [&](const W12Out& O, const AccT* v) {
        const OpGeom G = geom[O.task];
        const int row = O.row0 + r, col = O.col0 + c;
        if constexpr (kF64) {
            double* d = static_cast<double*>(dst) + G.base + (int64_t)row * G.ld + col;
#pragma unroll
            for (int u = 0; u < 4; ++u) d[u] = v[u];
        } else {
            uint16_t* d = static_cast<uint16_t*>(dst) +
                          (G.base + (int64_t)(row >> 7) * G.ld + (col >> 6)) * (int64_t)(P * kTcTileElems) +
                          swz(row & 127, col & 63);
            uint32_t w0[3], w1[3];
            split2<P>(v[0], v[1], w0);
            split2<P>(v[2], v[3], w1);
#pragma unroll
            for (int pl = 0; pl < P; ++pl)
                *reinterpret_cast<uint2*>(d + pl * kTcTileElems) = make_uint2(w0[pl], w1[pl]);
        }
    };
    // T1 rows are padded to multiples of 4 columns with zeros (S1 multiplies
    // zero rows of its psi operand there): four loads never leave the row's
    // padded segment. The cell's terms are walked in chunks of kB in their
    // stored order (each output's terms contiguous, output after output, at
    // least one per output): a chunk's loads are issued together even where
    // it spans several outputs (most outputs have one or two terms), and an
    // output is stored as soon as its last term is added. Each output's sum
    // runs in term order.
    constexpr int kB = 4;
    int o = 0;
    int oend = C.nout > 0 ? po[0].t1 - tb : 0;   // end of output o's terms, relative to tb
    AccT v[4] = {AccT(0), AccT(0), AccT(0), AccT(0)};
    for (int j0 = 0; j0 < nterm; j0 += kB) {
        const int nb = min(kB, nterm - j0);
        SrcT x[kB][4];
        AccT cf[kB];
#pragma unroll
        for (int u = 0; u < kB; ++u) {
            if (u < nb) {
                const W12Term& t = pt[j0 + u];
                load4(src + t.base + (int64_t)r * t.ld + c, x[u]);
                cf[u] = kF64 ? (AccT)t.coef : (AccT)t.coef32;
            }
        }
#pragma unroll
        for (int u = 0; u < kB; ++u) {
            if (u < nb) {
#pragma unroll
                for (int k = 0; k < 4; ++k) v[k] = fma(cf[u], (AccT)x[u][k], v[k]);
                if (j0 + u + 1 == oend) {
                    store(po[o], v);
                    v[0] = v[1] = v[2] = v[3] = AccT(0);
                    if (++o < C.nout) oend = po[o].t1 - tb;
                }
            }
        }
    }
}

template <class SrcT, bool kF64, int P>
void launch_w12_one(const W12Job& J, const OpGeom* geom, const SrcT* src, void* dst, cudaStream_t s) {
    w12_kernel<SrcT, kF64, P><<<(int)J.ctas.size(), kW12Threads, 0, s>>>(
        J.d_ctas.as<W12Cta>(), J.d_cells.as<W12Cell>(), J.d_ins.as<W12In>(), J.d_outs.as<W12Out>(),
        J.d_terms.as<W12Term>(), geom, src, dst);
}

template <class SrcT>
void launch_w12_t(const W12Job& J, const OpGeom* geom, const SrcT* src, void* dst, int planes, cudaStream_t s) {
    if (J.ctas.empty()) return;
    KScope ks("heff_w12", s);
    if (planes == 0) launch_w12_one<SrcT, true, 1>(J, geom, src, dst, s);
    else if (planes == 1) launch_w12_one<SrcT, false, 1>(J, geom, src, dst, s);
    else if (planes == 2) launch_w12_one<SrcT, false, 2>(J, geom, src, dst, s);
    else launch_w12_one<SrcT, false, 3>(J, geom, src, dst, s);
}

template <class SrcT, bool kF64, int P>
void launch_one(const GatherJob& J, const OpGeom* geom, const SrcT* src, void* dst, cudaStream_t s) {
    static bool configured = false;
    if (!configured) {
        CUDA_CHECK(cudaFuncSetAttribute(gather_kernel<SrcT, kF64, P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        kSmemBytes));
        configured = true;
    }
    gather_kernel<SrcT, kF64, P><<<kTileParts * J.ntiles, 256, kSmemBytes, s>>>(
        J.d_tiles.as<GatherTile>(), J.d_segs.as<GatherSeg>(), J.d_terms.as<GatherTerm>(), geom, src, dst);
}

template <class SrcT>
void launch_t(const GatherJob& J, const OpGeom* geom, const SrcT* src, void* dst, int planes, cudaStream_t s) {
    if (planes == 0) launch_one<SrcT, true, 1>(J, geom, src, dst, s);
    else if (planes == 1) launch_one<SrcT, false, 1>(J, geom, src, dst, s);
    else if (planes == 2) launch_one<SrcT, false, 2>(J, geom, src, dst, s);
    else launch_one<SrcT, false, 3>(J, geom, src, dst, s);
}

}  // namespace

void W12Job::upload_all(cudaStream_t s) {
    d_cells = upload(cells, s);
    d_ins = upload(ins, s);
    d_outs = upload(outs, s);
    d_terms = upload(terms, s);
    d_ctas = upload(ctas, s);
}

void launch_w12(const W12Job& J, const OpGeom* d_geom, const double* src, void* dst, int planes, cudaStream_t s) {
    launch_w12_t<double>(J, d_geom, src, dst, planes, s);
}

void launch_w12(const W12Job& J, const OpGeom* d_geom, const float* src, void* dst, int planes, cudaStream_t s) {
    launch_w12_t<float>(J, d_geom, src, dst, planes, s);
}

void GatherJob::upload_all(cudaStream_t s) {
    ntiles = (int)tiles.size();
    d_tiles = upload(tiles, s);
    d_segs = upload(segs, s);
    d_terms = upload(terms, s);
}

void launch_gather(const GatherJob& J, const OpGeom* d_geom, const double* src, void* dst, int planes,
                   cudaStream_t s, const char* name) {
    if (J.ntiles == 0) return;
    KScope ks(name, s);
    launch_t<double>(J, d_geom, src, dst, planes, s);
}

void launch_gather(const GatherJob& J, const OpGeom* d_geom, const float* src, void* dst, int planes,
                   cudaStream_t s, const char* name) {
    if (J.ntiles == 0) return;
    KScope ks(name, s);
    launch_t<float>(J, d_geom, src, dst, planes, s);
}

}  // namespace tnh
