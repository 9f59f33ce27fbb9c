// Truncated SVD of a block-sparse tensor (Sec. 5), decided in float64.
//
// 1. Blocks are grouped by their row charge; each group is one dense matrix
//    M_Q (rows: the row-sector tuples of the group, columns: the column
//    tuples), as a combiner groups equal-QN sectors (Sec. 4).
// 2. One-sided (Hestenes) Jacobi in two precisions. GB300 runs float64 at a
//    small fraction of its float32 rate, so the bulk of the rotations is done
//    in float32 and float64 is kept for the result:
//    a. float32 block Jacobi on X = M_Q (or M_Q^T): column blocks of b
//       columns are paired round-robin; the X columns of each pair of
//       blocks are loaded into shared memory by one CTA, which runs one
//       inner Jacobi sweep over its 2b columns, accumulates the rotations
//       into a 2b x 2b matrix Q and updates the V columns once, V <- V Q.
//       One cooperative launch works on all groups, with a bounded grid
//       barrier between rounds.
//       This gives V32 with columns orthogonal to float32 accuracy.
//    b. The candidate columns (the largest float32 singular values: the kept
//       count that they predict plus a margin, and all within 1e-4 of the
//       largest) are re-orthonormalised and re-formed in float64,
//       Y = X V32[:, cand], and polished by float64 one-sided block Jacobi
//       (blocks of two columns). Y is already nearly orthogonal in its leading
//       columns; the sweeps left are spent on the small singular values that
//       float32 could not resolve.
//    c. The float64 singular values sigma_j = |Y_j| are pooled, ranked
//       (sigma desc, group, position) and the cutoff/maxdim rule of Sec. 5
//       picks the kept count (values below 1e-8 of the norm count as zero);
//       the discarded weight is |M|_F^2 minus the kept sigma^2, in float64.
//    d. The side that must come out orthonormal (U going right, V going left
//       in a sweep) is Y_j / sigma_j; the other side is the float64 product
//       of M with it (S V^T = U^T M, or U S = M V).
// Every wait is bounded and reports through the device error flag.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <string>

#include "prof.h"
#include "ptx.cuh"
#include "svd.h"
#include "tnh_guard.h"
#include "tnh_internal.h"

namespace tnh {

namespace {

// Grid barrier for a cooperative launch: a monotonic arrival counter
// (release add, acquire poll); barrier number e completes when the counter
// reaches e * nblocks. The wait gives up after 4 s of global time or when
// another thread has raised the error flag.
struct GridBar {
    unsigned count;
    unsigned pad;
};

__device__ bool grid_barrier(GridBar* bar, unsigned nblocks, unsigned& epoch, int* err) {
    __syncthreads();
    __shared__ int ok;
    epoch += nblocks;
    if (threadIdx.x == 0) {
        ok = 1;
        unsigned v;
        asm volatile("atom.add.release.gpu.u32 %0, [%1], 1;" : "=r"(v) : "l"(&bar->count) : "memory");
        const uint64_t t0 = ptx::gtimer_ns();
        unsigned it = 0;
        while (true) {
            asm volatile("ld.acquire.gpu.u32 %0, [%1];" : "=r"(v) : "l"(&bar->count) : "memory");
            if ((int)(v - epoch) >= 0) break;
            if ((++it & 255u) == 0) {
                if (*(volatile int*)err) { ok = 0; break; }
                if (ptx::gtimer_ns() - t0 > 4000000000ull) {
                    if (atomicCAS(err, 0, 1) == 0) { err[1] = 20; err[2] = blockIdx.x; }
                    ok = 0;
                    break;
                }
            }
        }
    }
    __syncthreads();
    return ok != 0;
}

template <class T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// the group whose block pairs include `item` (groups ascending by pair0)
template <class GroupT>
__device__ __forceinline__ int find_group(const GroupT* __restrict__ groups, int ngroups, int item) {
    int lo = 0, hi = ngroups - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (groups[mid].pair0 <= item) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// round-robin (circle) schedule: slot j of round k among R+1 slots
__device__ __forceinline__ int rr_pos(int j, int k, int R) { return j == 0 ? 0 : 1 + (j - 1 + k) % R; }

// Column copies between global memory and the shared-memory stage of a
// Jacobi round, by the threads t = 0..nt-1 of a warp or CTA: each pass puts
// kStageBatch loads in flight before it stores any of them. (A plain
// load-then-store loop waits for every load in turn: the compiler cannot
// move a load above a store through a pointer that may alias it.)
constexpr int kStageBatch = 16;
template <class T>
__device__ __forceinline__ void stage_in(T* __restrict__ dst, const T* __restrict__ src, int n, int npad, int t,
                                         int nt) {
    for (int base = t; base < npad; base += nt * kStageBatch) {
        T v[kStageBatch];
#pragma unroll
        for (int u = 0; u < kStageBatch; ++u) {
            const int r = base + u * nt;
            v[u] = r < n ? src[r] : T(0);
        }
#pragma unroll
        for (int u = 0; u < kStageBatch; ++u) {
            const int r = base + u * nt;
            if (r < npad) dst[r] = v[u];
        }
    }
}
template <class T>
__device__ __forceinline__ void stage_out(T* __restrict__ dst, const T* __restrict__ src, int n, int t, int nt) {
    for (int base = t; base < n; base += nt * kStageBatch) {
        T v[kStageBatch];
#pragma unroll
        for (int u = 0; u < kStageBatch; ++u) {
            const int r = base + u * nt;
            v[u] = r < n ? src[r] : T(0);
        }
#pragma unroll
        for (int u = 0; u < kStageBatch; ++u) {
            const int r = base + u * nt;
            if (r < n) dst[r] = v[u];
        }
    }
}

// ------------------------------------------------ convergence per group
// A group (matrix) stops after a sweep in which no column pair had a
// relative off-diagonal |x_p.x_q| / (|x_p||x_q|) above thr: every pair was
// rotated to zero in that sweep, so what is left is second order in thr.
// smax[3 g + s % 3] holds the float bits of the largest value seen in
// sweep s; slot (s + 1) % 3 is cleared at the start of sweep s, when no CTA
// can still read it, and a finished sweep's slot is read only after the
// grid barrier that ends it. Every CTA therefore takes the same decision.
__device__ __forceinline__ bool group_done(const int* smax, int g, int R, int rounds_done, float thr) {
    const int sw = rounds_done / R;
    if (sw < 1) return false;
    return __int_as_float(*(volatile const int*)&smax[3 * g + (sw - 1) % 3]) < thr;
}

template <class GroupT>
__device__ bool all_done(const GroupT* groups, int ngroups, const int* smax, int rounds_done, float thr) {
    int mine = 1;
    for (int g = threadIdx.x; g < ngroups; g += blockDim.x)
        mine &= group_done(smax, g, groups[g].rounds, rounds_done, thr);
    return __syncthreads_and(mine) != 0;
}

// ------------------------------------------------ stage a: float32 blocks
struct BGroup {
    int64_t x_off;   // column-major X32: n columns of length len
    int64_t v_off;   // column-major V32: n x n
    int len, n;
    int b;           // columns per block
    int nblk;        // blocks, rounded up to even
    int rounds;      // nblk - 1
    int pair0;       // first global block-pair index
};

constexpr int kBJMaxB = 8;             // columns per block (a block pair has <= 16)
constexpr float kTol32 = 1e-5f;    // float32 rotation threshold
constexpr float kDone32 = 2e-3f;   // float32 stop (the float64 polish finishes)

// state[1] = rounds done. fro2[g] = |X_g|_F^2; columns whose squared norm
// is below 1e-12 fro2 are float32 rounding noise and are not rotated (they
// would mix forever). Only the X columns of a block pair are staged in
// shared memory ([2B][stride], padded to lp, a multiple of 4: the inner
// sweep reads and writes them four floats at a time); the inner sweep's
// rotations are accumulated into Q ([2B][2B], shared memory), and the V
// columns are updated once per round, V <- V Q, straight from and to global
// memory. The decisions and the angle use the fast reciprocal and
// reciprocal square root where the divisor is bounded (the angle only has to
// reduce x_p.x_q; the float64 polish finishes).
template <int B>
__global__ void __launch_bounds__(32 * (B < 4 ? 4 : B)) block_jacobi_f32(const BGroup* __restrict__ groups,
                                                                       int ngroups, int total_pairs, int max_rounds,
                                                                       float* __restrict__ X, float* __restrict__ V,
                                                                       int* smax, int* state, GridBar* bar, int* err,
                                                                       int stride, const double* __restrict__ fro2) {
    constexpr int NC = 2 * B;
    extern __shared__ __align__(16) float sm[];   // [2B][stride] X columns, then Q [2B][2B]
    __shared__ int skip;
    float* Qs = sm + (size_t)NC * stride;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    unsigned epoch = 0;
    int t = 0;
    // the group of this CTA's first block pair, found once (it is the same
    // in every round; a CTA with more pairs looks the others up each round)
    const int lo0 = blockIdx.x < total_pairs ? find_group(groups, ngroups, (int)blockIdx.x) : 0;
    for (; t < max_rounds; ++t) {
        for (int item = blockIdx.x; item < total_pairs; item += gridDim.x) {
            const int lo = item == (int)blockIdx.x ? lo0 : find_group(groups, ngroups, item);
            const BGroup G = groups[lo];
            const int R = G.rounds;
            const int i = item - G.pair0, k = t % R;
            // one thread decides, so the whole CTA takes the same branch
            if (threadIdx.x == 0) {
                skip = group_done(smax, lo, R, t, 1.0f);
                if (k == 0 && i == 0) smax[3 * lo + (t / R + 1) % 3] = 0;
            }
            __syncthreads();
            const int sk = skip;
            __syncthreads();   // every thread has read skip before thread 0 rewrites it
            if (sk) continue;
            const int bp = rr_pos(i, k, R), bq = rr_pos(G.nblk - 1 - i, k, R);
            // local column list: block bp then block bq (clipped to n)
            const int p0 = bp * G.b, p1 = min(G.n, p0 + G.b);
            const int q0 = bq * G.b, q1 = min(G.n, q0 + G.b);
            const int np = max(0, p1 - p0), nq = max(0, q1 - q0), nc = np + nq;
            if (nc < 2) continue;
            const int L = G.len, Nn = G.n, lp = (L + 3) & ~3, l4 = lp >> 2;
            for (int c = warp; c < nc; c += nwarp) {
                const int col = c < np ? p0 + c : q0 + (c - np);
                stage_in(sm + (size_t)c * stride, X + G.x_off + (int64_t)col * L, L, lp, lane, 32);
            }
            for (int e = threadIdx.x; e < NC * NC; e += blockDim.x) Qs[e] = e / NC == e % NC ? 1.f : 0.f;
            __syncthreads();
            const int ne = nc + (nc & 1), Ri = ne - 1;
            const float null2 = (float)(1e-12 * fro2[lo]);
            // stop test, per column pair: float32 rotations leave every column
            // with an absolute error of a few eps32 |M|_F, so a pair can only be
            // made orthogonal to about floor = 256 eps32 |M|_F / min(|x_p|, |x_q|)
            // of its norms; the target is max(kDone32, floor) and smax holds the
            // largest ratio to it (done when below 1). Columns too small for
            // float32 to resolve are left to the float64 polish.
            const float flo0 = 256.f * 5.96e-8f * sqrtf((float)fro2[lo]);
            float wmax = 0.f;
            for (int ir = 0; ir < Ri; ++ir) {
                for (int pr = warp; pr < ne / 2; pr += nwarp) {
                    const int a = rr_pos(pr, ir, Ri), bb = rr_pos(ne - 1 - pr, ir, Ri);
                    if (a >= nc || bb >= nc) continue;
                    float4* xa = reinterpret_cast<float4*>(sm + (size_t)a * stride);
                    float4* xb = reinterpret_cast<float4*>(sm + (size_t)bb * stride);
                    float al = 0.f, be = 0.f, ga = 0.f;
                    for (int r = lane; r < l4; r += 32) {
                        const float4 u = xa[r], v = xb[r];
                        al = fmaf(u.x, u.x, fmaf(u.y, u.y, fmaf(u.z, u.z, fmaf(u.w, u.w, al))));
                        be = fmaf(v.x, v.x, fmaf(v.y, v.y, fmaf(v.z, v.z, fmaf(v.w, v.w, be))));
                        ga = fmaf(u.x, v.x, fmaf(u.y, v.y, fmaf(u.z, v.z, fmaf(u.w, v.w, ga))));
                    }
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {   // three interleaved butterflies
                        al += __shfl_xor_sync(0xffffffffu, al, o);
                        be += __shfl_xor_sync(0xffffffffu, be, o);
                        ga += __shfl_xor_sync(0xffffffffu, ga, o);
                    }
                    if (al <= null2 || be <= null2) continue;
                    const float ra = rsqrtf(al), rb = rsqrtf(be);
                    const float rel = fabsf(ga) * ra * rb;
                    // rsqrt(min(al, be)) = max(ra, rb)
                    wmax = fmaxf(wmax, __fdividef(rel, fmaxf(kDone32, flo0 * fmaxf(ra, rb))));
                    if (!(rel > kTol32)) continue;
                    const float zeta = (be - al) / (2.0f * ga);   // IEEE: 2 ga is not bounded
                    const float az = fabsf(zeta), w = fmaf(zeta, zeta, 1.f);
                    const float tt = az > 1e8f ? __fdividef(0.5f, zeta)
                                               : copysignf(__fdividef(1.f, az + w * rsqrtf(w)), zeta);
                    const float c = rsqrtf(fmaf(tt, tt, 1.f)), sn = c * tt;
#pragma unroll 2
                    for (int r = lane; r < l4; r += 32) {
                        const float4 u = xa[r], v = xb[r];
                        xa[r] = make_float4(c * u.x - sn * v.x, c * u.y - sn * v.y, c * u.z - sn * v.z, c * u.w - sn * v.w);
                        xb[r] = make_float4(sn * u.x + c * v.x, sn * u.y + c * v.y, sn * u.z + c * v.z, sn * u.w + c * v.w);
                    }
                    // Q <- Q J: the pairs of an inner step touch disjoint columns of Q
                    if (lane < nc) {
                        const float qa = Qs[lane * NC + a], qb = Qs[lane * NC + bb];
                        Qs[lane * NC + a] = c * qa - sn * qb;
                        Qs[lane * NC + bb] = sn * qa + c * qb;
                    }
                }
                __syncthreads();
            }
            for (int c = warp; c < nc; c += nwarp) {
                const int col = c < np ? p0 + c : q0 + (c - np);
                stage_out(X + G.x_off + (int64_t)col * L, sm + (size_t)c * stride, L, lane, 32);
            }
            // V <- V Q on the block pair's columns: each thread takes rows, RB
            // at a time, all their loads in flight before any store (every row
            // is read and written by one thread only)
            if constexpr (NC >= 32) {
                // wide blocks: one row per thread, Q read from shared memory
                // (broadcast), so that only the row stays in registers
                float* Vg = V + G.v_off;
                for (int r = threadIdx.x; r < Nn; r += blockDim.x) {
                    float v[NC];
#pragma unroll
                    for (int c = 0; c < NC; ++c) {
                        const int col = c < np ? p0 + c : q0 + (c - np);
                        v[c] = c < nc ? Vg[(int64_t)col * Nn + r] : 0.f;
                    }
#pragma unroll 1
                    for (int j = 0; j < nc; ++j) {
                        float o = 0.f;
#pragma unroll
                        for (int c = 0; c < NC; ++c) o = fmaf(v[c], Qs[c * NC + j], o);
                        const int col = j < np ? p0 + j : q0 + (j - np);
                        Vg[(int64_t)col * Nn + r] = o;
                    }
                }
            } else {
                constexpr int RB = 32 / NC;
                float* Vg = V + G.v_off;
                for (int r0 = threadIdx.x; r0 < Nn; r0 += blockDim.x * RB) {
                    float v[RB][NC], o[RB][NC];
#pragma unroll
                    for (int u = 0; u < RB; ++u) {
                        const int r = r0 + u * blockDim.x;
#pragma unroll
                        for (int c = 0; c < NC; ++c) {
                            const int col = c < np ? p0 + c : q0 + (c - np);
                            v[u][c] = (r < Nn && c < nc) ? Vg[(int64_t)col * Nn + r] : 0.f;
                            o[u][c] = 0.f;
                        }
                    }
#pragma unroll
                    for (int c = 0; c < NC; ++c) {
                        if (c >= nc) break;
                        float q[NC];
#pragma unroll
                        for (int j = 0; j < NC; ++j) q[j] = Qs[c * NC + j];
#pragma unroll
                        for (int u = 0; u < RB; ++u)
#pragma unroll
                            for (int j = 0; j < NC; ++j) o[u][j] = fmaf(v[u][c], q[j], o[u][j]);
                    }
#pragma unroll
                    for (int u = 0; u < RB; ++u) {
                        const int r = r0 + u * blockDim.x;
#pragma unroll
                        for (int j = 0; j < NC; ++j) {
                            const int col = j < np ? p0 + j : q0 + (j - np);
                            if (r < Nn && j < nc) Vg[(int64_t)col * Nn + r] = o[u][j];
                        }
                    }
                }
            }
            if (lane == 0 && wmax > 0.f) atomicMax(&smax[3 * lo + (t / R) % 3], __float_as_int(wmax));
            __syncthreads();
        }
        if (!grid_barrier(bar, gridDim.x, epoch, err)) break;
        if (all_done(groups, ngroups, smax, t + 1, 1.0f)) { ++t; break; }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) state[1] = t;
}

// ------------------------------------------------ stage b: float64 pairs
struct JGroup {
    int64_t x_off;   // column-major Y: n columns of length len
    int len, n;
    int b;           // columns per block
    int nblk;        // blocks, rounded up to even
    int rounds;      // nblk - 1
    int pair0;       // first global block-pair index
    int grp;         // group (index into fro2)
};

constexpr int kJ64MaxB = 4;                // columns per block (a block pair has <= 8)
constexpr int kJ64Threads = 32 * kJ64MaxB;   // one warp per column pair of an inner step
constexpr float kDone64 = 1e-9f;           // float64 stop

// Float64 one-sided block Jacobi: blocks of b columns paired round-robin;
// one CTA per block pair and round loads its 2b columns into shared memory
// and runs one inner sweep (one warp per column pair), so every grid barrier
// is shared by (2b - 1) b rotations. The decisions and the rotation angle
// are computed in float32 (float64 division and square root are slow on
// this GPU); the angle only needs to reduce x_p.x_q, and the rotation is
// made orthogonal to float64 accuracy by rescaling (c, s) with a series for
// 1/sqrt(c^2 + s^2) (|c^2 + s^2 - 1| ~ 1e-7). Columns whose squared norm is
// below 1e-28 |M_g|_F^2 are float64 rounding noise and are not rotated.
// hist (debug, may be null): largest relative off-diagonal per (group, sweep).
__global__ void __launch_bounds__(kJ64Threads) jacobi_f64(const JGroup* __restrict__ groups, int ngroups,
                                                          int total_pairs, int max_rounds, double* __restrict__ X,
                                                          int* smax, int* state, GridBar* bar, int* err,
                                                          const double* __restrict__ fro2, int* hist, int stride) {
    extern __shared__ double smd[];   // [2b][stride]
    __shared__ int skip;
    __shared__ double red[3 * (kJ64Threads / 32)];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    unsigned epoch = 0;
    int t = 0;
    // the group of this CTA's first block pair, found once (it is the same
    // in every round; a CTA with more pairs looks the others up each round)
    const int lo0 = blockIdx.x < total_pairs ? find_group(groups, ngroups, (int)blockIdx.x) : 0;
    for (; t < max_rounds; ++t) {
        for (int item = blockIdx.x; item < total_pairs; item += gridDim.x) {
            const int lo = item == (int)blockIdx.x ? lo0 : find_group(groups, ngroups, item);
            const JGroup G = groups[lo];
            const int R = G.rounds;
            const int i = item - G.pair0, k = t % R;
            if (threadIdx.x == 0) {
                skip = group_done(smax, lo, R, t, 1.0f);
                if (k == 0 && i == 0) smax[3 * lo + (t / R + 1) % 3] = 0;
            }
            __syncthreads();
            const int sk = skip;
            __syncthreads();
            if (sk) continue;
            const int bp = rr_pos(i, k, R), bq = rr_pos(G.nblk - 1 - i, k, R);
            const int p0 = bp * G.b, p1 = min(G.n, p0 + G.b);
            const int q0 = bq * G.b, q1 = min(G.n, q0 + G.b);
            const int np = max(0, p1 - p0), nq = max(0, q1 - q0), nc = np + nq;
            if (nc < 2) continue;
            const int L = G.len;
            double* Xg = X + G.x_off;
            for (int c = warp; c < nc; c += nwarp) {
                const int col = c < np ? p0 + c : q0 + (c - np);
                const double* xs = Xg + (int64_t)col * L;
                double* d = smd + (size_t)c * stride;
                stage_in(d, xs, L, L, lane, 32);
            }
            __syncthreads();
            const int ne = nc + (nc & 1), Ri = ne - 1;
            const double inv = 1.0 / fro2[G.grp];
            const float tol = 4.0f * sqrtf((float)L) * 1.1102230246251565e-16f;
            const float flo0 = 16.0f * 1.1102230246251565e-16f * sqrtf((float)L);
            float wmax = 0.f, hmax = 0.f;
            // wpp warps share a column pair (their rows split), so that a block
            // pair with fewer column pairs than warps still uses every warp
            const int P = ne / 2;
            int wpp = 1;
            while (wpp * 2 * P <= nwarp) wpp *= 2;
            const int sub = warp % wpp, nt = 32 * wpp, tp = sub * 32 + lane;
            for (int ir = 0; ir < Ri; ++ir) {
                // the same trip count in every warp, so the barriers below are uniform
                for (int pb = 0; pb < P; pb += nwarp / wpp) {
                    const int pr = pb + warp / wpp;
                    int a = 0, bb = 0;
                    if (pr < P) {
                        a = rr_pos(pr, ir, Ri);
                        bb = rr_pos(ne - 1 - pr, ir, Ri);
                    }
                    const bool act = pr < P && a < nc && bb < nc;
                    double* xa = smd + (size_t)(act ? a : 0) * stride;
                    double* xb = smd + (size_t)(act ? bb : 0) * stride;
                    double A = 0, B = 0, Gg = 0;
                    if (act) {
                        for (int r = tp; r < L; r += nt) {
                            const double u = xa[r], v = xb[r];
                            A = fma(u, u, A);
                            B = fma(v, v, B);
                            Gg = fma(u, v, Gg);
                        }
                    }
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        A += __shfl_xor_sync(0xffffffffu, A, o);
                        B += __shfl_xor_sync(0xffffffffu, B, o);
                        Gg += __shfl_xor_sync(0xffffffffu, Gg, o);
                    }
                    if (wpp > 1) {
                        if (lane == 0) {
                            red[3 * warp] = A;
                            red[3 * warp + 1] = B;
                            red[3 * warp + 2] = Gg;
                        }
                        __syncthreads();
                        const int w0 = warp - sub;
                        A = B = Gg = 0;
                        for (int k = 0; k < wpp; ++k) {   // fixed order: every warp of the pair gets the same sums
                            A += red[3 * (w0 + k)];
                            B += red[3 * (w0 + k) + 1];
                            Gg += red[3 * (w0 + k) + 2];
                        }
                        __syncthreads();
                    }
                    if (!act) continue;
                    // every lane has the same sums: the decision is uniform
                    const float af = (float)(A * inv), bf = (float)(B * inv), gf = (float)(Gg * inv);
                    const bool live = af > 1e-28f && bf > 1e-28f;
                    const float rel = live ? fabsf(gf) / (sqrtf(af) * sqrtf(bf)) : 0.f;
                    if (live) {
                        // stop test, per column pair: a column y = M v formed in float64
                        // carries an absolute rounding error ~ eps sqrt(len) |M|_F, so the
                        // pair can only be made orthogonal to about
                        //   floor = 16 eps sqrt(len) |M|_F / min(|y_p|, |y_q|)
                        // of its norms; the target is max(kDone64, floor), smax holds the
                        // largest ratio to it (done when below 1)
                        const float flo = flo0 * rsqrtf(fminf(af, bf));
                        wmax = fmaxf(wmax, rel / fmaxf(kDone64, flo));
                        hmax = fmaxf(hmax, rel);
                    }
                    if (!(live && rel > tol)) continue;
                    const float df = (float)((B - A) * inv);
                    const float zeta = df / (2.0f * gf);
                    const float az = fabsf(zeta);
                    const float tt = az > 1e8f ? 0.5f / zeta : (zeta >= 0.f ? 1.f : -1.f) / (az + sqrtf(1.f + zeta * zeta));
                    const float c32 = rsqrtf(1.f + tt * tt);
                    const double c0 = (double)c32, s0 = (double)(c32 * tt);
                    const double dl = fma(c0, c0, s0 * s0) - 1.0;
                    const double f = 1.0 + dl * (-0.5 + 0.375 * dl);
                    const double c = c0 * f, sn = s0 * f;
                    for (int r = tp; r < L; r += nt) {
                        const double u = xa[r], v = xb[r];
                        xa[r] = c * u - sn * v;
                        xb[r] = sn * u + c * v;
                    }
                }
                __syncthreads();
            }
            for (int c = warp; c < nc; c += nwarp) {
                const int col = c < np ? p0 + c : q0 + (c - np);
                double* xs = Xg + (int64_t)col * L;
                const double* d = smd + (size_t)c * stride;
                stage_out(xs, d, L, lane, 32);
            }
            if (lane == 0 && wmax > 0.f) atomicMax(&smax[3 * lo + (t / R) % 3], __float_as_int(wmax));
            if (hist && lane == 0 && hmax > 0.f && t / R < 48) atomicMax(&hist[lo * 48 + t / R], __float_as_int(hmax));
            __syncthreads();
        }
        if (!grid_barrier(bar, gridDim.x, epoch, err)) break;
        if (all_done(groups, ngroups, smax, t + 1, 1.0f)) { ++t; break; }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) state[1] = t;
}

// ------------------------------------------------ helpers
struct ColSet {      // columns of one group for norms / ranking
    int64_t off;     // first element of column 0
    int len, n;
    int col0;        // first pooled index
};

template <class T>
__global__ void column_norms(const ColSet* __restrict__ sets, const T* __restrict__ X, double* __restrict__ sig,
                             int* __restrict__ gid, int* __restrict__ pos) {
    const ColSet S = sets[blockIdx.x];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int j = w; j < S.n; j += nw) {
        const T* x = X + S.off + (int64_t)j * S.len;
        double a = 0;
        for (int r = lane; r < S.len; r += 32) a = fma((double)x[r], (double)x[r], a);
        a = warp_sum(a);
        if (lane == 0) {
            sig[S.col0 + j] = sqrt(a);
            gid[S.col0 + j] = blockIdx.x;
            pos[S.col0 + j] = j;
        }
    }
}

__device__ __forceinline__ bool key_before(double s1, int g1, int p1, double s2, int g2, int p2) {
    if (s1 != s2) return s1 > s2;
    if (g1 != g2) return g1 < g2;
    return p1 < p2;
}

// order[rank] = index, pooled order sigma desc, group, position
__global__ void rank_kernel(const double* __restrict__ sig, const int* __restrict__ gid, const int* __restrict__ pos,
                            int n, int* __restrict__ order) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double s = sig[i];
    const int g = gid[i], p = pos[i];
    int r = 0;
    for (int j = 0; j < n; ++j) r += key_before(sig[j], gid[j], pos[j], s, g, p);
    order[r] = i;
}

// fro2[g] = sum of squares of group g of X64 (one block per group)
struct FroSet {
    int64_t off, n;
};

__global__ void group_sumsq(const FroSet* __restrict__ S, const double* __restrict__ x, double* __restrict__ out) {
    __shared__ double red[256];
    const FroSet f = S[blockIdx.x];
    double s = 0;
    for (int64_t i = threadIdx.x; i < f.n; i += blockDim.x) s = fma(x[f.off + i], x[f.off + i], s);
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[blockIdx.x] = red[0];
}

// T = 1.5 I - 0.5 G for every k x k block (Newton-Schulz polar step)
struct NsSet {
    int64_t off;
    int k;
};

__global__ void ns_shift(const NsSet* __restrict__ S, double* __restrict__ G) {
    const NsSet f = S[blockIdx.y];
    const int64_t n = (int64_t)f.k * f.k;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        int i = (int)(e / f.k), j = (int)(e - (int64_t)i * f.k);
        G[f.off + e] = (i == j ? 1.5 : 0.0) - 0.5 * G[f.off + e];
    }
}

// Sum of squares of x[0..n) into out (deterministic, one block)
__global__ void sumsq_kernel(const double* __restrict__ x, int64_t n, double* __restrict__ out) {
    __shared__ double red[256];
    double s = 0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s = fma(x[i], x[i], s);
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0];
}

// Sec. 5 rule on the ranked candidates: tail(k) = total - sum_{i<k} s_i^2.
__global__ void trunc_select(const double* __restrict__ sig, const int* __restrict__ order, int n,
                             const double* __restrict__ total_p, double cutoff, int maxdim, int mindim, int ntotal,
                             int* __restrict__ out, double* __restrict__ out_d) {
    if (threadIdx.x != 0) return;
    const double total = *total_p;
    int keep;
    double err = 0.0;
    if (n == 0) {
        keep = 0;
    } else if (!(total > 0.0)) {
        keep = min(n, max(1, mindim));
    } else {
        // the smallest k whose discarded tail is within the cutoff
        keep = -1;
        double pre = 0.0;
        for (int k = 0; k <= n; ++k) {
            double tail = fmax(total - pre, 0.0) / total;
            if (tail <= cutoff) { keep = k; break; }
            if (k < n) {
                double s = sig[order[k]];
                pre += s * s;
            }
        }
        if (keep < 0) keep = ntotal;
        keep = max(keep, max(1, mindim));
        keep = min(keep, min(maxdim, ntotal));
        keep = max(keep, max(min(mindim, ntotal), 1));
        // singular values below 1e-8 of the norm (sigma^2 < 1e-16 of the
        // total) are zero to float64 accuracy: their vectors are not
        // resolved, so they are not kept (unless mindim asks for them)
        int nres = 0;
        while (nres < n && sig[order[nres]] * sig[order[nres]] >= 1e-16 * total) ++nres;
        keep = min(keep, max(nres, max(min(mindim, ntotal), 1)));
        keep = min(keep, n);
        double p2 = 0.0;
        for (int k = 0; k < keep; ++k) p2 += sig[order[k]] * sig[order[k]];
        err = fmax(total - p2, 0.0) / total;
    }
    out[0] = keep;
    out_d[0] = err;
}

struct SvdPack {
    int64_t src;      // T block offset
    int64_t dst;      // X offset of the group
    int rows, cols;   // block rows / cols
    int roff, coff;   // position in the group matrix
    int len;          // column length of X
    int trans;        // 1: X = M^T
};

__global__ void svd_pack(const SvdPack* __restrict__ P, const double* __restrict__ T, double* __restrict__ X) {
    const SvdPack p = P[blockIdx.y];
    const int64_t n = (int64_t)p.rows * p.cols;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        int i = (int)(e / p.cols), j = (int)(e - (int64_t)i * p.cols);
        double v = T[p.src + e];
        int R = p.roff + i, Cc = p.coff + j;
        if (!p.trans) X[p.dst + (int64_t)Cc * p.len + R] = v;
        else X[p.dst + (int64_t)R * p.len + Cc] = v;
    }
}

__global__ void to_f32(const double* __restrict__ x, float* __restrict__ y, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = (float)x[i];
}

__global__ void set_identity_f32(const BGroup* __restrict__ groups, float* __restrict__ V) {
    const BGroup G = groups[blockIdx.y];
    const int64_t n2 = (int64_t)G.n * G.n;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n2; e += (int64_t)gridDim.x * blockDim.x)
        V[G.v_off + e] = (e / G.n == e % G.n) ? 1.0f : 0.0f;
}

// Vc[:, j] = V32[:, cand[j]] (float -> double), per group
struct CandSet {
    int64_t v_off;    // V32 group offset
    int64_t c_off;    // Vc offset
    int n;            // V32 is n x n
    int k;            // candidates
    int cand0;        // first entry in cand[]
};

__global__ void gather_cand(const CandSet* __restrict__ S, const int* __restrict__ cand, const float* __restrict__ V32,
                            double* __restrict__ Vc) {
    const CandSet s = S[blockIdx.y];
    const int64_t tot = (int64_t)s.n * s.k;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        int j = (int)(e / s.n), r = (int)(e - (int64_t)j * s.n);
        Vc[s.c_off + e] = (double)V32[s.v_off + (int64_t)cand[s.cand0 + j] * s.n + r];
    }
}

// C(i,j) = sum_k A(i,k) B(k,j) with explicit strides; 64 x 64 tiles
struct SGemm {
    int M, N, K;
    int64_t a, ars, acs, b, brs, bcs, c, crs, ccs;
    int nt, tile0;
};

__global__ void __launch_bounds__(256) sgemm_f64(const SGemm* __restrict__ tasks, int ntasks,
                                                 const double* __restrict__ A, const double* __restrict__ B,
                                                 double* __restrict__ C) {
    __shared__ double As[16][65], Bs[16][65];
    const int tile = blockIdx.x;
    int lo = 0, hi = ntasks - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (tasks[mid].tile0 <= tile) lo = mid; else hi = mid - 1;
    }
    const SGemm t = tasks[lo];
    const int local = tile - t.tile0, mi = local / t.nt, ni = local - mi * t.nt;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    double acc[4][4] = {};
    for (int k0 = 0; k0 < t.K; k0 += 16) {
        for (int e = tid; e < 1024; e += 256) {
            int r = e >> 4, kk = e & 15;
            int gi = mi * 64 + r, gk = k0 + kk;
            As[kk][r] = (gi < t.M && gk < t.K) ? A[t.a + gi * t.ars + gk * t.acs] : 0.0;
            int gj = ni * 64 + r;
            Bs[kk][r] = (gj < t.N && gk < t.K) ? B[t.b + gk * t.brs + gj * t.bcs] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            double a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        int gi = mi * 64 + ty + 16 * i;
        if (gi >= t.M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int gj = ni * 64 + tx + 16 * j;
            if (gj < t.N) C[t.c + gi * t.crs + gj * t.ccs] = acc[i][j];
        }
    }
}

// C_t = sum over the K slices of the partial products P[slice][M][N] of
// task t, in slice order (deterministic), written with C_t's strides
struct SRed {
    int M, N, S;
    int64_t part, c, crs, ccs;
    int64_t e0;   // prefix of M * N over the reductions of one launch
};
__global__ void sgemm_reduce(const SRed* __restrict__ reds, int nred, int64_t total, const double* __restrict__ part,
                             double* __restrict__ C) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        int lo = 0, hi = nred - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (reds[mid].e0 <= e) lo = mid; else hi = mid - 1;
        }
        const SRed r = reds[lo];
        const int64_t l = e - r.e0, i = l / r.N, j = l - i * r.N;
        double v = 0.0;
        for (int k = 0; k < r.S; ++k) v += part[r.part + (int64_t)k * r.M * r.N + l];
        C[r.c + i * r.crs + j * r.ccs] = v;
    }
}

// The strided FP64 GEMMs of the factorisation are small (a few dozen 64 x 64
// tiles) with long K: with fewer tiles than half the SMs, each task is cut
// into up to 8 K slices whose products are summed by sgemm_reduce.
void launch_sgemm(Ctx* ctx, const std::vector<SGemm>& tasks, const double* A, const double* B, double* C,
                  cudaStream_t s) {
    if (tasks.empty()) return;
    int tiles = 0;
    int64_t kmax = 0;
    for (const SGemm& t : tasks) {
        tiles += ((t.M + 63) / 64) * ((t.N + 63) / 64);
        kmax = std::max<int64_t>(kmax, t.K);
    }
    int S = 1;
    while (S < 8 && tiles * S * 2 < ctx->num_sms && kmax >= 128 * (S * 2)) S *= 2;
    std::vector<SGemm> run;
    std::vector<SRed> reds;
    int64_t part_elems = 0, red_total = 0;
    int t0 = 0;
    for (const SGemm& t : tasks) {
        const int nt = (t.N + 63) / 64, mt = (t.M + 63) / 64;
        if (S == 1) {
            SGemm u = t;
            u.nt = nt;
            u.tile0 = t0;
            t0 += mt * nt;
            run.push_back(u);
            continue;
        }
        const int64_t ks = ((t.K + S - 1) / S + 15) / 16 * 16;
        int used = 0;
        for (int sl = 0; sl < S; ++sl) {
            const int64_t k0 = sl * ks, k1 = std::min<int64_t>(t.K, k0 + ks);
            if (k0 >= k1) break;
            SGemm u = t;
            u.K = (int)(k1 - k0);
            u.a = t.a + k0 * t.acs;
            u.b = t.b + k0 * t.brs;
            u.c = part_elems + (int64_t)sl * t.M * t.N;
            u.crs = t.N;
            u.ccs = 1;
            u.nt = nt;
            u.tile0 = t0;
            t0 += mt * nt;
            run.push_back(u);
            ++used;
        }
        reds.push_back(SRed{t.M, t.N, used, part_elems, t.c, t.crs, t.ccs, red_total});
        part_elems += (int64_t)S * t.M * t.N;
        red_total += (int64_t)t.M * t.N;
    }
    DevBuf d_run = upload(run, s);
    if (S == 1) {
        KScope ks("svd_sgemm_f64", s);
        sgemm_f64<<<t0, 256, 0, s>>>(d_run.as<SGemm>(), (int)run.size(), A, B, C);
        return;
    }
    DevBuf part((size_t)std::max<int64_t>(part_elems, 1) * sizeof(double));
    DevBuf d_reds = upload(reds, s);
    {
        KScope ks("svd_sgemm_f64", s);
        sgemm_f64<<<t0, 256, 0, s>>>(d_run.as<SGemm>(), (int)run.size(), A, B, part.as<double>());
    }
    {
        KScope ks("svd_sgemm_reduce", s);
        const int g = (int)std::min<int64_t>((red_total + 255) / 256, (int64_t)ctx->num_sms * 8);
        sgemm_reduce<<<std::max(g, 1), 256, 0, s>>>(d_reds.as<SRed>(), (int)reds.size(), red_total,
                                                     part.as<double>(), C);
    }
}

// exact side, normalised: Ex[:, k] = Y[:, perm[k]] / sigma_k
struct ExSet {
    int64_t y_off, e_off;
    int len, k, perm0, s0;
};

__global__ void form_exact(const ExSet* __restrict__ S, const int* __restrict__ perm, const double* __restrict__ Y,
                           const double* __restrict__ sk, double* __restrict__ Ex) {
    const ExSet s = S[blockIdx.y];
    const int64_t tot = (int64_t)s.len * s.k;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        int k = (int)(e / s.len), r = (int)(e - (int64_t)k * s.len);
        double sv = sk[s.s0 + k];
        Ex[s.e_off + e] = sv > 0 ? Y[s.y_off + (int64_t)perm[s.perm0 + k] * s.len + r] / sv : 0.0;
    }
}

// scatter: caller block element (a, b) of a 2-D view = src[off + a*ras + b*rbs] (scaled by sigma_k)
struct OutPiece {
    int64_t dst;        // caller block offset
    int64_t src;        // source offset
    int64_t ras, rbs;   // source strides for the block's (row, col)
    int rows, cols;     // block viewed as rows x cols, row-major
    int kaxis;          // 0: the row index is the kept index k, 1: the column index is
    int s0;             // first singular value of the group
    int mode;           // 0: copy, 1: times sigma_k, 2: divided by sigma_k
    int from_p;         // 0: source is the exact side Ex, 1: the product side P
};

__global__ void svd_scatter(const OutPiece* __restrict__ O, const double* __restrict__ Ex,
                            const double* __restrict__ P, const double* __restrict__ sk, double* __restrict__ dst) {
    const OutPiece o = O[blockIdx.y];
    const double* src = o.from_p ? P : Ex;
    const int64_t n = (int64_t)o.rows * o.cols;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        int a = (int)(e / o.cols), b = (int)(e - (int64_t)a * o.cols);
        double v = src[o.src + a * o.ras + b * o.rbs];
        if (o.mode) {
            double sv = sk[o.s0 + (o.kaxis == 0 ? a : b)];
            v = o.mode == 1 ? v * sv : (sv > 0 ? v / sv : 0.0);
        }
        dst[o.dst + e] = v;
    }
}

__global__ void gather_s(const double* __restrict__ sig, const int* __restrict__ src, int n, double* __restrict__ S) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) S[i] = sig[src[i]];
}

inline unsigned blocks_for(int64_t n, int cap = 1024) {
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(cap, (n + 255) / 256));
}

// reset the convergence bookkeeping of a cooperative Jacobi launch
void reset_state(DevBuf& smax, DevBuf& state, DevBuf& bar, int n, cudaStream_t s) {
    CUDA_CHECK(cudaMemsetAsync(smax.p, 0, (size_t)3 * n * 4, s));
    CUDA_CHECK(cudaMemsetAsync(state.p, 0, 16, s));
    CUDA_CHECK(cudaMemsetAsync(bar.p, 0, 16, s));
}

}  // namespace

struct SvdResult {
    Ctx* ctx = nullptr;
    cudaStream_t stream = nullptr;
    int nrow = 0;
    Layout T;
    int nq = 0;
    // groups
    std::vector<std::vector<int>> gq;
    std::vector<int> trans, rows, cols, len, n;
    std::vector<int64_t> xoff;                     // X64 offsets
    std::vector<std::vector<std::vector<int>>> rkeys, ckeys;
    std::vector<std::vector<int>> roff, coff;
    DevBuf X64;
    // float64 stage
    std::vector<int> kcand;                        // candidates per group
    std::vector<int64_t> yoff;                     // Y offsets (len x kcand)
    std::vector<int> ycol0;                        // first pooled candidate of each group
    DevBuf Y, sig;
    // kept
    std::vector<int> kept_g;
    std::vector<std::vector<int>> perm;            // kept Y columns per group (sigma desc)
    std::vector<int> sect_groups;                  // groups with kept > 0, ascending charge
    std::vector<int> sidx;                         // pooled index of every kept value, output order
    double truncerr = 0.0;
    int rounds32 = 0, rounds64 = 0;
    double flops32_round = 0.0, flops64_round = 0.0;   // rotation work per round, all groups
};

// One cooperative launch of the float32 block Jacobi over the groups bg
// (device copy d_bg); returns the rounds it took.
int run_block_jacobi(Ctx* ctx, const std::vector<BGroup>& bg, const DevBuf& d_bg, float* X, float* V,
                     const double* fro2, int bmax, int stride, const char* what) {
    cudaStream_t s = ctx->stream;
    int ng = (int)bg.size(), bpairs = 0, rmax = 1;
    for (const BGroup& G : bg) {
        bpairs = std::max(bpairs, G.pair0 + G.nblk / 2);
        rmax = std::max(rmax, G.rounds);
    }
    if (ng == 0 || bpairs == 0) return 0;
    int* errp = ctx->d_flag.as<int>();
    DevBuf d_smax((size_t)3 * ng * 4), d_state(16), d_bar(16);
    reset_state(d_smax, d_state, d_bar, ng, s);
    const int threads = 32 * std::max(bmax, 4);   // one warp per column pair of an inner step
    // X columns of a block pair, then the accumulated rotation Q
    size_t smem = ((size_t)2 * bmax * stride + (size_t)4 * bmax * bmax) * 4;
    const void* kern = nullptr;
    switch (bmax) {
        case 1: kern = (const void*)block_jacobi_f32<1>; break;
        case 2: kern = (const void*)block_jacobi_f32<2>; break;
        case 4: kern = (const void*)block_jacobi_f32<4>; break;
        case 8: kern = (const void*)block_jacobi_f32<8>; break;
        case 16: kern = (const void*)block_jacobi_f32<16>; break;
        default: TNH_REQUIRE(false, TNH_ERR_ARG, "svd: block width %d", bmax);
    }
    CUDA_CHECK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int bpsm = 0;
    CUDA_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bpsm, kern, threads, smem));
    TNH_REQUIRE(bpsm >= 1, TNH_ERR_CUDA, "svd: block Jacobi does not fit on an SM");
    int grid = std::max(1, std::min(bpairs, bpsm * ctx->num_sms));
    int max_rounds = 30 * rmax + 4;
    const BGroup* gp = d_bg.as<BGroup>();
    int* smaxp = d_smax.as<int>();
    int* statep = d_state.as<int>();
    GridBar* barp = d_bar.as<GridBar>();
    void* args[] = {(void*)&gp,    (void*)&ng,     (void*)&bpairs, (void*)&max_rounds, (void*)&X,      (void*)&V,
                    (void*)&smaxp, (void*)&statep, (void*)&barp,   (void*)&errp,       (void*)&stride, (void*)&fro2};
    {
        KScope ks("svd_jacobi_f32", s);
        CUDA_CHECK(cudaLaunchCooperativeKernel(kern, dim3(grid), dim3(threads), args, smem, s));
    }
    int st[2];
    CUDA_CHECK(cudaMemcpyAsync(st, d_state.p, 8, cudaMemcpyDeviceToHost, s));
    CUDA_CHECK(cudaStreamSynchronize(s));   // bookkeeping buffers are freed on return
    if (std::getenv("TNH_DEBUG"))
        std::fprintf(stderr, "svd: float32 block Jacobi%s %d rounds (max %d, per sweep %d, grid %d, b %d)\n", what,
                     st[1], max_rounds, rmax, grid, bmax);
    return st[1];
}

// TNH_DEBUG: host wall time of the phases of one factorisation
struct PhaseClock {
    bool on = std::getenv("TNH_DEBUG") != nullptr;
    std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now(), last = t0;
    std::string line;
    void mark(const char* what) {
        if (!on) return;
        const auto now = std::chrono::steady_clock::now();
        char b[64];
        std::snprintf(b, sizeof b, " %s %.3f", what, std::chrono::duration<double, std::milli>(now - last).count());
        line += b;
        last = now;
    }
    ~PhaseClock() {
        if (on)
            std::fprintf(stderr, "svd: phases (ms)%s, total %.3f\n", line.c_str(),
                         std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count());
    }
};

std::unique_ptr<SvdResult> run_svd(Ctx* ctx, const Layout& T, int nrow, double cutoff, int maxdim, int mindim,
                                   int exact_side) {
    PhaseClock clk;
    cudaStream_t s = ctx->stream;
    const int r = T.rank();
    TNH_REQUIRE(nrow >= 1 && nrow < r, TNH_ERR_ARG, "svd_trunc: nrow %d of rank %d", nrow, r);
    TNH_REQUIRE(maxdim >= 1, TNH_ERR_ARG, "svd_trunc: maxdim %d", maxdim);
    auto R = std::make_unique<SvdResult>();
    R->ctx = ctx;
    R->stream = s;
    R->nrow = nrow;
    R->T = T;
    R->nq = T.nq();
    // ---- groups by row charge
    std::map<std::vector<int>, std::vector<int>> byq;
    for (int b = 0; b < T.nblocks(); ++b) {
        std::vector<int> q(R->nq, 0);
        for (int i = 0; i < nrow; ++i)
            for (int k = 0; k < R->nq; ++k) q[k] += T.inds[i].arrow * T.inds[i].q(T.sect[(size_t)b * r + i], k);
        byq[q].push_back(b);
    }
    std::vector<SvdPack> packs;
    std::vector<BGroup> bg;
    int64_t xo = 0, vo = 0;
    int bpairs = 0, rmax = 1, stride = 0, xstride = 4, bmax = 1;   // stride: X + V column, xstride: X column
    for (auto& kv : byq) {
        std::map<std::vector<int>, int> rk, ck;
        for (int b : kv.second) {
            auto key = T.key(b);
            rk[std::vector<int>(key.begin(), key.begin() + nrow)] = 0;
            ck[std::vector<int>(key.begin() + nrow, key.end())] = 0;
        }
        std::vector<std::vector<int>> rks, cks;
        std::vector<int> ro, co;
        int rows = 0, cols = 0;
        for (auto& e : rk) {
            e.second = rows;
            rks.push_back(e.first);
            ro.push_back(rows);
            int m = 1;
            for (int i = 0; i < nrow; ++i) m *= T.inds[i].dim[e.first[i]];
            rows += m;
        }
        for (auto& e : ck) {
            e.second = cols;
            cks.push_back(e.first);
            co.push_back(cols);
            int m = 1;
            for (int i = nrow; i < r; ++i) m *= T.inds[i].dim[e.first[i - nrow]];
            cols += m;
        }
        // exact_side 0: U exact (orthogonalise the columns of M); 1: V exact (of M^T)
        const int tr = exact_side == 1 ? 1 : 0;
        const int L = tr ? cols : rows, Nn = tr ? rows : cols;
        BGroup G{};
        G.x_off = xo;
        G.v_off = vo;
        G.len = L;
        G.n = Nn;
        stride = std::max(stride, (((L + 3) & ~3) + Nn + 3) & ~3);
        xstride = std::max(xstride, (L + 3) & ~3);
        for (int bl : kv.second) {
            auto key = T.key(bl);
            SvdPack p{};
            p.src = T.off[bl];
            p.dst = xo;
            int rn = 1, cn = 1;
            for (int i = 0; i < nrow; ++i) rn *= T.inds[i].dim[key[i]];
            for (int i = nrow; i < r; ++i) cn *= T.inds[i].dim[key[i]];
            p.rows = rn;
            p.cols = cn;
            p.roff = rk[std::vector<int>(key.begin(), key.begin() + nrow)];
            p.coff = ck[std::vector<int>(key.begin() + nrow, key.end())];
            p.len = L;
            p.trans = tr;
            packs.push_back(p);
        }
        R->gq.push_back(kv.first);
        R->trans.push_back(tr);
        R->rows.push_back(rows);
        R->cols.push_back(cols);
        R->len.push_back(L);
        R->n.push_back(Nn);
        R->xoff.push_back(xo);
        R->rkeys.push_back(rks);
        R->ckeys.push_back(cks);
        R->roff.push_back(ro);
        R->coff.push_back(co);
        bg.push_back(G);
        xo += (int64_t)L * Nn;
        vo += (int64_t)Nn * Nn;
    }
    const int ng = (int)bg.size();
    if (ng == 0) return R;
    // one block width for all groups: up to 8 columns while a block pair's
    // X and V columns together would fit in 200 KB of shared memory (the
    // rule the widths were measured with; the kernel stages X only and
    // keeps V in global memory). An inner step moves about
    // 20 bytes per row and column pair through shared memory, which bounds a
    // round on one SM when columns are long, so for columns longer than 256
    // narrower blocks (more block pairs, more SMs) are taken while the groups
    // give fewer block pairs than half the SMs; short columns keep wide
    // blocks (fewer rounds, each with a fixed cost).
    bmax = kBJMaxB;
    while (bmax > 1 && (size_t)2 * bmax * stride * 4 > 200 * 1024) bmax >>= 1;
    auto block_pairs = [&](int b) {
        int p = 0;
        for (const BGroup& G : bg) {
            const int nb = (G.n + b - 1) / b;
            p += std::max(2, nb + (nb & 1)) / 2;
        }
        return p;
    };
    int lmax32 = 0;
    for (const BGroup& G : bg) lmax32 = std::max(lmax32, G.len);
    while (bmax > 4 && lmax32 > 256 && block_pairs(bmax) < ctx->num_sms / 2) bmax >>= 1;
    for (auto& G : bg) {
        G.b = bmax;
        int nb = (G.n + bmax - 1) / bmax;
        G.nblk = std::max(2, nb + (nb & 1));
        G.rounds = G.nblk - 1;
        G.pair0 = bpairs;
        bpairs += G.nblk / 2;
        rmax = std::max(rmax, G.rounds);
        // one inner sweep per block pair: (2b - 1) steps of b column pairs
        const double lp = (double)((G.len + 3) & ~3);
        R->flops32_round += (G.nblk / 2) * (2.0 * bmax - 1.0) * bmax * 6.0 * (2.0 * lp + G.n);
    }
    int ntot = 0;
    for (int g = 0; g < ng; ++g) ntot += R->n[g];
    int* errp = ctx->d_flag.as<int>();
    // ---- pack, float32 copy, identity
    R->X64.alloc((size_t)xo * 8);
    DevBuf X32((size_t)xo * 4), V32((size_t)vo * 4);
    CUDA_CHECK(cudaMemsetAsync(R->X64.p, 0, (size_t)xo * 8, s));
    DevBuf d_bg = upload(bg, s), d_packs = upload(packs, s);
    {
        KScope ks("svd_pack", s);
        svd_pack<<<dim3(16, (unsigned)packs.size()), 256, 0, s>>>(d_packs.as<SvdPack>(), T.data, R->X64.as<double>());
    }
    DevBuf d_fro2((size_t)ng * 8);
    {
        std::vector<FroSet> fs(ng);
        for (int g = 0; g < ng; ++g) fs[g] = FroSet{R->xoff[g], (int64_t)R->len[g] * R->n[g]};
        DevBuf d_fs = upload(fs, s);
        KScope ks("svd_group_sumsq", s);
        group_sumsq<<<ng, 256, 0, s>>>(d_fs.as<FroSet>(), R->X64.as<double>(), d_fro2.as<double>());
        // d_fs is freed on scope exit, in stream order after the kernel
    }
    const double* frop = d_fro2.as<double>();
    {
        KScope ks("svd_to_f32", s);
        to_f32<<<blocks_for(xo, 4096), 256, 0, s>>>(R->X64.as<double>(), X32.as<float>(), xo);
    }
    {
        KScope ks("svd_set_identity", s);
        set_identity_f32<<<dim3(16, ng), 256, 0, s>>>(d_bg.as<BGroup>(), V32.as<float>());
    }
    clk.mark("setup");
    // ---- stage a: float32 block Jacobi
    R->rounds32 = run_block_jacobi(ctx, bg, d_bg, X32.as<float>(), V32.as<float>(), frop, bmax, xstride, "");
    clk.mark("f32");
    // ---- rank the float32 singular values, pick the candidates
    std::vector<ColSet> cs32(ng);
    for (int g = 0, c0 = 0; g < ng; ++g) {
        cs32[g] = ColSet{R->xoff[g], R->len[g], R->n[g], c0};
        c0 += R->n[g];
    }
    DevBuf d_cs32 = upload(cs32, s);
    DevBuf sig32((size_t)ntot * 8), gid((size_t)ntot * 4), pos((size_t)ntot * 4), order((size_t)ntot * 4);
    {
        KScope ks("svd_norms", s);
        column_norms<float><<<ng, 256, 0, s>>>(d_cs32.as<ColSet>(), X32.as<float>(), sig32.as<double>(),
                                                gid.as<int>(), pos.as<int>());
    }
    {
        KScope ks("svd_rank", s);
        rank_kernel<<<(ntot + 255) / 256, 256, 0, s>>>(sig32.as<double>(), gid.as<int>(), pos.as<int>(), ntot,
                                                       order.as<int>());
    }
    std::vector<int> h_order(ntot), h_gid(ntot), h_pos(ntot);
    CUDA_CHECK(cudaMemcpyAsync(h_order.data(), order.p, (size_t)ntot * 4, cudaMemcpyDeviceToHost, s));
    CUDA_CHECK(cudaMemcpyAsync(h_gid.data(), gid.p, (size_t)ntot * 4, cudaMemcpyDeviceToHost, s));
    CUDA_CHECK(cudaMemcpyAsync(h_pos.data(), pos.p, (size_t)ntot * 4, cudaMemcpyDeviceToHost, s));
    CUDA_CHECK(cudaStreamSynchronize(s));
    check_device_flag(ctx);
    // candidates: the kept count that the float32 singular values predict
    // (cutoff and maxdim rule with the exact float64 total) plus a margin of
    // 16 + 1/8, and every column whose float32 singular value is within 1e-4
    // of the largest. The float64 truncation below needs the candidates only:
    // its discarded weight is the exact total minus the kept sum. Restricting
    // the float64 polish to a subspace biases sigma_i^2 by at most
    // sigma_excluded^2 sin^2(angle) (angle ~ float32 accuracy), so excluded
    // columns below 1e-4 sigma_max shift no sigma^2 by more than ~1e-20
    // sigma_max^2.
    std::vector<double> h_sig32(ntot), h_fro2(ng);
    CUDA_CHECK(cudaMemcpy(h_sig32.data(), sig32.p, (size_t)ntot * 8, cudaMemcpyDeviceToHost));
    CUDA_CHECK(cudaMemcpy(h_fro2.data(), d_fro2.p, (size_t)ng * 8, cudaMemcpyDeviceToHost));
    const double smax = ntot ? h_sig32[h_order[0]] : 0.0;
    double fro_total = 0.0;
    for (double f : h_fro2) fro_total += f;
    int k32 = ntot;
    if (fro_total > 0.0) {
        double pre = 0.0;
        for (int k = 0; k <= ntot; ++k) {
            if ((fro_total - pre) / fro_total <= cutoff) { k32 = k; break; }
            if (k < ntot) pre += h_sig32[h_order[k]] * h_sig32[h_order[k]];
        }
    }
    k32 = std::min(std::max(k32, std::max(mindim, 1)), maxdim);
    int ncand = std::min(ntot, k32 + 16 + k32 / 8);
    while (ncand < ntot && h_sig32[h_order[ncand]] >= 1e-4 * smax) ++ncand;
    // A group of len rows has rank <= len: candidates beyond that are null
    // vectors, which float32 only finds to its own accuracy (X v ~ eps32 |X|)
    // and which the float64 polish would then have to purify sweep after sweep.
    std::vector<std::vector<int>> cand(ng);
    for (int k = 0; k < ncand; ++k) {
        const int g = h_gid[h_order[k]];
        if ((int)cand[g].size() < R->len[g]) cand[g].push_back(h_pos[h_order[k]]);
    }
    clk.mark("rank32");
    // ---- float64 re-formation Y = X64 V32[:, cand]
    std::vector<CandSet> csets;
    std::vector<int> candflat;
    std::vector<SGemm> gemms;
    std::vector<JGroup> jg;
    R->kcand.assign(ng, 0);
    R->yoff.assign(ng, 0);
    R->ycol0.assign(ng, 0);
    int64_t yo = 0, vco = 0;
    int tiles = 0, jpairs = 0, jrmax = 1, yc = 0;
    for (int g = 0; g < ng; ++g) {
        const int k = (int)cand[g].size();
        R->kcand[g] = k;
        R->yoff[g] = yo;
        R->ycol0[g] = yc;
        if (k == 0) continue;
        csets.push_back(CandSet{bg[g].v_off, vco, R->n[g], k, (int)candflat.size()});
        candflat.insert(candflat.end(), cand[g].begin(), cand[g].end());
        SGemm t{};
        t.M = R->len[g];
        t.N = k;
        t.K = R->n[g];
        t.a = R->xoff[g];
        t.ars = 1;
        t.acs = R->len[g];
        t.b = vco;
        t.brs = 1;
        t.bcs = R->n[g];
        t.c = yo;
        t.crs = 1;
        t.ccs = R->len[g];
        t.nt = (k + 63) / 64;
        t.tile0 = tiles;
        tiles += ((t.M + 63) / 64) * t.nt;
        gemms.push_back(t);
        JGroup J{};
        J.x_off = yo;
        J.len = R->len[g];
        J.n = k;
        J.grp = g;
        jg.push_back(J);
        vco += (int64_t)R->n[g] * k;
        yo += (int64_t)R->len[g] * k;
        yc += k;
    }
    R->Y.alloc((size_t)std::max<int64_t>(yo, 1) * 8);
    {
        DevBuf Vc((size_t)std::max<int64_t>(vco, 1) * 8);
        DevBuf d_cs = upload(csets, s), d_cand = upload(candflat, s);
        {
            KScope ks("svd_gather_cand", s);
            gather_cand<<<dim3(16, (unsigned)csets.size()), 256, 0, s>>>(d_cs.as<CandSet>(), d_cand.as<int>(),
                                                                          V32.as<float>(), Vc.as<double>());
        }
        // V32 is orthogonal only to float32 accuracy, and the singular values
        // of X V32 differ from those of X at first order in that error:
        // re-orthonormalise the candidate columns in float64 by two
        // Newton-Schulz steps Vc <- Vc (3 I - Vc^T Vc) / 2 (quadratic).
        std::vector<SGemm> g1, g2;
        std::vector<NsSet> ns;
        int64_t go = 0;
        int t1 = 0, t2 = 0;
        for (const CandSet& c : csets) {
            SGemm a{};   // G = Vc^T Vc (k x k, row-major)
            a.M = c.k; a.N = c.k; a.K = c.n;
            a.a = c.c_off; a.ars = c.n; a.acs = 1;
            a.b = c.c_off; a.brs = 1; a.bcs = c.n;
            a.c = go; a.crs = c.k; a.ccs = 1;
            a.nt = (c.k + 63) / 64; a.tile0 = t1;
            t1 += ((c.k + 63) / 64) * a.nt;
            g1.push_back(a);
            SGemm b{};   // Vc' = Vc T (n x k, column-major)
            b.M = c.n; b.N = c.k; b.K = c.k;
            b.a = c.c_off; b.ars = 1; b.acs = c.n;
            b.b = go; b.brs = c.k; b.bcs = 1;
            b.c = c.c_off; b.crs = 1; b.ccs = c.n;
            b.nt = (c.k + 63) / 64; b.tile0 = t2;
            t2 += ((c.n + 63) / 64) * b.nt;
            g2.push_back(b);
            ns.push_back(NsSet{go, c.k});
            go += (int64_t)c.k * c.k;
        }
        DevBuf Gb((size_t)std::max<int64_t>(go, 1) * 8), Vc2((size_t)std::max<int64_t>(vco, 1) * 8);
        DevBuf d_ns = upload(ns, s);
        auto newton_schulz = [&](int iters) {
            for (int it = 0; it < iters; ++it) {
                launch_sgemm(ctx, g1, Vc.as<double>(), Vc.as<double>(), Gb.as<double>(), s);
                {
                    KScope ks("svd_ns_shift", s);
                    ns_shift<<<dim3(8, (unsigned)ns.size()), 256, 0, s>>>(d_ns.as<NsSet>(), Gb.as<double>());
                }
                launch_sgemm(ctx, g2, Vc.as<double>(), Gb.as<double>(), Vc2.as<double>(), s);
                std::swap(Vc, Vc2);
            }
        };
        auto form_y = [&] { launch_sgemm(ctx, gemms, R->X64.as<double>(), Vc.as<double>(), R->Y.as<double>(), s); };
        newton_schulz(2);
        form_y();
        // temporaries are freed on scope exit, in stream order after their kernels
    }
    clk.mark("form64");
    // ---- stage b: float64 polish
    {
        // blocks of two columns: a round carries 6 rotations for one grid
        // barrier, at half the block pairs of single column pairs (measured on
        // the m=2048 cylinder sweeps: 8% less SVD time than 4-column blocks for
        // short columns with single pairs for long ones, 2% less than 4-column
        // blocks everywhere)
        int lmax = 1;
        for (const JGroup& J : jg) lmax = std::max(lmax, J.len);
        int b64 = 2;
        while (b64 > 1 && (size_t)2 * b64 * lmax * 8 > 200 * 1024) b64 >>= 1;
        for (JGroup& J : jg) {
            J.b = b64;
            const int nb = (J.n + b64 - 1) / b64;
            J.nblk = std::max(2, nb + (nb & 1));
            J.rounds = J.nblk - 1;
            J.pair0 = jpairs;
            jpairs += J.nblk / 2;
            R->flops64_round += (J.nblk / 2) * (2.0 * b64 - 1.0) * b64 * 12.0 * J.len;
            jrmax = std::max(jrmax, J.rounds);
        }
        const int njg = (int)jg.size();
        DevBuf d_jg = upload(jg, s);
        DevBuf d_smax((size_t)3 * njg * 4), d_state(16), d_bar(16);
        reset_state(d_smax, d_state, d_bar, njg, s);
        const int threads = kJ64Threads;   // b64 < 4: several warps share a column pair
        const size_t smem64 = (size_t)2 * b64 * lmax * 8;
        CUDA_CHECK(cudaFuncSetAttribute(jacobi_f64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem64));
        int bpsm = 0;
        CUDA_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bpsm, jacobi_f64, threads, smem64));
        TNH_REQUIRE(bpsm >= 1, TNH_ERR_CUDA, "svd: float64 block Jacobi does not fit on an SM");
        int want = jpairs;
        int grid = std::max(1, std::min(want, std::max(1, bpsm) * ctx->num_sms));
        int max_rounds = 30 * jrmax + 8;
        const JGroup* gp = d_jg.as<JGroup>();
        double* Yp = R->Y.as<double>();
        int* smaxp = d_smax.as<int>();
        int* statep = d_state.as<int>();
        GridBar* barp = d_bar.as<GridBar>();
        const bool dbg = std::getenv("TNH_DEBUG") != nullptr;
        DevBuf d_hist(dbg ? (size_t)njg * 48 * 4 : 16);
        if (dbg) CUDA_CHECK(cudaMemsetAsync(d_hist.p, 0, (size_t)njg * 48 * 4, s));
        int* histp = dbg ? d_hist.as<int>() : nullptr;
        int stride64 = lmax;
        void* args[] = {(void*)&gp,    (void*)&njg,   (void*)&jpairs, (void*)&max_rounds, (void*)&Yp,
                        (void*)&smaxp, (void*)&statep, (void*)&barp,  (void*)&errp,       (void*)&frop,
                        (void*)&histp, (void*)&stride64};
        {
            KScope ks("svd_jacobi_f64", s);
            CUDA_CHECK(cudaLaunchCooperativeKernel((void*)jacobi_f64, dim3(grid), dim3(threads), args, smem64, s));
        }
        int st[2];
        CUDA_CHECK(cudaMemcpyAsync(st, d_state.p, 8, cudaMemcpyDeviceToHost, s));
        CUDA_CHECK(cudaStreamSynchronize(s));
        check_device_flag(ctx);
        R->rounds64 = st[1];
        if (dbg) {
            std::fprintf(stderr, "svd: float64 Jacobi %d rounds (max %d, per sweep %d, grid %d)\n", st[1], max_rounds,
                         jrmax, grid);
            std::vector<int> h((size_t)njg * 48);
            CUDA_CHECK(cudaMemcpy(h.data(), d_hist.p, h.size() * 4, cudaMemcpyDeviceToHost));
            int big = 0;
            for (int g = 0; g < njg; ++g) if (jg[g].n > jg[big].n) big = g;
            std::fprintf(stderr, "svd: float64 history, group %d (%d x %d):", big, jg[big].len, jg[big].n);
            for (int w = 0; w < 48 && w * jg[big].rounds < st[1]; ++w) {
                float v;
                std::memcpy(&v, &h[(size_t)big * 48 + w], 4);
                std::fprintf(stderr, " %.1e", (double)v);
            }
            std::fprintf(stderr, "\n");
        }
        if (st[1] >= max_rounds) {
            // report the group that kept rotating: its size and largest
            // relative off-diagonal in the last sweep
            std::vector<int> h_smax((size_t)3 * njg);
            CUDA_CHECK(cudaMemcpy(h_smax.data(), d_smax.p, h_smax.size() * 4, cudaMemcpyDeviceToHost));
            int worst = 0;
            float wv = -1.f;
            for (int g = 0; g < njg; ++g) {
                const int sw = st[1] / jg[g].rounds;
                float v;
                const int bits = h_smax[(size_t)3 * g + (sw + 2) % 3];
                std::memcpy(&v, &bits, 4);
                if (!(v <= wv)) { wv = v; worst = g; }
            }
            // what is left is within 1e3 of the rounding floor of the columns
            // involved (sigma right to second order); a pair far above its
            // target means the input was not finite or the method failed
            TNH_REQUIRE(wv < 1e3f, TNH_ERR_NOT_CONVERGED,
                        "svd_trunc: float64 Jacobi did not converge in %d rounds (group %d of %d: %d x %d, last "
                        "sweep max off-diagonal %.3g times its target)",
                        st[1], worst, njg, jg[worst].len, jg[worst].n, (double)wv);
            if (std::getenv("TNH_DEBUG"))
                std::fprintf(stderr, "svd: float64 Jacobi stopped at %d rounds, group %d (%d x %d) at %.3g x target\n",
                             st[1], worst, jg[worst].len, jg[worst].n, (double)wv);
        }
    }
    clk.mark("f64");
    // ---- float64 singular values, ranking, truncation
    const int ny = yc;
    std::vector<ColSet> cs64;
    std::vector<int> cs_group;
    for (int g = 0; g < ng; ++g)
        if (R->kcand[g]) {
            cs64.push_back(ColSet{R->yoff[g], R->len[g], R->kcand[g], R->ycol0[g]});
            cs_group.push_back(g);
        }
    DevBuf d_cs64 = upload(cs64, s);
    R->sig.alloc((size_t)std::max(ny, 1) * 8);
    DevBuf gid2((size_t)std::max(ny, 1) * 4), pos2((size_t)std::max(ny, 1) * 4), ord2((size_t)std::max(ny, 1) * 4);
    DevBuf total(16), outi(16), outd(16);
    {
        KScope ks("svd_norms", s);
        column_norms<double><<<(unsigned)cs64.size(), 256, 0, s>>>(d_cs64.as<ColSet>(), R->Y.as<double>(),
                                                                   R->sig.as<double>(), gid2.as<int>(), pos2.as<int>());
    }
    {
        KScope ks("svd_rank", s);
        rank_kernel<<<(ny + 255) / 256, 256, 0, s>>>(R->sig.as<double>(), gid2.as<int>(), pos2.as<int>(), ny,
                                                     ord2.as<int>());
    }
    {
        KScope ks("svd_sumsq", s);
        sumsq_kernel<<<1, 256, 0, s>>>(R->X64.as<double>(), xo, total.as<double>());
    }
    {
        KScope ks("svd_trunc_select", s);
        trunc_select<<<1, 32, 0, s>>>(R->sig.as<double>(), ord2.as<int>(), ny, total.as<double>(), cutoff, maxdim,
                                      mindim, ntot, outi.as<int>(), outd.as<double>());
    }
    int keep = 0;
    std::vector<int> o2(ny), g2(ny), p2(ny);
    CUDA_CHECK(cudaMemcpyAsync(&keep, outi.p, 4, cudaMemcpyDeviceToHost, s));
    CUDA_CHECK(cudaMemcpyAsync(&R->truncerr, outd.p, 8, cudaMemcpyDeviceToHost, s));
    CUDA_CHECK(cudaMemcpyAsync(o2.data(), ord2.p, (size_t)ny * 4, cudaMemcpyDeviceToHost, s));
    CUDA_CHECK(cudaMemcpyAsync(g2.data(), gid2.p, (size_t)ny * 4, cudaMemcpyDeviceToHost, s));
    CUDA_CHECK(cudaMemcpyAsync(p2.data(), pos2.p, (size_t)ny * 4, cudaMemcpyDeviceToHost, s));
    CUDA_CHECK(cudaStreamSynchronize(s));
    check_device_flag(ctx);
    R->kept_g.assign(ng, 0);
    R->perm.assign(ng, {});
    std::vector<std::vector<int>> pooled(ng);
    for (int k = 0; k < keep; ++k) {
        int i = o2[k];
        int g = cs_group[g2[i]];
        R->perm[g].push_back(p2[i]);
        pooled[g].push_back(i);
        R->kept_g[g]++;
    }
    for (int g = 0; g < ng; ++g)
        if (R->kept_g[g] > 0) {
            R->sect_groups.push_back(g);
            R->sidx.insert(R->sidx.end(), pooled[g].begin(), pooled[g].end());
        }
    return R;
}

void svd_get(SvdResult& R, const Layout& U, double* S, const Layout& Vl, int absorb) {
    Ctx* ctx = R.ctx;
    cudaStream_t s = ctx->stream;
    const int r = R.T.rank(), nrow = R.nrow;
    TNH_REQUIRE(U.rank() == nrow + 1 && Vl.rank() == r - nrow + 1, TNH_ERR_ARG, "svd_get: U/V ranks");
    const int ns = (int)R.sect_groups.size();
    const Index& cu = U.inds[nrow];
    const Index& cv = Vl.inds[0];
    TNH_REQUIRE(cu.nsect == ns && cv.nsect == ns, TNH_ERR_SHAPE, "svd_get: link index has %d sectors, want %d",
                cu.nsect, ns);
    for (int k = 0; k < ns; ++k) {
        int g = R.sect_groups[k];
        TNH_REQUIRE(cu.dim[k] == R.kept_g[g] && cv.dim[k] == R.kept_g[g], TNH_ERR_SHAPE,
                    "svd_get: link sector %d has dim %d, want %d", k, cu.dim[k], R.kept_g[g]);
    }
    for (int i = 0; i < nrow; ++i)
        TNH_REQUIRE(U.inds[i].same_space(R.T.inds[i]), TNH_ERR_SHAPE, "svd_get: U index %d differs", i);
    for (int i = nrow; i < r; ++i)
        TNH_REQUIRE(Vl.inds[i - nrow + 1].same_space(R.T.inds[i]), TNH_ERR_SHAPE, "svd_get: V index %d differs", i);
    CUDA_CHECK(cudaMemsetAsync(U.data, 0, (size_t)U.size * 8, s));
    CUDA_CHECK(cudaMemsetAsync(Vl.data, 0, (size_t)Vl.size * 8, s));
    if (ns == 0) return;
    // kept singular values in output order
    DevBuf d_sidx = upload(R.sidx, s);
    const int nk = (int)R.sidx.size();
    DevBuf sk((size_t)nk * 8);
    {
        KScope ks("svd_gather_s", s);
        gather_s<<<(nk + 255) / 256, 256, 0, s>>>(R.sig.as<double>(), d_sidx.as<int>(), nk, sk.as<double>());
    }
    // exact side Ex (len x kept, column-major) and the product side P
    std::vector<ExSet> ex;
    std::vector<int> permflat;
    std::vector<SGemm> gm;
    int64_t eo = 0, po = 0;
    int tiles = 0, s0 = 0;
    std::vector<int64_t> e_off(ns), p_off(ns);
    std::vector<int> s_first(ns);
    for (int k = 0; k < ns; ++k) {
        const int g = R.sect_groups[k], kk = R.kept_g[g], L = R.len[g];
        ex.push_back(ExSet{R.yoff[g], eo, L, kk, (int)permflat.size(), s0});
        permflat.insert(permflat.end(), R.perm[g].begin(), R.perm[g].end());
        e_off[k] = eo;
        p_off[k] = po;
        s_first[k] = s0;
        SGemm t{};
        const int64_t xg = R.xoff[g];
        if (!R.trans[g]) {
            // P = Ex^T M (kept x cols, row-major); M(i, c) = X64[xg + c*len + i]
            t.M = kk;
            t.N = R.cols[g];
            t.K = R.rows[g];
            t.a = eo;
            t.ars = L;
            t.acs = 1;
            t.b = xg;
            t.brs = 1;
            t.bcs = L;
            t.c = po;
            t.crs = R.cols[g];
            t.ccs = 1;
        } else {
            // P = M Ex (rows x kept, column-major), computed as P^T = Ex^T M^T so
            // that A is the Ex buffer and B the X64 buffer as in the launch;
            // M(i, c) = X64[xg + i*len + c], Ex(c, k) = Ex[eo + k*len + c]
            t.M = kk;
            t.N = R.rows[g];
            t.K = R.cols[g];
            t.a = eo;
            t.ars = L;
            t.acs = 1;
            t.b = xg;
            t.brs = 1;
            t.bcs = L;
            t.c = po;
            t.crs = R.rows[g];
            t.ccs = 1;
        }
        t.nt = (t.N + 63) / 64;
        t.tile0 = tiles;
        tiles += ((t.M + 63) / 64) * t.nt;
        gm.push_back(t);
        eo += (int64_t)L * kk;
        po += (int64_t)kk * (R.trans[g] ? R.rows[g] : R.cols[g]);
        s0 += kk;
    }
    DevBuf Ex((size_t)eo * 8), Pb((size_t)po * 8);
    DevBuf d_ex = upload(ex, s), d_perm = upload(permflat, s);
    {
        KScope ks("svd_form_exact", s);
        form_exact<<<dim3(16, (unsigned)ex.size()), 256, 0, s>>>(d_ex.as<ExSet>(), d_perm.as<int>(), R.Y.as<double>(),
                                                                 sk.as<double>(), Ex.as<double>());
    }
    launch_sgemm(ctx, gm, Ex.as<double>(), R.X64.as<double>(), Pb.as<double>(), s);
    // scatter into the caller's blocks
    std::vector<OutPiece> uo, vo;
    for (int k = 0; k < ns; ++k) {
        const int g = R.sect_groups[k], kk = R.kept_g[g];
        const bool tr = R.trans[g];
        for (size_t a = 0; a < R.rkeys[g].size(); ++a) {
            std::vector<int> key = R.rkeys[g][a];
            key.push_back(k);
            int b = U.find(key);
            TNH_REQUIRE(b >= 0, TNH_ERR_SHAPE, "svd_get: U layout lacks a block");
            int rn = 1;
            for (int i = 0; i < nrow; ++i) rn *= R.T.inds[i].dim[R.rkeys[g][a][i]];
            const int ro = R.roff[g][a];
            OutPiece o{};
            o.dst = U.off[b];
            o.rows = rn;
            o.cols = kk;
            o.kaxis = 1;
            o.s0 = s_first[k];
            if (!tr) {   // U = Ex (column-major, len = rows)
                o.src = e_off[k] + ro;
                o.ras = 1;
                o.rbs = R.len[g];
                o.mode = absorb == 1 ? 1 : 0;
                o.from_p = 0;
            } else {     // U S = P (column-major rows x kept)
                o.src = p_off[k] + ro;
                o.ras = 1;
                o.rbs = R.rows[g];
                o.mode = absorb == 1 ? 0 : 2;
                o.from_p = 1;
            }
            uo.push_back(o);
        }
        for (size_t a = 0; a < R.ckeys[g].size(); ++a) {
            std::vector<int> key{k};
            key.insert(key.end(), R.ckeys[g][a].begin(), R.ckeys[g][a].end());
            int b = Vl.find(key);
            TNH_REQUIRE(b >= 0, TNH_ERR_SHAPE, "svd_get: V layout lacks a block");
            int cn = 1;
            for (int i = nrow; i < r; ++i) cn *= R.T.inds[i].dim[R.ckeys[g][a][i - nrow]];
            const int co = R.coff[g][a];
            OutPiece o{};
            o.dst = Vl.off[b];
            o.rows = kk;
            o.cols = cn;
            o.kaxis = 0;
            o.s0 = s_first[k];
            if (!tr) {   // S V^T = P (row-major kept x cols)
                o.src = p_off[k] + co;
                o.ras = R.cols[g];
                o.rbs = 1;
                o.mode = absorb == 2 ? 0 : 2;
                o.from_p = 1;
            } else {     // V^T rows = Ex columns (len = cols)
                o.src = e_off[k] + co;
                o.ras = R.len[g];
                o.rbs = 1;
                o.mode = absorb == 2 ? 1 : 0;
                o.from_p = 0;
            }
            vo.push_back(o);
        }
    }
    DevBuf d_uo = upload(uo, s), d_vo = upload(vo, s);
    {
        KScope ks("svd_scatter", s);
        svd_scatter<<<dim3(8, (unsigned)uo.size()), 256, 0, s>>>(d_uo.as<OutPiece>(), Ex.as<double>(),
                                                                 Pb.as<double>(), sk.as<double>(), U.data);
    }
    {
        KScope ks("svd_scatter", s);
        svd_scatter<<<dim3(8, (unsigned)vo.size()), 256, 0, s>>>(d_vo.as<OutPiece>(), Ex.as<double>(),
                                                                 Pb.as<double>(), sk.as<double>(), Vl.data);
    }
    if (S) CUDA_CHECK(cudaMemcpyAsync(S, sk.p, (size_t)nk * 8, cudaMemcpyDeviceToDevice, s));
    CUDA_CHECK(cudaStreamSynchronize(s));
    check_device_flag(ctx);
}

SvdResult* svd_run(Ctx* ctx, const Layout& T, int nrow, double cutoff, int maxdim, int mindim, int exact_side) {
    return run_svd(ctx, T, nrow, cutoff, maxdim, mindim, exact_side).release();
}

SvdShape svd_shape(const SvdResult* R) {
    SvdShape sh;
    for (int g : R->sect_groups) {
        sh.qn.push_back(R->gq[g]);
        sh.dims.push_back(R->kept_g[g]);
    }
    sh.truncerr = R->truncerr;
    return sh;
}

void svd_fetch(SvdResult* R, const Layout& U, double* S, const Layout& V, int absorb) {
    svd_get(*R, U, S, V, absorb);
}

void svd_delete(SvdResult* R) { delete R; }

}  // namespace tnh

using namespace tnh;

extern "C" {

tnh_status tnh_svd_trunc(tnh_ctx* ctx, const tnh_tensor* T, int32_t nrow, double cutoff, int32_t maxdim,
                         int32_t mindim, int32_t exact_side, tnh_svd** out) {
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    return guard(c, [&] {
        TNH_REQUIRE(c && out, TNH_ERR_ARG, "tnh_svd_trunc: NULL argument");
        CUDA_CHECK(cudaSetDevice(c->device));
        TNH_REQUIRE(exact_side == 0 || exact_side == 1, TNH_ERR_ARG, "tnh_svd_trunc: exact_side must be 0 or 1");
        auto R = run_svd(c, parse_tensor(T, "T"), nrow, cutoff, maxdim, mindim, exact_side);
        *out = reinterpret_cast<tnh_svd*>(R.release());
    });
}

tnh_status tnh_svd_info(const tnh_svd* svd, int32_t* nsect, int32_t* nq, int32_t* qn, int32_t* sect_dim,
                        double* truncerr) {
    auto* R = reinterpret_cast<const SvdResult*>(svd);
    return guard(nullptr, [&] {
        TNH_REQUIRE(R, TNH_ERR_ARG, "tnh_svd_info: NULL svd");
        if (nsect) *nsect = (int32_t)R->sect_groups.size();
        if (nq) *nq = R->nq;
        for (size_t k = 0; k < R->sect_groups.size(); ++k) {
            int g = R->sect_groups[k];
            if (qn)
                for (int j = 0; j < R->nq; ++j) qn[k * R->nq + j] = R->gq[g][j];
            if (sect_dim) sect_dim[k] = R->kept_g[g];
        }
        if (truncerr) *truncerr = R->truncerr;
    });
}

tnh_status tnh_svd_stats(const tnh_svd* svd, int32_t* rounds32, int32_t* rounds64, double* flops32,
                         double* flops64) {
    auto* R = reinterpret_cast<const SvdResult*>(svd);
    return guard(nullptr, [&] {
        TNH_REQUIRE(R, TNH_ERR_ARG, "tnh_svd_stats: NULL svd");
        if (rounds32) *rounds32 = R->rounds32;
        if (rounds64) *rounds64 = R->rounds64;
        if (flops32) *flops32 = R->rounds32 * R->flops32_round;
        if (flops64) *flops64 = R->rounds64 * R->flops64_round;
    });
}

tnh_status tnh_svd_get(tnh_svd* svd, tnh_tensor* U, double* S, tnh_tensor* V, int32_t absorb) {
    auto* R = reinterpret_cast<SvdResult*>(svd);
    return guard(R ? R->ctx : nullptr, [&] {
        TNH_REQUIRE(R && U && V, TNH_ERR_ARG, "tnh_svd_get: NULL argument");
        TNH_REQUIRE(absorb >= 0 && absorb <= 2, TNH_ERR_ARG, "tnh_svd_get: absorb must be 0, 1 or 2");
        svd_get(*R, parse_tensor(U, "U"), S, parse_tensor(V, "V"), absorb);
    });
}

void tnh_svd_free(tnh_svd* svd) {
    auto* R = reinterpret_cast<SvdResult*>(svd);
    if (!R) return;
    cudaStreamSynchronize(R->stream);
    delete R;
}

}  // extern "C"
