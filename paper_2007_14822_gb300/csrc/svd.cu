// Truncated SVD of a block-sparse tensor (Sec. 5), float64 on the device.
//
// 1. Blocks are grouped by their row charge; each group is one dense matrix
//    M_Q (rows: the row-sector tuples of the group, columns: the column
//    tuples), as a combiner groups equal-QN sectors (Sec. 4).
// 2. Every M_Q is factorised by one-sided (Hestenes) Jacobi: the columns of
//    X = M_Q (or M_Q^T when it is wide) are rotated pairwise until all are
//    orthogonal, X V = U Sigma. Pairs follow the round-robin (circle)
//    schedule; one cooperative launch works on all groups at once, a warp
//    per column pair, with a bounded grid barrier between rounds. A group
//    stops after a full sweep without a rotation.
// 3. The singular values of all groups are pooled and ranked (sigma desc,
//    group, position); the cutoff/maxdim rule of Sec. 5 picks the kept count
//    (the only host synchronisation: it sizes the factors).
// 4. tnh_svd_get scatters U, S, V into the caller's block layouts.
#include <algorithm>
#include <cmath>
#include <map>

#include "prof.h"
#include "ptx.cuh"
#include "tnh_guard.h"
#include "tnh_internal.h"
#include "svd.h"

namespace tnh {

namespace {

struct JGroup {
    int64_t x_off;   // column-major X: n columns of length len
    int64_t v_off;   // column-major V: n x n
    int len, n;
    int rounds;      // rounds per sweep (n rounded up to even, minus one)
    int pair0;       // first global pair index
    int npairs;
};

struct GridBar {
    unsigned count;
    unsigned gen;
};

__device__ bool grid_barrier(GridBar* bar, unsigned nblocks, int* err) {
    __syncthreads();
    __shared__ int ok;
    if (threadIdx.x == 0) {
        ok = 1;
        volatile unsigned* vgen = &bar->gen;
        unsigned g = *vgen;
        __threadfence();
        if (atomicAdd(&bar->count, 1u) == nblocks - 1) {
            atomicExch(&bar->count, 0u);
            __threadfence();
            atomicAdd(&bar->gen, 1u);
        } else {
            const uint64_t t0 = ptx::gtimer_ns();
            unsigned it = 0;
            while (*vgen == g) {
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
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ int rr_pos(int j, int k, int R) { return j == 0 ? 0 : 1 + (j - 1 + k) % R; }

// state[0] = last round with any rotation (global), state[1] = rounds done
__global__ void jacobi_kernel(const JGroup* __restrict__ groups, int ngroups, int total_pairs, int max_rounds,
                              int rmax, double* __restrict__ X, double* __restrict__ V, int* __restrict__ last_rot,
                              int* state, GridBar* bar, int* err) {
    const int lane = threadIdx.x & 31;
    const int gw = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int nw = gridDim.x * (blockDim.x >> 5);
    const double tol = 1e-15;
    int t = 0;
    for (; t < max_rounds; ++t) {
        for (int pi = gw; pi < total_pairs; pi += nw) {
            int lo = 0, hi = ngroups - 1;
            while (lo < hi) {
                int mid = (lo + hi + 1) >> 1;
                if (groups[mid].pair0 <= pi) lo = mid; else hi = mid - 1;
            }
            const JGroup G = groups[lo];
            const int R = G.rounds;
            if (t - *(volatile int*)&last_rot[lo] > R) continue;        // converged
            const int i = pi - G.pair0;
            const int ne = R + 1;
            const int k = t % R;
            int p = rr_pos(i, k, R), q = rr_pos(ne - 1 - i, k, R);
            if (p >= G.n || q >= G.n) continue;
            double* xp = X + G.x_off + (int64_t)p * G.len;
            double* xq = X + G.x_off + (int64_t)q * G.len;
            double a = 0, b = 0, g = 0;
            for (int r = lane; r < G.len; r += 32) {
                double u = xp[r], v = xq[r];
                a = fma(u, u, a);
                b = fma(v, v, b);
                g = fma(u, v, g);
            }
            a = warp_sum(a);
            b = warp_sum(b);
            g = warp_sum(g);
            if (!(fabs(g) > tol * sqrt(a * b)) || a == 0.0 || b == 0.0) continue;
            const double zeta = (b - a) / (2.0 * g);
            const double tt = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
            const double c = 1.0 / sqrt(1.0 + tt * tt), s = c * tt;
            for (int r = lane; r < G.len; r += 32) {
                double u = xp[r], v = xq[r];
                xp[r] = c * u - s * v;
                xq[r] = s * u + c * v;
            }
            double* vp = V + G.v_off + (int64_t)p * G.n;
            double* vq = V + G.v_off + (int64_t)q * G.n;
            for (int r = lane; r < G.n; r += 32) {
                double u = vp[r], v = vq[r];
                vp[r] = c * u - s * v;
                vq[r] = s * u + c * v;
            }
            if (lane == 0) {
                atomicMax(&last_rot[lo], t);
                atomicMax(&state[0], t);
            }
        }
        if (!grid_barrier(bar, gridDim.x, err)) break;
        if (t - *(volatile int*)&state[0] > rmax) { ++t; break; }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) state[1] = t;
}

// sigma of every column; key for ranking
__global__ void column_norms(const JGroup* __restrict__ groups, int ngroups, const int* __restrict__ col0,
                             const double* __restrict__ X, double* __restrict__ sig, int* __restrict__ gid,
                             int* __restrict__ pos) {
    const int g = blockIdx.x;
    const JGroup G = groups[g];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int j = w; j < G.n; j += nw) {
        const double* x = X + G.x_off + (int64_t)j * G.len;
        double a = 0;
        for (int r = lane; r < G.len; r += 32) a = fma(x[r], x[r], a);
        a = warp_sum(a);
        if (lane == 0) {
            sig[col0[g] + j] = sqrt(a);
            gid[col0[g] + j] = g;
            pos[col0[g] + j] = j;
        }
    }
}

__device__ __forceinline__ bool key_before(double s1, int g1, int p1, double s2, int g2, int p2) {
    if (s1 != s2) return s1 > s2;
    if (g1 != g2) return g1 < g2;
    return p1 < p2;
}

// rank of every singular value in the pooled descending order
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

// Sec. 5 truncation on the sorted values: out[0] = kept, out_d[0] = truncerr
__global__ void trunc_select(const double* __restrict__ sig, const int* __restrict__ order, int n, double cutoff,
                             int maxdim, int mindim, int* __restrict__ out, double* __restrict__ out_d) {
    if (threadIdx.x != 0) return;
    double total = 0.0;
    for (int k = n - 1; k >= 0; --k) total += sig[order[k]] * sig[order[k]];
    int keep;
    double err = 0.0;
    if (n == 0) {
        keep = 0;
    } else if (total == 0.0) {
        keep = min(n, max(1, mindim));
    } else {
        // tail(k) = sum_{i >= k} s_i^2 / total, summed from the smallest
        keep = n;
        double acc = 0.0;
        for (int k = n; k >= 1; --k) {
            double s = sig[order[k - 1]];
            acc += s * s;
            if (acc / total <= cutoff) keep = k - 1;
            else break;
        }
        keep = max(keep, max(1, mindim));
        keep = min(keep, min(maxdim, n));
        keep = max(keep, max(min(mindim, n), 1));
        double tail = 0.0;
        for (int k = n - 1; k >= keep; --k) tail += sig[order[k]] * sig[order[k]];
        err = tail / total;
    }
    out[0] = keep;
    out_d[0] = err;
}

// copy one block of T into its group matrix (column-major X, maybe transposed)
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

__global__ void set_identity(const JGroup* __restrict__ groups, double* __restrict__ V) {
    const JGroup G = groups[blockIdx.y];
    const int64_t n2 = (int64_t)G.n * G.n;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n2; e += (int64_t)gridDim.x * blockDim.x)
        V[G.v_off + e] = (e / G.n == e % G.n) ? 1.0 : 0.0;
}

// scatter of the kept factors into caller blocks
struct SvdOut {
    int64_t dst;      // caller block offset
    int64_t x_off, v_off;
    int len, n, trans;
    int which;        // 0: U block (rows x kept), 1: V block (kept x cols)
    int rows, cols;   // U: block rows; V: block cols
    int off;          // roff (U) or coff (V) inside the group matrix
    int kept;         // kept in this group
    int perm0;        // first entry in the kept-column permutation
    int s0;           // first singular value of the group in S
};

// absorb: 0 none, 1 multiply S into U, 2 multiply S into V
__global__ void svd_scatter(const SvdOut* __restrict__ O, const int* __restrict__ perm, const double* __restrict__ X,
                            const double* __restrict__ V, const double* __restrict__ sk, int absorb,
                            double* __restrict__ U, double* __restrict__ Vt) {
    const SvdOut o = O[blockIdx.y];
    const int64_t n = (int64_t)(o.which == 0 ? o.rows : o.cols) * o.kept;
    const bool into_this = (o.which == 0 && absorb == 1) || (o.which == 1 && absorb == 2);
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        int k, idx;
        if (o.which == 0) { idx = (int)(e / o.kept); k = (int)(e - (int64_t)idx * o.kept); }
        else { k = (int)(e / o.cols); idx = (int)(e - (int64_t)k * o.cols); }
        const int j = perm[o.perm0 + k];             // source column in the group
        const double sv = sk[o.s0 + k];
        const int g = o.off + idx;                   // row (U) or column (V) of M_Q
        const bool from_x = (o.which == 0) ? !o.trans : o.trans;
        double v;
        if (from_x) {
            // rotated column j of X is sigma_j times a singular vector
            const double x = X[o.x_off + (int64_t)j * o.len + g];
            v = into_this ? x : (sv > 0 ? x / sv : 0.0);
        } else {
            const double x = V[o.v_off + (int64_t)j * o.n + g];
            v = into_this ? x * sv : x;
        }
        if (o.which == 0) U[o.dst + e] = v;
        else Vt[o.dst + e] = v;
    }
}

__global__ void gather_s(const double* __restrict__ sig, const int* __restrict__ src, int n, double* __restrict__ S) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) S[i] = sig[src[i]];
}

}  // namespace

struct SvdResult {
    Ctx* ctx = nullptr;
    cudaStream_t stream = nullptr;
    int nrow = 0;
    Layout T;
    std::vector<std::vector<int>> gq;        // charge of each group
    std::vector<JGroup> groups;
    std::vector<int> trans;
    std::vector<std::vector<std::vector<int>>> rkeys, ckeys;
    std::vector<std::vector<int>> roff, coff;
    std::vector<int> col0;                   // first pooled sigma of each group
    DevBuf X, V, sig;
    int total = 0;
    // kept
    std::vector<int> kept_g;                 // kept per group
    std::vector<std::vector<int>> perm;      // kept columns per group (sigma desc)
    std::vector<int> sect_groups;            // groups with kept > 0, ascending charge
    double truncerr = 0.0;
    int nq = 0;
};

std::unique_ptr<SvdResult> run_svd(Ctx* ctx, const Layout& T, int nrow, double cutoff, int maxdim,
                                          int mindim) {
    cudaStream_t s = ctx->stream;
    const int r = T.rank();
    TNH_REQUIRE(nrow >= 1 && nrow < r, TNH_ERR_ARG, "svd_trunc: nrow %d of rank %d", nrow, r);
    TNH_REQUIRE(maxdim >= 1, TNH_ERR_ARG, "svd_trunc: maxdim %d", maxdim);
    auto R = std::make_unique<SvdResult>();
    R->ctx = ctx;
    R->stream = ctx->stream;
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
    int64_t xo = 0, vo = 0;
    int pairs = 0, tot = 0, rmax = 1;
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
            int n = 1;
            for (int i = 0; i < nrow; ++i) n *= T.inds[i].dim[e.first[i]];
            rows += n;
        }
        for (auto& e : ck) {
            e.second = cols;
            cks.push_back(e.first);
            co.push_back(cols);
            int n = 1;
            for (int i = nrow; i < r; ++i) n *= T.inds[i].dim[e.first[i - nrow]];
            cols += n;
        }
        const int tr = rows < cols ? 1 : 0;
        JGroup G{};
        G.len = tr ? cols : rows;
        G.n = tr ? rows : cols;
        G.x_off = xo;
        G.v_off = vo;
        G.rounds = std::max(1, G.n + (G.n & 1) - 1);
        G.pair0 = pairs;
        G.npairs = (G.n + 1) / 2;
        rmax = std::max(rmax, G.rounds);
        for (int b : kv.second) {
            auto key = T.key(b);
            SvdPack p{};
            p.src = T.off[b];
            p.dst = xo;
            int rn = 1, cn = 1;
            for (int i = 0; i < nrow; ++i) rn *= T.inds[i].dim[key[i]];
            for (int i = nrow; i < r; ++i) cn *= T.inds[i].dim[key[i]];
            p.rows = rn;
            p.cols = cn;
            p.roff = rk[std::vector<int>(key.begin(), key.begin() + nrow)];
            p.coff = ck[std::vector<int>(key.begin() + nrow, key.end())];
            p.len = G.len;
            p.trans = tr;
            packs.push_back(p);
        }
        xo += (int64_t)G.len * G.n;
        vo += (int64_t)G.n * G.n;
        pairs += G.npairs;
        R->col0.push_back(tot);
        tot += G.n;
        R->groups.push_back(G);
        R->trans.push_back(tr);
        R->gq.push_back(kv.first);
        R->rkeys.push_back(rks);
        R->ckeys.push_back(cks);
        R->roff.push_back(ro);
        R->coff.push_back(co);
    }
    R->total = tot;
    const int ng = (int)R->groups.size();
    if (ng == 0) return R;
    R->X.alloc((size_t)xo * 8);
    R->V.alloc((size_t)vo * 8);
    R->sig.alloc((size_t)tot * 8);
    CUDA_CHECK(cudaMemsetAsync(R->X.p, 0, (size_t)xo * 8, s));
    DevBuf d_groups = upload(R->groups, s);
    DevBuf d_packs = upload(packs, s);
    DevBuf d_col0 = upload(R->col0, s);
    { KScope ks_("svd_pack", s);
    svd_pack<<<dim3(16, (unsigned)packs.size()), 256, 0, s>>>(d_packs.as<SvdPack>(), T.data, R->X.as<double>());
    }
    { KScope ks_("set_identity", s);
    set_identity<<<dim3(16, ng), 256, 0, s>>>(d_groups.as<JGroup>(), R->V.as<double>());
    }
    // ---- Jacobi
    DevBuf d_last((size_t)ng * 4), d_state(16), d_bar(16);
    std::vector<int> minus1(ng, -1);
    CUDA_CHECK(cudaMemcpyAsync(d_last.p, minus1.data(), (size_t)ng * 4, cudaMemcpyHostToDevice, s));
    int st0[4] = {-1, 0, 0, 0};
    CUDA_CHECK(cudaMemcpyAsync(d_state.p, st0, 16, cudaMemcpyHostToDevice, s));
    CUDA_CHECK(cudaMemsetAsync(d_bar.p, 0, 16, s));
    int bpsm = 0;
    const int threads = 256;
    CUDA_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bpsm, jacobi_kernel, threads, 0));
    int want = (pairs + (threads / 32) - 1) / (threads / 32);
    int grid = std::max(1, std::min(want, std::max(1, bpsm) * ctx->num_sms));
    int max_rounds = 40 * rmax + 8;
    const JGroup* gp = d_groups.as<JGroup>();
    double* Xp = R->X.as<double>();
    double* Vp = R->V.as<double>();
    int* lastp = d_last.as<int>();
    int* statep = d_state.as<int>();
    GridBar* barp = d_bar.as<GridBar>();
    int* errp = ctx->d_flag.as<int>();
    void* args[] = {(void*)&gp, (void*)&ng, (void*)&pairs, (void*)&max_rounds, (void*)&rmax, (void*)&Xp,
                    (void*)&Vp, (void*)&lastp, (void*)&statep, (void*)&barp, (void*)&errp};
    {
        KScope ks("jacobi_svd", s);
        CUDA_CHECK(cudaLaunchCooperativeKernel((void*)jacobi_kernel, dim3(grid), dim3(threads), args, 0, s));
    }
    // ---- sigma, ranking, truncation
    DevBuf d_gid((size_t)tot * 4), d_pos((size_t)tot * 4), d_order((size_t)tot * 4), d_out(16), d_outd(16);
    { KScope ks_("column_norms", s);
    column_norms<<<ng, 256, 0, s>>>(gp, ng, d_col0.as<int>(), Xp, R->sig.as<double>(), d_gid.as<int>(),
                                     d_pos.as<int>());
    }
    { KScope ks_("rank_kernel", s);
    rank_kernel<<<(tot + 255) / 256, 256, 0, s>>>(R->sig.as<double>(), d_gid.as<int>(), d_pos.as<int>(), tot,
                                                  d_order.as<int>());
    }
    { KScope ks_("trunc_select", s);
    trunc_select<<<1, 32, 0, s>>>(R->sig.as<double>(), d_order.as<int>(), tot, cutoff, maxdim, mindim,
                                  d_out.as<int>(), d_outd.as<double>());
    }
    int keep = 0;
    int state_h[2];
    CUDA_CHECK(cudaMemcpyAsync(&keep, d_out.p, 4, cudaMemcpyDeviceToHost, s));
    CUDA_CHECK(cudaMemcpyAsync(&R->truncerr, d_outd.p, 8, cudaMemcpyDeviceToHost, s));
    CUDA_CHECK(cudaMemcpyAsync(state_h, d_state.p, 8, cudaMemcpyDeviceToHost, s));
    std::vector<int> order(tot), gid(tot), pos(tot);
    CUDA_CHECK(cudaMemcpyAsync(order.data(), d_order.p, (size_t)tot * 4, cudaMemcpyDeviceToHost, s));
    CUDA_CHECK(cudaMemcpyAsync(gid.data(), d_gid.p, (size_t)tot * 4, cudaMemcpyDeviceToHost, s));
    CUDA_CHECK(cudaMemcpyAsync(pos.data(), d_pos.p, (size_t)tot * 4, cudaMemcpyDeviceToHost, s));
    CUDA_CHECK(cudaStreamSynchronize(s));
    check_device_flag(ctx);
    TNH_REQUIRE(state_h[1] < max_rounds, TNH_ERR_NOT_CONVERGED,
                "svd_trunc: Jacobi did not converge in %d rounds", max_rounds);
    R->kept_g.assign(ng, 0);
    R->perm.assign(ng, {});
    for (int k = 0; k < keep; ++k) {
        int i = order[k];
        R->perm[gid[i]].push_back(pos[i]);
        R->kept_g[gid[i]]++;
    }
    for (int g = 0; g < ng; ++g)
        if (R->kept_g[g] > 0) R->sect_groups.push_back(g);
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
    std::vector<SvdOut> outs;
    std::vector<int> perm, sidx;
    for (int k = 0; k < ns; ++k) {
        const int g = R.sect_groups[k];
        const JGroup& G = R.groups[g];
        const int p0 = (int)perm.size();
        const int s0 = (int)sidx.size();
        for (int j : R.perm[g]) {
            perm.push_back(j);
            sidx.push_back(R.col0[g] + j);
        }
        for (size_t a = 0; a < R.rkeys[g].size(); ++a) {
            std::vector<int> key = R.rkeys[g][a];
            key.push_back(k);
            int b = U.find(key);
            TNH_REQUIRE(b >= 0, TNH_ERR_SHAPE, "svd_get: U layout lacks a block");
            SvdOut o{};
            o.dst = U.off[b];
            o.x_off = G.x_off;
            o.v_off = G.v_off;
            o.len = G.len;
            o.n = G.n;
            o.trans = R.trans[g];
            o.which = 0;
            int rn = 1;
            for (int i = 0; i < nrow; ++i) rn *= R.T.inds[i].dim[R.rkeys[g][a][i]];
            o.rows = rn;
            o.cols = 0;
            o.off = R.roff[g][a];
            o.kept = R.kept_g[g];
            o.perm0 = p0;
            o.s0 = s0;
            outs.push_back(o);
        }
        for (size_t a = 0; a < R.ckeys[g].size(); ++a) {
            std::vector<int> key{k};
            key.insert(key.end(), R.ckeys[g][a].begin(), R.ckeys[g][a].end());
            int b = Vl.find(key);
            TNH_REQUIRE(b >= 0, TNH_ERR_SHAPE, "svd_get: V layout lacks a block");
            SvdOut o{};
            o.dst = Vl.off[b];
            o.x_off = G.x_off;
            o.v_off = G.v_off;
            o.len = G.len;
            o.n = G.n;
            o.trans = R.trans[g];
            o.which = 1;
            int cn = 1;
            for (int i = nrow; i < r; ++i) cn *= R.T.inds[i].dim[R.ckeys[g][a][i - nrow]];
            o.rows = 0;
            o.cols = cn;
            o.off = R.coff[g][a];
            o.kept = R.kept_g[g];
            o.perm0 = p0;
            o.s0 = s0;
            outs.push_back(o);
        }
    }
    if (outs.empty()) return;
    DevBuf d_outs = upload(outs, s), d_perm = upload(perm, s), d_sidx = upload(sidx, s);
    // singular values in output order (sector, desc)
    DevBuf d_sk((size_t)std::max<size_t>(sidx.size(), 1) * 8);
    { KScope ks_("gather_s", s);
    gather_s<<<((int)sidx.size() + 255) / 256, 256, 0, s>>>(R.sig.as<double>(), d_sidx.as<int>(), (int)sidx.size(),
                                                            d_sk.as<double>());
    }
    { KScope ks_("svd_scatter", s);
    svd_scatter<<<dim3(8, (unsigned)outs.size()), 256, 0, s>>>(d_outs.as<SvdOut>(), d_perm.as<int>(),
                                                               R.X.as<double>(), R.V.as<double>(), d_sk.as<double>(),
                                                               absorb, U.data, Vl.data);
    }
    if (S)
        CUDA_CHECK(cudaMemcpyAsync(S, d_sk.p, sidx.size() * 8, cudaMemcpyDeviceToDevice, s));
    CUDA_CHECK(cudaStreamSynchronize(s));
    check_device_flag(ctx);
}

}  // namespace tnh

using namespace tnh;

extern "C" {

tnh_status tnh_svd_trunc(tnh_ctx* ctx, const tnh_tensor* T, int32_t nrow, double cutoff, int32_t maxdim,
                         int32_t mindim, tnh_svd** out) {
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    return guard(c, [&] {
        TNH_REQUIRE(c && out, TNH_ERR_ARG, "tnh_svd_trunc: NULL argument");
        CUDA_CHECK(cudaSetDevice(c->device));
        auto R = run_svd(c, parse_tensor(T, "T"), nrow, cutoff, maxdim, mindim);
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

namespace tnh {

SvdResult* svd_run(Ctx* ctx, const Layout& T, int nrow, double cutoff, int maxdim, int mindim) {
    return run_svd(ctx, T, nrow, cutoff, maxdim, mindim).release();
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
