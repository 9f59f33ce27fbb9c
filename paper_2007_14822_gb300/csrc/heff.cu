// Effective-Hamiltonian plan: y = H_eff . x for two-site DMRG (Sec. 7.2).
//
//   y[a',s1',s2',b'] = sum L[a,w,a'] W1[w,w1,s1,s1'] W2[w1,w2,s2,s2']
//                          R[b,w2,b'] x[a,s1,s2,b]
//
// One application is four launches on the plan's stream (plus one ordered
// reduction of float32 partial tiles after each GEMM that the autotuner
// splits along K), replayed from a CUDA graph after the first calls:
//   1. gather  x -> operand B of S1 (split-bfloat16 tiles or float64 rows)
//   2. S1      T1[(w,a'), (s1,s2,b)] = sum_a L[a,w,a'] x[a,s1,s2,b]: a grouped
//              GEMM with one task per a-sector (Sec. 9.4: blocks whose
//              contracted sectors agree)
//   3. MPO     T3[(s1',s2',a'), (w2,b)] = sum W12[w,s1,s2; w2,s1',s2'] T1:
//              the contractions with W1 and W2 (S2, S3) fused into one pass
//              through the two-site MPO product W12 = sum_w1 W1 W2; one CTA
//              stages the T1 sub-blocks of an (a'-sector, b-sector) pair once
//              and writes every T3 sub-block of that pair, directly as
//              operand A of S4
//   4. S4      y[(s1',s2',a'), b'] = sum_(w2,b) T3 R[b,w2,b']: a grouped GEMM
//              with one task per b'-sector whose epilogue writes every row
//              to its place in psi's block layout
// L and R are packed into GEMM operands when the plan is made: they are the
// same for every application of the Lanczos iteration. The plan keeps no
// reference to the caller's L, W1, W2, R.
//
// In the split-bfloat16 modes the tensor cores accumulate in float32, T1 is
// stored in float32 and the packing and MPO-step arithmetic is float32 (the
// operands are three bfloat16 parts: 24 significant bits). An FP64 plan uses
// the FP64 GEMM throughout. A split-mode plan can also apply in FP64 (for the
// final energy and residual), so it keeps the float64 operands of L and R too.
#include <algorithm>
#include <array>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <set>
#include <string>

#include "heff.h"
#include "prof.h"
#include "tnh_guard.h"

namespace tnh {

namespace {

enum : int64_t { La = 1, Lw = 2, Lap = 3, Ls1 = 4, Ls2 = 5, Lb = 6, Lw1 = 7, Ls1p = 8, Lw2 = 9, Ls2p = 10, Lbp = 11 };

int64_t rup(int64_t x, int64_t m) { return (x + m - 1) / m * m; }
int64_t cdiv(int64_t x, int64_t m) { return (x + m - 1) / m; }

Layout with_labels(Layout T, std::initializer_list<int64_t> labels) {
    int i = 0;
    for (int64_t l : labels) T.inds[i++].label = l;
    return T;
}

std::vector<int> add_flux(const std::vector<int>& a, const std::vector<int>& b) {
    std::vector<int> r(a.size());
    for (size_t k = 0; k < a.size(); ++k) r[k] = a[k] + b[k];
    return r;
}

void check_pair(const Index& a, const Index& b, const char* what) {
    TNH_REQUIRE(a.same_space(b), TNH_ERR_SHAPE, "heff_plan: %s: the two indices have different sectors", what);
    TNH_REQUIRE(a.arrow != b.arrow, TNH_ERR_ARROW, "heff_plan: %s: contracted indices have equal arrows", what);
}

// sector of element e of an index and its position inside the sector
std::pair<int, int> locate(const Index& ix, int64_t e) {
    int s = 0;
    while (s + 1 < ix.nsect && e >= ix.off[s + 1]) ++s;
    return {s, (int)(e - ix.off[s])};
}

std::vector<double> to_host(const Layout& T, cudaStream_t s) {
    std::vector<double> h((size_t)T.size);
    if (T.size) {
        CUDA_CHECK(cudaMemcpyAsync(h.data(), T.data, (size_t)T.size * sizeof(double), cudaMemcpyDeviceToHost, s));
        CUDA_CHECK(cudaStreamSynchronize(s));
    }
    return h;
}

// Nonzero entries of a rank-4 MPO tensor, global element numbers per index.
struct MpoEntry {
    int l, r, s, sp;
    double v;
};
std::vector<MpoEntry> mpo_entries(const Layout& W, cudaStream_t s) {
    std::vector<double> h = to_host(W, s);
    std::vector<MpoEntry> out;
    for (int b = 0; b < W.nblocks(); ++b) {
        int d[4];
        int64_t o[4];
        for (int i = 0; i < 4; ++i) {
            d[i] = W.bdim(b, i);
            o[i] = W.inds[i].off[W.sect[(size_t)b * 4 + i]];
        }
        int64_t e = W.off[b];
        for (int i0 = 0; i0 < d[0]; ++i0)
            for (int i1 = 0; i1 < d[1]; ++i1)
                for (int i2 = 0; i2 < d[2]; ++i2)
                    for (int i3 = 0; i3 < d[3]; ++i3, ++e)
                        if (h[(size_t)e] != 0.0)
                            out.push_back({(int)(o[0] + i0), (int)(o[1] + i1), (int)(o[2] + i2), (int)(o[3] + i3),
                                           h[(size_t)e]});
    }
    return out;
}

// ---- diagonal of H_eff (the preconditioner of the Davidson eigensolver)
//   diag[a,s1,s2,b] = sum_(w,w2) Ld[a,w] W12[(w,s1,s2) -> (w2,s1,s2)] Rd[b,w2]
// with Ld[a,w] = L[a,w,a] and Rd[b,w2] = R[b,w2,b].
struct EnvDiagSeg {
    int64_t src;     // block (S, w-sector, S) of L or R
    int D, Dw;       // its sector dimensions
    int64_t dst;     // element (row a_off, column w_off) of the dense [m][w] diagonal
    int ld;          // that array's row pitch (w total)
};
struct DiagBlock {
    int64_t off;                   // psi block
    int Da, d1, d2, Db;
    int a_off, b_off, s1_off, s2_off;
};
struct DiagTerm {
    int w, z;
    double c;
};

__global__ void env_diag_kernel(const EnvDiagSeg* __restrict__ segs, const double* __restrict__ E,
                                double* __restrict__ out) {
    const EnvDiagSeg g = segs[blockIdx.x];
    const int n = g.D * g.Dw;
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
        const int i = e / g.Dw, x = e - i * g.Dw;
        out[g.dst + (int64_t)i * g.ld + x] = E[g.src + ((int64_t)i * g.Dw + x) * g.D + i];
    }
}

__global__ void heff_diag_kernel(const DiagBlock* __restrict__ blocks, const int* __restrict__ tstart,
                                 const DiagTerm* __restrict__ terms, const double* __restrict__ Ld,
                                 const double* __restrict__ Rd, int wdim, int zdim, int d2tot,
                                 double* __restrict__ diag) {
    const DiagBlock B = blocks[blockIdx.y];
    const int64_t n = (int64_t)B.Da * B.d1 * B.d2 * B.Db;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        int64_t r = e;
        const int k = (int)(r % B.Db);
        r /= B.Db;
        const int u2 = (int)(r % B.d2);
        r /= B.d2;
        const int u1 = (int)(r % B.d1);
        const int i = (int)(r / B.d1);
        const int ss = (B.s1_off + u1) * d2tot + B.s2_off + u2;
        const double* lrow = Ld + (int64_t)(B.a_off + i) * wdim;
        const double* rrow = Rd + (int64_t)(B.b_off + k) * zdim;
        double acc = 0.0;
        for (int t = tstart[ss]; t < tstart[ss + 1]; ++t) acc = fma(terms[t].c, lrow[terms[t].w] * rrow[terms[t].z], acc);
        diag[B.off + e] = acc;
    }
}

// Collects the segments of one gather job and orders them by tile.
struct JobBuilder {
    struct Task { int64_t tile0; int mt, kt; };
    struct Pending { int64_t tile; GatherSeg s; };
    std::vector<Task> tasks;
    std::vector<Pending> segs;
    std::vector<GatherTerm> terms;
    int64_t ntiles = 0;

    void task(int64_t rows, int64_t K) {
        Task t{ntiles, (int)cdiv(rows, kGatherRows), (int)cdiv(K, kGatherCols)};
        tasks.push_back(t);
        ntiles += (int64_t)t.mt * t.kt;
    }
    // rows [row0, row0+nr) x cols [col0, col0+nc) of task t: element (r, c)
    // is sum over terms of coef * src[off + r rs + c cs]
    void rect(int t, int64_t row0, int64_t col0, int64_t nr, int64_t nc, const std::vector<GatherTerm>& tm,
              bool keep_empty = false) {
        if ((tm.empty() && !keep_empty) || nr <= 0 || nc <= 0) return;
        const Task& T = tasks[t];
        for (int64_t R = row0; R < row0 + nr;) {
            const int64_t mi = R / kGatherRows, Re = std::min(row0 + nr, (mi + 1) * kGatherRows);
            for (int64_t Cc = col0; Cc < col0 + nc;) {
                const int64_t ki = Cc / kGatherCols, Ce = std::min(col0 + nc, (ki + 1) * kGatherCols);
                GatherSeg s{(int)(R - mi * kGatherRows), (int)(Cc - ki * kGatherCols), (int)(Re - R), (int)(Ce - Cc),
                            (int)terms.size(), 0};
                for (const GatherTerm& g : tm)
                    terms.push_back({g.coef, g.off + (R - row0) * g.rs + (Cc - col0) * g.cs, g.rs, g.cs, g.coef32});
                s.t1 = (int)terms.size();
                segs.push_back({T.tile0 + mi * T.kt + ki, s});
                Cc = Ce;
            }
            R = Re;
        }
    }
    void finish(GatherJob& J, cudaStream_t s) {
        std::stable_sort(segs.begin(), segs.end(), [](const Pending& a, const Pending& b) { return a.tile < b.tile; });
        TNH_REQUIRE(terms.size() < (size_t)INT32_MAX && ntiles < INT32_MAX, TNH_ERR_SHAPE,
                    "heff_plan: gather job too large");
        J.tiles.clear();
        J.segs.clear();
        J.terms.clear();
        J.terms.reserve(terms.size());
        size_t k = 0;
        for (int t = 0; t < (int)tasks.size(); ++t) {
            for (int mi = 0; mi < tasks[t].mt; ++mi)
                for (int ki = 0; ki < tasks[t].kt; ++ki) {
                    const int64_t id = tasks[t].tile0 + (int64_t)mi * tasks[t].kt + ki;
                    GatherTile g{t, mi, ki, (int)J.segs.size(), 0};
                    for (; k < segs.size() && segs[k].tile == id; ++k) {
                        GatherSeg sg = segs[k].s;
                        const int t0 = (int)J.terms.size();
                        for (int j = sg.t0; j < sg.t1; ++j) J.terms.push_back(terms[(size_t)j]);
                        sg.t0 = t0;
                        sg.t1 = (int)J.terms.size();
                        J.segs.push_back(sg);
                    }
                    g.seg1 = (int)J.segs.size();
                    J.tiles.push_back(g);
                }
        }
        J.upload_all(s);
    }
};

// Collects the outputs of the fused S2+S3 step per cell (a'-sector, b-sector);
// the terms of one output that read the same T1 sub-block are merged.
struct CellBuilder {
    struct Term { int64_t base, ld; double coef; };
    struct Out { int task; int64_t row0, col0; std::vector<Term> terms; };
    struct Cell { int Da = 0, Db = 0; std::vector<Out> outs; };
    std::map<std::pair<int, int>, Cell> cells;

    void add(int Ap, int B, int Da, int Db, int task, int64_t row0, int64_t col0, std::vector<Term> tm) {
        if (tm.empty()) return;
        Cell& c = cells[{Ap, B}];
        c.Da = Da;
        c.Db = Db;
        c.outs.push_back({task, row0, col0, std::move(tm)});
    }
    void finish(W12Job& J, cudaStream_t s) {
        J = W12Job();
        for (auto& kv : cells) {
            Cell& c = kv.second;
            std::map<int64_t, int> local;   // input base -> index in J.ins
            W12Cell cell{(int)J.ins.size(), 0, (int)J.outs.size(), 0, c.Da, c.Db};
            for (const Out& out : c.outs) {
                std::map<int, double> acc;
                for (const Term& t : out.terms) {
                    auto it = local.find(t.base);
                    int li;
                    if (it == local.end()) {
                        li = (int)J.ins.size();
                        local[t.base] = li;
                        J.ins.push_back({t.base, t.ld});
                    } else {
                        li = it->second;
                    }
                    acc[li] += t.coef;
                }
                TNH_REQUIRE(out.row0 < INT32_MAX && out.col0 < INT32_MAX && (out.col0 & 3) == 0, TNH_ERR_SHAPE,
                            "heff_plan: MPO step output out of range");
                W12Out o{out.task, (int)out.row0, (int)out.col0, (int)J.terms.size(), 0};
                for (auto& a : acc) {
                    const W12In& in = J.ins[(size_t)a.first];
                    TNH_REQUIRE(in.ld < INT32_MAX, TNH_ERR_SHAPE, "heff_plan: T1 row pitch too large");
                    J.terms.push_back({in.base, a.second, (float)a.second, (int)in.ld});
                }
                o.t1 = (int)J.terms.size();
                // the MPO step stores an output with its last term: none may be empty
                TNH_REQUIRE(o.t1 > o.t0, TNH_ERR_SHAPE, "heff_plan: MPO step output without terms");
                J.outs.push_back(o);
            }
            cell.nin = (int)J.ins.size() - cell.in0;
            cell.nout = (int)J.outs.size() - cell.out0;
            const int ci = (int)J.cells.size();
            J.cells.push_back(cell);
            const int64_t quads = (int64_t)c.Da * ((c.Db + 3) / 4);
            for (int64_t q0 = 0; q0 < quads; q0 += kW12Threads) J.ctas.push_back({ci, (int)q0});
        }
        TNH_REQUIRE(J.terms.size() < (size_t)INT32_MAX && J.outs.size() < (size_t)INT32_MAX &&
                        J.ins.size() < (size_t)INT32_MAX && J.ctas.size() < (size_t)INT32_MAX,
                    TNH_ERR_SHAPE, "heff_plan: MPO step too large");
        J.upload_all(s);
    }
};

GemmTask gemm_task(int64_t M, int64_t N, int64_t K, const HeffOperand& A, int ta, const HeffOperand& B, int tb,
                   bool tc, int tile0) {
    TNH_REQUIRE(M < (1 << 30) && N < (1 << 30) && K < (1 << 30), TNH_ERR_SHAPE, "heff_plan: block too large");
    GemmTask g{};
    g.M = (int)M;
    g.N = (int)N;
    g.K = (int)K;
    if (tc) {
        g.mt = (int)cdiv(M, kTcTileM);
        g.nt = (int)cdiv(N, kTcTileN);
        g.kt = (int)cdiv(K, kTcTileK);
        g.a_base = A.gtc[ta].base;
        g.b_base = B.gtc[tb].base;
    } else {
        g.mt = (int)cdiv(M, kF64TileM);
        g.nt = (int)cdiv(N, kF64TileN);
        g.kt = (int)cdiv(K, kF64TileK);
        g.a_base = A.g64[ta].base;
        g.b_base = B.g64[tb].base;
        g.lda = A.g64[ta].ld;
        g.ldb = B.g64[tb].ld;
    }
    g.tile0 = tile0;
    return g;
}

void finish_gemm(HeffGemm& G, cudaStream_t s) {
    G.d_f64 = upload(G.f64, s);
    G.tc_base = G.tc;
    G.d_tc = upload(G.tc, s);
}

// K split of the FP64 GEMM: with fewer 64 x 64 tiles than half the SMs and
// long K, every task is cut into up to 8 slices of 16-multiples whose float64
// products are summed in slice order (the output, scatter included, is
// written by the reduction).
void set_split64(HeffGemm& G, int num_sms, cudaStream_t s) {
    int64_t kmax = 0;
    for (const GemmTask& t : G.f64) kmax = std::max<int64_t>(kmax, t.K);
    int S = 1;
    while (S < 8 && G.tiles64 * S * 2 < num_sms && kmax >= (int64_t)256 * S) S *= 2;
    G.split64 = S;
    G.f64run.clear();
    G.reds64.clear();
    G.red64_total = G.part64_elems = 0;
    G.tiles64run = 0;
    if (S == 1) return;
    for (const GemmTask& b : G.f64) {
        const int64_t mn = (int64_t)b.M * b.N;
        const int kt = b.kt, per = (kt + S - 1) / S;
        int used = 0;
        for (int k0 = 0; k0 < kt; k0 += per) {
            GemmTask t = b;
            t.kt = std::min(per, kt - k0);
            t.K = (int)std::min<int64_t>(b.K - (int64_t)k0 * kF64TileK, (int64_t)t.kt * kF64TileK);
            t.a_base = b.a_base + (int64_t)k0 * kF64TileK;
            t.b_base = b.b_base + (int64_t)k0 * kF64TileK;
            t.c_base = G.part64_elems + (int64_t)used * mn;
            t.ldc = b.N;
            t.use_roff = 0;
            t.tile0 = G.tiles64run;
            G.tiles64run += t.mt * t.nt;
            G.f64run.push_back(t);
            ++used;
        }
        SplitRed r{};
        r.M = b.M;
        r.N = b.N;
        r.S = used;
        r.use_roff = b.use_roff;
        r.out_f32 = 0;
        r.ldc = b.ldc;
        r.part = G.part64_elems;
        r.roff = b.roff;
        r.c_base = b.c_base;
        r.e0 = G.red64_total;
        G.reds64.push_back(r);
        G.part64_elems += (int64_t)used * mn;
        G.red64_total += mn;
    }
    G.d_f64run = upload(G.f64run, s);
    G.d_reds64 = upload(G.reds64, s);
    G.red64_blocks = reduction_blocks(G.reds64);
    G.d_red64_blocks = upload(G.red64_blocks, s);
}

// Rebuild the launched tcgen05 tasks of G for a K-split factor (1: the block
// tasks themselves). With split > 1 every block task goes through the
// partial slabs (also those too short to split), so that the reduction is
// the one launch that writes the output.
void set_split(HeffGemm& G, int split, cudaStream_t s) {
    G.split = split;
    G.tc.clear();
    G.reds.clear();
    G.red_total = G.part_elems = 0;
    int tile0 = 0;
    if (split <= 1) {
        for (GemmTask t : G.tc_base) {
            t.tile0 = tile0;
            tile0 += t.mt * t.nt;
            G.tc.push_back(t);
        }
    } else {
        for (const GemmTask& b : G.tc_base) {
            const int S = std::max(1, std::min(split, b.kt));
            const int64_t mn = (int64_t)b.M * b.N;
            SplitRed r{};
            r.M = b.M;
            r.N = b.N;
            r.S = S;
            r.use_roff = b.use_roff;
            r.out_f32 = b.c_f32;
            r.ldc = b.ldc;
            r.part = G.part_elems;
            r.roff = b.roff;
            r.c_base = b.c_base;
            r.e0 = G.red_total;
            for (int j = 0; j < S; ++j) {
                const int k0 = (int)((int64_t)j * b.kt / S), k1 = (int)((int64_t)(j + 1) * b.kt / S);
                GemmTask t = b;
                t.kstride = b.kt;
                t.a_base = b.a_base + k0;
                t.b_base = b.b_base + k0;
                t.kt = k1 - k0;
                t.K = std::min(b.K - k0 * kTcTileK, (k1 - k0) * kTcTileK);
                t.c_f32 = 1;
                t.use_roff = 0;
                t.c_base = G.part_elems + j * mn;
                t.ldc = b.N;
                t.tile0 = tile0;
                tile0 += t.mt * t.nt;
                G.tc.push_back(t);
            }
            G.part_elems += S * mn;
            G.red_total += mn;
            G.reds.push_back(r);
        }
    }
    G.tilestc = tile0;
    G.d_tc = upload(G.tc, s);
    G.d_reds = upload(G.reds, s);
    G.red_blocks = reduction_blocks(G.reds);
    G.d_red_blocks = upload(G.red_blocks, s);
    // (pageable uploads are staged before they return: the host vectors may change)
}

// One tcgen05 GEMM of the plan, and its reduction when K is split. With
// fusedA the GEMM (S4) forms its operand A from T1 by the plan's job jT.
void launch_stage(const HeffGemm& G, const HeffPlan& P, const uint16_t* A, const uint16_t* B, void* out,
                  const int64_t* row_off, cudaStream_t s, bool fusedA = false) {
    Ctx* ctx = P.ctx;
    int* err = ctx->d_flag.as<int>();
    double* C = G.split <= 1 ? static_cast<double*>(out) : P.part.as<double>();
    const int64_t* ro = G.split <= 1 ? row_off : nullptr;
    if (fusedA)
        launch_gemm_tc_fused(G.d_tc.as<GemmTask>(), (int)G.tc.size(), G.tilestc, P.jT.d_tiles.as<GatherTile>(),
                             P.jT.d_segs.as<GatherSeg>(), P.jT.d_terms.as<GatherTerm>(), P.t1.as<float>(), B, C,
                             ctx->num_sms, err, s, ro);
    else
        launch_gemm_tc(G.d_tc.as<GemmTask>(), (int)G.tc.size(), G.tilestc, A, B, C, P.planes, ctx->num_sms, err, s,
                       ro);
    if (G.split > 1) {
        launch_splitk_reduce(G.d_reds.as<SplitRed>(), G.d_red_blocks.as<RedBlock>(), (int)G.red_blocks.size(),
                             P.part.as<float>(), out, row_off, s);
    }
}

void upload_operand(HeffOperand& O, cudaStream_t s) {
    O.d_g64 = upload(O.g64, s);
    O.d_gtc = upload(O.gtc, s);
}

}  // namespace

void HeffOperand::add_task(int64_t rows, int64_t K) {
    // float64: rows padded to the gather tile (128), pitch to 64 columns
    g64.push_back(OpGeom{elems64, (int)rup(K, kGatherCols)});
    elems64 += rup(rows, kGatherRows) * rup(K, kGatherCols);
    gtc.push_back(OpGeom{tiles, (int)cdiv(K, kTcTileK)});
    tiles += cdiv(rows, kTcTileM) * cdiv(K, kTcTileK);
}

namespace {

void ensure_part(HeffPlan& P, int64_t elems) {
    const size_t need = (size_t)std::max<int64_t>(elems, 4) * sizeof(float);
    if (P.part.bytes < need) P.part.alloc(need);
}

int64_t base_tiles(const HeffGemm& G) {
    int64_t n = 0;
    for (const GemmTask& t : G.tc_base) n += (int64_t)t.mt * t.nt;
    return n;
}

// N tile width of a task under a tile policy. 0: always 128. 1: the width
// that moves the fewest operand bytes per K block (48 KB of A per tile plus
// 384 B of B per column, three planes): operand traffic bound. 2: the width
// that issues the fewest MMA columns (tiles x (width + 16), 16 standing for
// the per-tile cost): tensor bound. Ties keep the wider tile.
int tile_width(int N, int policy) {
    if (policy == 0) return kTcTileN;
    int best = kTcTileN;
    double bc = 1e300;
    for (int tn : {128, 64, 32}) {
        const double tiles = (double)cdiv(N, tn);
        const double c = policy == 1 ? tiles * (48.0 + 0.375 * tn) : tiles * (tn + 16.0);
        if (c < bc - 1e-9) {
            bc = c;
            best = tn;
        }
    }
    return best;
}

void set_tiles(HeffGemm& G, int policy) {
    G.tile_policy = policy;
    for (GemmTask& t : G.tc_base) {
        t.tn = tile_width(t.N, policy);
        t.nt = (int)cdiv(t.N, t.tn);
    }
}

// ---- tuning cache on disk: one line per shape signature,
//   "heff <key values...> : <tiles S1> <split S1> <tiles S4> <split S4> <S4 fused>"
// read when a context first tunes, appended to after every measurement.
// The file is named by TNH_TUNE_CACHE (no file: the choices live as long as
// the context).
std::string tune_line(const std::vector<int>& key, const std::array<int, 5>& c) {
    std::string l = "heff";
    for (int k : key) l += " " + std::to_string(k);
    l += " :";
    for (int v : c) l += " " + std::to_string(v);
    return l;
}

void load_tune_file(Ctx* ctx) {
    if (ctx->tune_loaded) return;
    ctx->tune_loaded = true;
    const char* path = std::getenv("TNH_TUNE_CACHE");
    if (!path || !*path) return;
    FILE* f = std::fopen(path, "r");
    if (!f) return;
    char line[512];
    while (std::fgets(line, sizeof line, f)) {
        std::string l(line);
        if (l.rfind("heff ", 0) != 0) continue;
        const size_t colon = l.find(':');
        if (colon == std::string::npos) continue;
        std::vector<int> key;
        std::array<int, 5> c{};
        int v, pos = 5, n = 0;
        const std::string a = l.substr(5, colon - 5), b = l.substr(colon + 1);
        const char* p = a.c_str();
        while (std::sscanf(p, "%d%n", &v, &n) == 1) {
            key.push_back(v);
            p += n;
        }
        p = b.c_str();
        int k = 0;
        while (k < 5 && std::sscanf(p, "%d%n", &v, &n) == 1) {
            c[k++] = v;
            p += n;
        }
        (void)pos;
        const bool valid = k == 5 && c[0] >= 0 && c[0] <= 2 && c[2] >= 0 && c[2] <= 2 && c[1] >= 1 && c[1] <= 8 &&
                           c[3] >= 1 && c[3] <= 8 && (c[4] == 0 || c[4] == 1);
        if (valid && !key.empty()) ctx->heff_tune[key] = c;
    }
    std::fclose(f);
}

void save_tune_line(const std::vector<int>& key, const std::array<int, 5>& c) {
    const char* path = std::getenv("TNH_TUNE_CACHE");
    if (!path || !*path) return;
    if (FILE* f = std::fopen(path, "a")) {
        std::fprintf(f, "%s\n", tune_line(key, c).c_str());
        std::fclose(f);
    }
}

// Autotuner of the two tcgen05 GEMMs of a plan: first the N tile policy
// (tile_width; 128-wide tiles against tiles fitted to the output blocks'
// widths by two cost models), then the K-split factor (1, 2, 4, 8; only
// splits that can fill the GPU better). Each candidate is timed with CUDA
// events on the plan's own operands, one warm-up and the best of three timed
// runs of the GEMM and its reduction; a candidate replaces the incumbent only
// when it is 3% faster. Choices are kept in the context by a coarse shape signature
// (tasks, tiles and mean K blocks per task, in half octaves), so the bonds
// of a sweep at similar sizes reuse them, and in the TNH_TUNE_CACHE file
// across processes. TNH_HEFF_SPLIT="s1,s4" and TNH_HEFF_TILES="p1,p4"
// force the choices.
void tune_plan(HeffPlan& P) {
    Ctx* ctx = P.ctx;
    cudaStream_t s = P.stream;
    set_tiles(P.g1, 0);
    set_tiles(P.g4, 0);
    auto bucket = [](double x) { return (int)std::lround(2.0 * std::log2(std::max(1.0, x))); };
    std::vector<int> key{P.planes};
    for (const HeffGemm* G : {&P.g1, &P.g4}) {
        int64_t kt = 0;
        for (const GemmTask& t : G->tc_base) kt += t.kt;
        key.push_back(bucket((double)G->tc_base.size()));
        key.push_back(bucket((double)base_tiles(*G)));
        key.push_back(bucket((double)kt / std::max<size_t>(1, G->tc_base.size())));
    }
    load_tune_file(ctx);
    // tiles S1, split S1, tiles S4, split S4, S4 forms its operand itself
    std::array<int, 5> choice{0, 1, 0, 1, 0};
    bool measured = false;
    const bool can_fuse = P.planes == 3 && P.jT.ntiles > 0;
    const char* fs = std::getenv("TNH_HEFF_SPLIT");
    const char* ft = std::getenv("TNH_HEFF_TILES");
    const char* ff = std::getenv("TNH_HEFF_FUSED");
    if (fs || ft || ff) {
        int a = 1, b = 1, c = 0, d = 0;
        if (fs && std::sscanf(fs, "%d,%d", &a, &b) != 2) a = b = 1;
        if (ft && std::sscanf(ft, "%d,%d", &c, &d) != 2) c = d = 0;
        const int f = ff && std::atoi(ff) == 1 && can_fuse ? 1 : 0;
        choice = {std::min(std::max(c, 0), 2), std::max(1, a), std::min(std::max(d, 0), 2), std::max(1, b), f};
    } else if (ctx->heff_tune.count(key)) {
        choice = ctx->heff_tune[key];
    } else {
        DevBuf ytmp((size_t)std::max<int64_t>(P.n, 1) * sizeof(double));
        cudaEvent_t e0, e1;
        CUDA_CHECK(cudaEventCreate(&e0));
        CUDA_CHECK(cudaEventCreate(&e1));
        bool fused = false;
        auto best_of_3 = [&](auto&& run) {
            run();
            // the best of three separately timed runs (the first plans of a
            // process run while clocks and caches settle)
            float best = 1e30f;
            for (int r = 0; r < 3; ++r) {
                CUDA_CHECK(cudaEventRecord(e0, s));
                run();
                CUDA_CHECK(cudaEventRecord(e1, s));
                CUDA_CHECK(cudaEventSynchronize(e1));
                float ms = 0.f;
                CUDA_CHECK(cudaEventElapsedTime(&ms, e0, e1));
                best = std::min(best, ms);
            }
            return best;
        };
        auto time_run = [&](HeffGemm& G, bool s1, int split) {
            set_split(G, split, s);
            ensure_part(P, G.part_elems);
            auto run = [&] {
                if (s1) launch_stage(G, P, P.Ltc.as<uint16_t>(), P.opX.as<uint16_t>(), P.t1.p, nullptr, s);
                else launch_stage(G, P, P.opTtc.as<uint16_t>(), P.Rtc.as<uint16_t>(), ytmp.p, P.row_off.as<int64_t>(),
                                  s, fused);
            };
            return best_of_3(run);
        };
        HeffGemm* Gs[2] = {&P.g1, &P.g4};
        for (int g = 0; g < 2; ++g) {
            HeffGemm& G = *Gs[g];
            // S4: the W1.W2 pass then the GEMM, or the GEMM forming its own
            // operand A from T1 (128-wide tiles, no split)
            if (g == 1 && can_fuse) {
                fused = false;
                const float tw = best_of_3([&] {
                    launch_w12(P.jW, P.oT.d_gtc.as<OpGeom>(), P.t1.as<float>(), P.opTtc.p, P.planes, s);
                });
                const float tu = tw + time_run(G, false, 1);
                fused = true;
                const float tf = time_run(G, false, 1);
                fused = tf < 0.97f * tu;
                choice[4] = fused ? 1 : 0;
            }
            // tile policy at split 1
            std::vector<int> widths0;
            for (const GemmTask& t : G.tc_base) widths0.push_back(t.tn);
            int bestp = 0;
            float tbest = time_run(G, g == 0, 1);
            std::vector<std::vector<int>> seen{widths0};
            for (int policy : {1, 2}) {
                set_tiles(G, policy);
                std::vector<int> w;
                for (const GemmTask& t : G.tc_base) w.push_back(t.tn);
                if (std::find(seen.begin(), seen.end(), w) != seen.end()) continue;   // same tiles
                seen.push_back(w);
                const float tm = time_run(G, g == 0, 1);
                if (tm < 0.97f * tbest) {
                    tbest = tm;
                    bestp = policy;
                }
            }
            set_tiles(G, bestp);
            // K split with the chosen tiles
            int maxkt = 1;
            for (const GemmTask& t : G.tc_base) maxkt = std::max(maxkt, t.kt);
            const int64_t tiles = base_tiles(G);
            int bests = 1;
            for (int split : {2, 4, 8}) {
                if (split > maxkt || tiles * (split / 2) >= 2 * (int64_t)ctx->num_sms) break;
                const float tm = time_run(G, g == 0, split);
                if (tm < 0.97f * tbest) {
                    tbest = tm;
                    bests = split;
                }
            }
            choice[2 * g] = bestp;
            choice[2 * g + 1] = bests;
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        check_device_flag(ctx);
        ctx->heff_tune[key] = choice;
        save_tune_line(key, choice);
        measured = true;
    }
    set_tiles(P.g1, choice[0]);
    set_tiles(P.g4, choice[2]);
    set_split(P.g1, choice[1], s);
    set_split(P.g4, choice[3], s);
    P.fusedS4 = choice[4] == 1 && can_fuse;
    ensure_part(P, std::max(P.g1.part_elems, P.g4.part_elems));
    P.tune = choice;
    P.tune_measured = measured;
    if (std::getenv("TNH_DEBUG"))
        std::fprintf(stderr, "heff_plan: S1 tiles %d split %d, S4 tiles %d split %d fused %d (%s; S1 %lld tiles, S4 %lld tiles)\n",
                     choice[0], choice[1], choice[2], choice[3], choice[4], measured ? "measured" : "cached or forced",
                     (long long)base_tiles(P.g1), (long long)base_tiles(P.g4));
}

}  // namespace

HeffPlan::~HeffPlan() {
    for (auto& g : graphs) {
        if (g.exec) cudaGraphExecDestroy(g.exec);
        if (g.graph) cudaGraphDestroy(g.graph);
    }
}

namespace {
// TNH_DEBUG: host wall time of the phases of one plan
struct PlanClock {
    bool on = std::getenv("TNH_DEBUG") != nullptr;
    std::chrono::steady_clock::time_point last = std::chrono::steady_clock::now();
    std::string line;
    void mark(const char* what) {
        if (!on) return;
        const auto now = std::chrono::steady_clock::now();
        char b[64];
        std::snprintf(b, sizeof b, " %s %.2f", what, std::chrono::duration<double, std::milli>(now - last).count());
        line += b;
        last = now;
    }
    ~PlanClock() {
        if (on) std::fprintf(stderr, "heff_plan: phases (ms)%s\n", line.c_str());
    }
};
}  // namespace

std::unique_ptr<HeffPlan> make_heff_strategy(Ctx* ctx, const Layout& L, const Layout& W1, const Layout& W2,
                                             const Layout& R, const Layout& X, tnh_precision prec, int strategy) {
    TNH_REQUIRE(L.rank() == 3 && R.rank() == 3 && W1.rank() == 4 && W2.rank() == 4 && X.rank() == 4,
                TNH_ERR_ARG, "heff_plan: ranks must be L 3, W 4, R 3, psi 4");
    TNH_REQUIRE(prec == TNH_FP64 || planes_of(prec) > 0, TNH_ERR_ARG, "heff_plan: bad precision");
    check_pair(L.inds[0], X.inds[0], "L and psi (a)");
    check_pair(L.inds[1], W1.inds[0], "L and W1 (w)");
    check_pair(W1.inds[2], X.inds[1], "W1 and psi (s1)");
    check_pair(W1.inds[1], W2.inds[0], "W1 and W2 (w1)");
    check_pair(W2.inds[2], X.inds[2], "W2 and psi (s2)");
    check_pair(R.inds[0], X.inds[3], "R and psi (b)");
    check_pair(R.inds[1], W2.inds[1], "R and W2 (w2)");
    const Index* Yi[4] = {&L.inds[2], &W1.inds[3], &W2.inds[3], &R.inds[2]};
    for (int i = 0; i < 4; ++i)
        TNH_REQUIRE(Yi[i]->same_space(X.inds[i]) && Yi[i]->arrow == X.inds[i].arrow, TNH_ERR_SHAPE,
                    "heff_plan: output index %d does not match psi's (sectors or arrow)", i);
    if (L.nblocks() && W1.nblocks() && W2.nblocks() && R.nblocks() && X.nblocks())
        TNH_REQUIRE(add_flux(add_flux(L.flux, W1.flux), add_flux(W2.flux, R.flux)) == std::vector<int>(X.nq(), 0),
                    TNH_ERR_FLUX, "heff_plan: L, W1, W2, R do not conserve psi's flux");
    TNH_REQUIRE(X.packed_total() <= X.size || X.nblocks() == 0, TNH_ERR_SHAPE, "heff_plan: psi too small");

    cudaStream_t s = ctx->stream;
    auto P = std::make_unique<HeffPlan>();
    P->ctx = ctx;
    P->stream = s;
    P->prec = prec;
    P->planes = prec == TNH_FP64 ? 0 : planes_of(prec);
    P->n = X.size;
    P->psi = X;
    const Index &ia = X.inds[0], &is1 = X.inds[1], &is2 = X.inds[2], &ib = X.inds[3];
    const Index &iw = L.inds[1], &iz = R.inds[1];

    PlanClock clk;
    // method flops: S1..S4 over the allowed blocks of the labelled chain
    {
        Layout Ll = with_labels(L, {La, Lw, Lap});
        Layout W1l = with_labels(W1, {Lw, Lw1, Ls1, Ls1p});
        Layout W2l = with_labels(W2, {Lw1, Lw2, Ls2, Ls2p});
        Layout Rl = with_labels(R, {Lb, Lw2, Lbp});
        Layout Xl = with_labels(X, {La, Ls1, Ls2, Lb});
        Layout T1 = make_layout({Ll.inds[1], Ll.inds[2], Xl.inds[1], Xl.inds[2], Xl.inds[3]}, add_flux(L.flux, X.flux));
        Layout T2 = make_layout({T1.inds[1], T1.inds[3], T1.inds[4], W1l.inds[1], W1l.inds[3]},
                                add_flux(T1.flux, W1.flux));
        Layout T3 = make_layout({T2.inds[0], T2.inds[2], T2.inds[4], W2l.inds[1], W2l.inds[3]},
                                add_flux(T2.flux, W2.flux));
        P->f_s1 = contract_flops(Ll, Xl);
        P->f_s23 = contract_flops(T1, W1l) + contract_flops(T2, W2l);
        P->f_s4 = contract_flops(T3, Rl);
        P->flops = P->f_s1 + P->f_s23 + P->f_s4;
    }

    clk.mark("flops");
    // ---------------- S1: per a-sector A with L and psi blocks. Strategy 0
    // (combine, then contract): one GEMM task per A, all L blocks of A along
    // M and all psi blocks of A along N. Strategy 1 (block pairs): one task
    // per (L block, psi block) pair, writing its sub-block of the same T1
    // layout. Both read L and psi packed once.
    struct RowRef { int task; int64_t row; };
    std::map<std::pair<int, int>, std::vector<RowRef>> t1_rows;   // (w element, a'-sector) -> rows
    std::map<std::array<int, 4>, std::pair<int, int64_t>> t1_cols; // psi block sectors -> (task, first col)
    std::vector<int64_t> t1_base, t1_ld;
    std::vector<int> t1_sector;   // a-sector of every T1 block row group
    JobBuilder bL, bX;
    int tf = 0, tt = 0;
    auto add_s1 = [&](int64_t M, int64_t N, int64_t K, int ta, int tb, int64_t c_base, int64_t ldc) {
        GemmTask g = gemm_task(M, N, K, P->oL, ta, P->oX, tb, false, tf);
        g.c_base = c_base;
        g.ldc = (int)ldc;
        GemmTask h = gemm_task(M, N, K, P->oL, ta, P->oX, tb, true, tt);
        h.c_base = c_base;
        h.ldc = (int)ldc;
        h.c_f32 = 1;
        tf += g.mt * g.nt;
        tt += h.mt * h.nt;
        P->g1.f64.push_back(g);
        P->g1.tc.push_back(h);
    };
    for (int A = 0; A < ia.nsect; ++A) {
        std::vector<int> lb, xb;
        for (int b = 0; b < L.nblocks(); ++b)
            if (L.sect[(size_t)b * 3] == A) lb.push_back(b);
        for (int b = 0; b < X.nblocks(); ++b)
            if (X.sect[(size_t)b * 4] == A) xb.push_back(b);
        if (lb.empty() || xb.empty()) continue;
        const int t = (int)t1_base.size();
        const int64_t K = ia.dim[A];
        int64_t M = 0, N = 0;
        for (int b : lb) M += (int64_t)L.bdim(b, 1) * L.bdim(b, 2);
        // columns (s1, s2, b): every (s1, s2) group of Db columns starts at a
        // multiple of 4, so that every T1 row segment the MPO step reads is
        // 16-byte aligned (the padding columns are zero)
        for (int b : xb) N += (int64_t)X.bdim(b, 1) * X.bdim(b, 2) * rup(X.bdim(b, 3), 4);
        // operand tasks: one per A (strategy 0) or one per block (strategy 1)
        std::vector<int> lt, xt;
        if (strategy == 0) {
            lt.assign(lb.size(), P->oL.count());
            xt.assign(xb.size(), P->oX.count());
            P->oL.add_task(M, K);
            P->oX.add_task(N, K);
            bL.task(M, K);
            bX.task(N, K);
        } else {
            for (int b : lb) {
                lt.push_back(P->oL.count());
                P->oL.add_task((int64_t)L.bdim(b, 1) * L.bdim(b, 2), K);
                bL.task((int64_t)L.bdim(b, 1) * L.bdim(b, 2), K);
            }
            for (int b : xb) {
                const int64_t nbp = (int64_t)X.bdim(b, 1) * X.bdim(b, 2) * rup(X.bdim(b, 3), 4);
                xt.push_back(P->oX.count());
                P->oX.add_task(nbp, K);
                bX.task(nbp, K);
            }
        }
        // rows (w, a'): operand A = L^T, element (r = a', c = a)
        int64_t row = 0;
        std::vector<int64_t> lrow0;
        for (size_t i = 0; i < lb.size(); ++i) {
            const int b = lb[i];
            const int Sx = L.sect[(size_t)b * 3 + 1], Ap = L.sect[(size_t)b * 3 + 2];
            const int Dx = L.bdim(b, 1), Dap = L.bdim(b, 2);
            lrow0.push_back(row);
            const int64_t r0 = strategy == 0 ? row : 0;   // row inside the operand task
            for (int xl = 0; xl < Dx; ++xl) {
                bL.rect(lt[i], r0 + (int64_t)xl * Dap, 0, Dap, K,
                        {GatherTerm{1.0, L.off[b] + (int64_t)xl * Dap, 1, (int64_t)Dx * Dap, 1.0f}});
                t1_rows[{(int)(iw.off[Sx] + xl), Ap}].push_back({t, row + (int64_t)xl * Dap});
            }
            row += (int64_t)Dx * Dap;
        }
        // columns (s1, s2, b): operand B = psi^T, element (r = (s1,s2,b), c = a);
        // group g = (s1, s2) of a block starts at column col + g * Dbp
        int64_t col = 0;
        std::vector<int64_t> xcol0;
        for (size_t i = 0; i < xb.size(); ++i) {
            const int b = xb[i];
            const int64_t nb = X.belems(b) / K;
            const int Db = X.bdim(b, 3), Dbp = (int)rup(Db, 4), ng = X.bdim(b, 1) * X.bdim(b, 2);
            xcol0.push_back(col);
            const int64_t c0 = strategy == 0 ? col : 0;
            for (int g = 0; g < ng; ++g)
                bX.rect(xt[i], c0 + (int64_t)g * Dbp, 0, Db, K, {GatherTerm{1.0, X.off[b] + (int64_t)g * Db, 1, nb, 1.0f}});
            t1_cols[{A, X.sect[(size_t)b * 4 + 1], X.sect[(size_t)b * 4 + 2], X.sect[(size_t)b * 4 + 3]}] = {t, col};
            col += (int64_t)ng * Dbp;
        }
        t1_base.push_back(P->t1_elems);
        t1_ld.push_back(N);
        t1_sector.push_back(A);
        if (strategy == 0) {
            add_s1(M, N, K, lt[0], xt[0], P->t1_elems, N);
        } else {
            for (size_t i = 0; i < lb.size(); ++i)
                for (size_t j = 0; j < xb.size(); ++j) {
                    const int bl = lb[i], bx = xb[j];
                    const int64_t Mi = (int64_t)L.bdim(bl, 1) * L.bdim(bl, 2);
                    const int64_t Nj = (int64_t)X.bdim(bx, 1) * X.bdim(bx, 2) * rup(X.bdim(bx, 3), 4);
                    add_s1(Mi, Nj, K, lt[i], xt[j], P->t1_elems + lrow0[i] * N + xcol0[j], N);
                }
        }
        P->t1_elems += rup(M * N, 4);
    }
    P->g1.tiles64 = tf;
    P->g1.tilestc = tt;

    clk.mark("s1");
    // ---------------- two-site MPO product W12[(w,s1,s2) -> (w2,s1',s2')]
    struct W12Term { int x, s1, s2; double v; };
    std::map<std::array<int, 3>, std::vector<W12Term>> w12;   // (w2, s1', s2') -> terms
    {
        auto e1 = mpo_entries(W1, s), e2 = mpo_entries(W2, s);
        std::map<int, std::vector<MpoEntry>> by_w1;
        for (auto& e : e2) by_w1[e.l].push_back(e);
        std::map<std::array<int, 6>, double> acc;
        for (auto& a : e1) {
            auto it = by_w1.find(a.r);
            if (it == by_w1.end()) continue;
            for (auto& b : it->second) acc[{b.r, a.sp, b.sp, a.l, a.s, b.s}] += a.v * b.v;
        }
        for (auto& kv : acc)
            if (kv.second != 0.0)
                w12[{kv.first[0], kv.first[1], kv.first[2]}].push_back({kv.first[3], kv.first[4], kv.first[5], kv.second});
    }

    clk.mark("w12");
    // ---------------- diagonal of H_eff: environment diagonals and the
    // diagonal W12 entries (s1' = s1, s2' = s2) per (s1, s2)
    {
        const int wdim = (int)iw.total, zdim = (int)iz.total;
        const int d1tot = (int)is1.total, d2tot = (int)is2.total;
        std::vector<std::vector<DiagTerm>> per(d1tot * d2tot);
        for (auto& kv : w12)
            for (const W12Term& e : kv.second)
                if (e.s1 == kv.first[1] && e.s2 == kv.first[2])
                    per[e.s1 * d2tot + e.s2].push_back(DiagTerm{e.x, kv.first[0], e.v});
        std::vector<int> tstart(1, 0);
        std::vector<DiagTerm> terms;
        for (auto& v : per) {
            terms.insert(terms.end(), v.begin(), v.end());
            tstart.push_back((int)terms.size());
        }
        std::vector<EnvDiagSeg> ls, rs;
        for (int b = 0; b < L.nblocks(); ++b) {
            const int A = L.sect[(size_t)b * 3], Sx = L.sect[(size_t)b * 3 + 1], Ap = L.sect[(size_t)b * 3 + 2];
            if (A != Ap) continue;
            ls.push_back(EnvDiagSeg{L.off[b], L.bdim(b, 0), L.bdim(b, 1), ia.off[A] * wdim + iw.off[Sx], wdim});
        }
        for (int b = 0; b < R.nblocks(); ++b) {
            const int B = R.sect[(size_t)b * 3], Sz = R.sect[(size_t)b * 3 + 1], Bp = R.sect[(size_t)b * 3 + 2];
            if (B != Bp) continue;
            rs.push_back(EnvDiagSeg{R.off[b], R.bdim(b, 0), R.bdim(b, 1), ib.off[B] * zdim + iz.off[Sz], zdim});
        }
        std::vector<DiagBlock> db;
        for (int b = 0; b < X.nblocks(); ++b) {
            const int* k = &X.sect[(size_t)b * 4];
            db.push_back(DiagBlock{X.off[b], X.bdim(b, 0), X.bdim(b, 1), X.bdim(b, 2), X.bdim(b, 3),
                                   (int)ia.off[k[0]], (int)ib.off[k[3]], (int)is1.off[k[1]], (int)is2.off[k[2]]});
        }
        P->dg_wdim = wdim;
        P->dg_zdim = zdim;
        P->dg_d2 = d2tot;
        P->dg_nblocks = (int)db.size();
        P->dg_maxblock = 0;
        for (const DiagBlock& d : db)
            P->dg_maxblock = std::max<int64_t>(P->dg_maxblock, (int64_t)d.Da * d.d1 * d.d2 * d.Db);
        P->Ld.alloc((size_t)std::max<int64_t>(ia.total * wdim, 1) * sizeof(double));
        P->Rd.alloc((size_t)std::max<int64_t>(ib.total * zdim, 1) * sizeof(double));
        CUDA_CHECK(cudaMemsetAsync(P->Ld.p, 0, P->Ld.bytes, s));
        CUDA_CHECK(cudaMemsetAsync(P->Rd.p, 0, P->Rd.bytes, s));
        DevBuf d_ls = upload(ls, s), d_rs = upload(rs, s);
        if (!ls.empty()) {
            KScope ks("heff_env_diag", s);
            env_diag_kernel<<<(unsigned)ls.size(), 128, 0, s>>>(d_ls.as<EnvDiagSeg>(), L.data, P->Ld.as<double>());
        }
        if (!rs.empty()) {
            KScope ks("heff_env_diag", s);
            env_diag_kernel<<<(unsigned)rs.size(), 128, 0, s>>>(d_rs.as<EnvDiagSeg>(), R.data, P->Rd.as<double>());
        }
        P->d_dblocks = upload(db, s);
        P->d_dstart = upload(tstart, s);
        P->d_dterms = upload(terms, s);
        // d_ls, d_rs are freed on scope exit, in stream order after the gathers
    }

    clk.mark("diag");
    // ---------------- S4: per b'-sector; the fused S2+S3 step fills operand A.
    // Strategy 0: one GEMM task per b'-sector, the rows of all its psi blocks
    // along M. Strategy 1: one task per psi block (its rows), all tasks of a
    // b'-sector reading the same packed R. K is the same: every (w2 element,
    // b-sector) piece of R for that b'.
    JobBuilder bR;
    CellBuilder bW;
    std::vector<int64_t> roff;
    // per operand-A task of S4: rows, K, row pieces (row0, rows) and K pieces
    // (col0, columns): the grid every W1.W2 output fills one cell of
    std::vector<int64_t> tM, tK;
    std::vector<std::vector<std::pair<int64_t, int>>> trows, tkp;
    std::vector<char> covered(X.nblocks(), 0);
    tf = tt = 0;
    const Index& ibp = R.inds[2];
    for (int Bp = 0; Bp < ibp.nsect; ++Bp) {
        std::vector<int> yb, rb;
        for (int b = 0; b < X.nblocks(); ++b)
            if (X.sect[(size_t)b * 4 + 3] == Bp) yb.push_back(b);
        for (int b = 0; b < R.nblocks(); ++b)
            if (R.sect[(size_t)b * 3 + 2] == Bp) rb.push_back(b);
        if (yb.empty() || rb.empty()) continue;
        const int tr = P->oR.count();
        const int64_t N = ibp.dim[Bp];
        int64_t M = 0, K = 0;
        for (int b : yb) M += X.belems(b) / N;
        // K pieces (w2 element, b-sector) of Db columns each start at a multiple
        // of 4, so the MPO step writes four columns with one store per plane
        for (int b : rb) K += rup(R.bdim(b, 0), 4) * R.bdim(b, 1);
        P->oR.add_task(N, K);
        bR.task(N, K);
        // operand A tasks: one per b'-sector, or one per psi block
        std::vector<int> at;
        if (strategy == 0) {
            at.assign(yb.size(), P->oT.count());
            P->oT.add_task(M, K);
            tM.push_back(M);
            tK.push_back(K);
        } else {
            for (int b : yb) {
                at.push_back(P->oT.count());
                P->oT.add_task(X.belems(b) / N, K);
                tM.push_back(X.belems(b) / N);
                tK.push_back(K);
            }
        }
        trows.resize(tM.size());
        tkp.resize(tM.size());
        // K pieces (w2 element z, b-sector B): operand B = R^T, element (r = b', c = b)
        struct KPiece { int z, B; int64_t col; int Db; };
        std::vector<KPiece> kp;
        int64_t col = 0;
        for (int b : rb) {
            const int B = R.sect[(size_t)b * 3], Sz = R.sect[(size_t)b * 3 + 1];
            const int Db = R.bdim(b, 0), Dz = R.bdim(b, 1);
            for (int zl = 0; zl < Dz; ++zl) {
                bR.rect(tr, 0, col, N, Db, {GatherTerm{1.0, R.off[b] + (int64_t)zl * N, 1, (int64_t)Dz * N, 1.0f}});
                kp.push_back({(int)(iz.off[Sz] + zl), B, col, Db});
                col += rup(Db, 4);
            }
        }
        for (int a : std::vector<int>(at.begin(), strategy == 0 ? at.begin() + 1 : at.end()))
            for (const KPiece& k : kp) tkp[a].push_back({k.col, (int)rup(k.Db, 4)});
        // row pieces (s1', s2', a'): every row of every psi block of this b'-sector
        int64_t row = 0;
        for (size_t yi = 0; yi < yb.size(); ++yi) {
            const int b = yb[yi];
            covered[b] = 1;
            const int Ap = X.sect[(size_t)b * 4], S1p = X.sect[(size_t)b * 4 + 1], S2p = X.sect[(size_t)b * 4 + 2];
            const int Dap = X.bdim(b, 0), d1 = X.bdim(b, 1), d2 = X.bdim(b, 2);
            const int64_t roff0 = (int64_t)roff.size();
            const int64_t brow0 = row;   // first row of this block in the b'-sector's rows
            for (int u1 = 0; u1 < d1; ++u1)
                for (int u2 = 0; u2 < d2; ++u2) {
                    const int s1p = (int)(is1.off[S1p] + u1), s2p = (int)(is2.off[S2p] + u2);
                    for (int al = 0; al < Dap; ++al)
                        roff.push_back(X.off[b] + (((int64_t)al * d1 + u1) * d2 + u2) * N);
                    trows[at[yi]].push_back({strategy == 0 ? row : row - brow0, Dap});
                    for (const KPiece& k : kp) {
                        auto it = w12.find({k.z, s1p, s2p});
                        if (it == w12.end()) continue;
                        std::vector<CellBuilder::Term> tm;
                        for (const W12Term& e : it->second) {
                            auto rr = t1_rows.find({e.x, Ap});
                            if (rr == t1_rows.end()) continue;
                            const auto ps1 = locate(is1, e.s1), ps2 = locate(is2, e.s2);
                            for (const RowRef& ref : rr->second) {
                                // T1 columns of the psi block (A of the row's task, S1, S2, B)
                                auto ci = t1_cols.find({t1_sector[ref.task], ps1.first, ps2.first, k.B});
                                if (ci == t1_cols.end()) continue;
                                const int ds2 = is2.dim[ps2.first];
                                const int64_t c0 =
                                    ci->second.second + ((int64_t)ps1.second * ds2 + ps2.second) * rup(k.Db, 4);
                                const int64_t ld = t1_ld[ref.task];
                                tm.push_back({t1_base[ref.task] + ref.row * ld + c0, ld, e.v});
                            }
                        }
                        bW.add(Ap, k.B, Dap, k.Db, at[yi], strategy == 0 ? row : row - brow0, k.col, std::move(tm));
                    }
                    row += Dap;
                }
            if (strategy == 1) {
                const int64_t Mb = X.belems(b) / N;
                GemmTask g = gemm_task(Mb, N, K, P->oT, at[yi], P->oR, tr, false, tf);
                GemmTask h = gemm_task(Mb, N, K, P->oT, at[yi], P->oR, tr, true, tt);
                g.use_roff = h.use_roff = 1;
                g.roff = h.roff = roff0;
                tf += g.mt * g.nt;
                tt += h.mt * h.nt;
                P->g4.f64.push_back(g);
                P->g4.tc.push_back(h);
            }
        }
        if (strategy == 0) {
            GemmTask g = gemm_task(M, N, K, P->oT, at[0], P->oR, tr, false, tf);
            GemmTask h = gemm_task(M, N, K, P->oT, at[0], P->oR, tr, true, tt);
            g.use_roff = h.use_roff = 1;
            g.roff = h.roff = (int64_t)roff.size() - M;
            tf += g.mt * g.nt;
            tt += h.mt * h.nt;
            P->g4.f64.push_back(g);
            P->g4.tc.push_back(h);
        }
    }
    P->g4.tiles64 = tf;
    P->g4.tilestc = tt;
    for (int b = 0; b < X.nblocks(); ++b) P->zero_y |= !covered[b];
    if (X.packed_total() < X.size) P->zero_y = true;

    clk.mark("s4");
    // ---------------- device side
    bX.finish(P->jX, s);
    bW.finish(P->jW, s);
    // the W1.W2 step as gather segments of S4's operand A (split formats):
    // every cell (row piece, K piece) of every task is one output rectangle
    // (its terms) or zero, and the K tail of the last K tile is zero, so the
    // GEMM that forms A itself writes every element it multiplies
    if (P->planes == 3) {
        JobBuilder bT;
        for (size_t t = 0; t < tM.size(); ++t) bT.task(tM[t], tK[t]);
        std::vector<std::set<std::pair<int64_t, int64_t>>> covered_cells(tM.size());
        for (const W12Cell& cell : P->jW.cells)
            for (int o = cell.out0; o < cell.out0 + cell.nout; ++o) {
                const W12Out& out = P->jW.outs[(size_t)o];
                std::vector<GatherTerm> tm;
                for (int j = out.t0; j < out.t1; ++j) {
                    const tnh::W12Term& w = P->jW.terms[(size_t)j];
                    tm.push_back(GatherTerm{w.coef, w.base, w.ld, 1, w.coef32});
                }
                bT.rect(out.task, out.row0, out.col0, cell.Da, rup(cell.Db, 4), tm);
                covered_cells[(size_t)out.task].insert({out.row0, out.col0});
            }
        for (size_t t = 0; t < tM.size(); ++t) {
            for (const auto& rp : trows[t])
                for (const auto& kq : tkp[t])
                    if (!covered_cells[t].count({rp.first, kq.first}))
                        bT.rect((int)t, rp.first, kq.first, rp.second, kq.second, {}, true);
            const int64_t Kp = rup(tK[t], kGatherCols);
            if (Kp > tK[t]) bT.rect((int)t, 0, tK[t], tM[t], Kp - tK[t], {}, true);
        }
        bT.finish(P->jT, s);
    }
    GatherJob jL, jR;
    bL.finish(jL, s);
    bR.finish(jR, s);
    for (HeffOperand* o : {&P->oL, &P->oX, &P->oT, &P->oR}) upload_operand(*o, s);
    finish_gemm(P->g1, s);
    finish_gemm(P->g4, s);
    set_split64(P->g1, ctx->num_sms, s);
    set_split64(P->g4, ctx->num_sms, s);
    {
        const int64_t p64 = std::max(P->g1.part64_elems, P->g4.part64_elems);
        if (p64 > 0) P->part64.alloc((size_t)p64 * sizeof(double));
    }
    P->row_off = upload(roff, s);
    P->t1.alloc((size_t)std::max<int64_t>(P->t1_elems, 1) * sizeof(double));
    const int pl = P->planes;
    auto tc_bytes = [&](const HeffOperand& o) { return (size_t)o.tiles * pl * kTcTileElems * 2; };
    auto f64_bytes = [](const HeffOperand& o) { return (size_t)o.elems64 * sizeof(double); };
    P->opX.alloc(std::max<size_t>({f64_bytes(P->oX), tc_bytes(P->oX), 16}));
    CUDA_CHECK(cudaMemsetAsync(P->opX.p, 0, P->opX.bytes, s));
    // operand A of S4: the MPO step writes only the covered sub-blocks, the
    // rest (padding, sub-blocks without a W12 entry) stays zero from here on
    P->opT64.alloc(std::max<size_t>(f64_bytes(P->oT), 16));
    CUDA_CHECK(cudaMemsetAsync(P->opT64.p, 0, P->opT64.bytes, s));
    if (pl > 0) {
        P->opTtc.alloc(std::max<size_t>(tc_bytes(P->oT), 16));
        CUDA_CHECK(cudaMemsetAsync(P->opTtc.p, 0, P->opTtc.bytes, s));
    }
    P->L64.alloc(std::max<size_t>(f64_bytes(P->oL), 16));
    P->R64.alloc(std::max<size_t>(f64_bytes(P->oR), 16));
    launch_gather(jL, P->oL.d_g64.as<OpGeom>(), L.data, P->L64.p, 0, s, "heff_pack_env");
    launch_gather(jR, P->oR.d_g64.as<OpGeom>(), R.data, P->R64.p, 0, s, "heff_pack_env");
    if (pl > 0) {
        P->Ltc.alloc(std::max<size_t>(tc_bytes(P->oL), 16));
        P->Rtc.alloc(std::max<size_t>(tc_bytes(P->oR), 16));
        launch_gather(jL, P->oL.d_gtc.as<OpGeom>(), L.data, P->Ltc.p, pl, s, "heff_pack_env");
        launch_gather(jR, P->oR.d_gtc.as<OpGeom>(), R.data, P->Rtc.p, pl, s, "heff_pack_env");
    }
    CUDA_CHECK(cudaGetLastError());
    clk.mark("device");
    if (pl > 0 && !P->g1.tc_base.empty() && !P->g4.tc_base.empty()) tune_plan(*P);
    clk.mark("tune");
    if (std::getenv("TNH_DEBUG"))
        std::fprintf(stderr,
                     "heff_plan: n %lld, S1 %zu tasks %d tiles, T1 %lld, S4 %zu tasks %d tiles, T3 %lld, "
                     "MPO step %zu cells %zu ctas %zu inputs %zu outputs %zu terms\n",
                     (long long)P->n, P->g1.tc.size(), P->g1.tilestc, (long long)P->t1_elems, P->g4.tc.size(),
                     P->g4.tilestc, (long long)P->oT.elems64, P->jW.cells.size(), P->jW.ctas.size(),
                     P->jW.ins.size(), P->jW.outs.size(), P->jW.terms.size());
    // the host tables and the caller's L, R must stay alive until these ran
    CUDA_CHECK(cudaStreamSynchronize(s));
    return P;
}

namespace {

// Device time of one application of a plan (the best of three, after one
// untimed), in its own precision, on zero vectors.
float time_plan(HeffPlan& P) {
    cudaStream_t s = P.stream;
    DevBuf x((size_t)std::max<int64_t>(P.n, 1) * sizeof(double)), y((size_t)std::max<int64_t>(P.n, 1) * sizeof(double));
    CUDA_CHECK(cudaMemsetAsync(x.p, 0, x.bytes, s));
    cudaEvent_t e0, e1;
    CUDA_CHECK(cudaEventCreate(&e0));
    CUDA_CHECK(cudaEventCreate(&e1));
    heff_apply(P, P.prec, x.as<double>(), y.as<double>());
    float best = 1e30f;
    for (int r = 0; r < 3; ++r) {
        CUDA_CHECK(cudaEventRecord(e0, s));
        heff_apply(P, P.prec, x.as<double>(), y.as<double>());
        CUDA_CHECK(cudaEventRecord(e1, s));
        CUDA_CHECK(cudaEventSynchronize(e1));
        float ms = 0.f;
        CUDA_CHECK(cudaEventElapsedTime(&ms, e0, e1));
        best = std::min(best, ms);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    check_device_flag(P.ctx);
    return best;
}

}  // namespace

// The block-contraction strategy is chosen per shape (the paper notes that
// neither combining blocks before contracting nor contracting block pairs
// always wins, Sec. 9.4): both plans are built and timed once for a shape
// signature (precision, psi size, block counts and mean sector dimension of
// psi, in half octaves), the faster one (block pairs only when 3% faster)
// is kept in the context for later plans of the same signature.
// TNH_HEFF_STRATEGY=0 / 1 forces combine-then-contract / block pairs.
std::unique_ptr<HeffPlan> make_heff(Ctx* ctx, const Layout& L, const Layout& W1, const Layout& W2,
                                    const Layout& R, const Layout& X, tnh_precision prec) {
    if (const char* f = std::getenv("TNH_HEFF_STRATEGY")) {
        const int st = std::atoi(f) == 1 ? 1 : 0;
        auto P = make_heff_strategy(ctx, L, W1, W2, R, X, prec, st);
        P->strategy = st;
        return P;
    }
    auto bucket = [](double x) { return (int)std::lround(2.0 * std::log2(std::max(1.0, x))); };
    double dsum = 0.0;
    for (int b = 0; b < X.nblocks(); ++b) dsum += X.bdim(b, 0) + X.bdim(b, 3);
    std::vector<int> key{-1, (int)prec, bucket((double)X.size), bucket((double)X.nblocks()), bucket((double)L.nblocks()),
                         bucket((double)R.nblocks()), bucket(dsum / std::max(1, 2 * X.nblocks()))};
    auto it = ctx->heff_strategy.find(key);
    if (it != ctx->heff_strategy.end()) {
        auto P = make_heff_strategy(ctx, L, W1, W2, R, X, prec, it->second);
        P->strategy = it->second;
        return P;
    }
    auto P0 = make_heff_strategy(ctx, L, W1, W2, R, X, prec, 0);
    auto P1 = make_heff_strategy(ctx, L, W1, W2, R, X, prec, 1);
    const float t0 = time_plan(*P0), t1 = time_plan(*P1);   // per product
    const int st = t1 < 0.97f * t0 ? 1 : 0;
    ctx->heff_strategy[key] = st;
    auto& P = st == 1 ? P1 : P0;
    P->strategy = st;
    P->strategy_measured = true;
    P->strategy_ms[0] = t0;
    P->strategy_ms[1] = t1;
    if (std::getenv("TNH_DEBUG"))
        std::fprintf(stderr, "heff_plan: strategy %s (combine %.3f ms, block pairs %.3f ms per product)\n",
                     st == 1 ? "block pairs" : "combine", t0, t1);
    return std::move(P);
}

namespace {

cudaGraphNode_t last_node(cudaStream_t s) {
    cudaStreamCaptureStatus st;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    CUDA_CHECK(cudaStreamGetCaptureInfo(s, &st, nullptr, nullptr, &deps, nullptr, &nd));
    TNH_REQUIRE(st == cudaStreamCaptureStatusActive && nd == 1, TNH_ERR_CUDA, "heff: unexpected capture state");
    return deps[0];
}

// The launches of one application (x -> y) on stream s. While capturing
// (G != nullptr) the node that reads x and the node that writes y are
// recorded with the position of that pointer among their arguments:
// gather_kernel(tiles, segs, terms, geom, src, dst) reads x as argument 4;
// y is written by gemm_f64_kernel(tasks, ntasks, A, B, C, row_off) as
// argument 4, gemm_tc_kernel(tasks, ntasks, tiles, A, B, C, err, row_off,
// atiles, asegs, aterms, asrc) as argument 5, or splitk_reduce(reds, blocks,
// part, out, row_off) as argument 3.
void launch_chain(HeffPlan& P, bool f64, const double* x, double* y, cudaStream_t s, HeffPlan::Graph* G) {
    const int n1 = (int)P.g1.f64.size(), n4 = (int)P.g4.f64.size();
    if (f64) {
        // the FP64 GEMM of one stage, K-split or not; the last launch writes out
        auto f64_stage = [&](const HeffGemm& Gm, int ntasks, const double* A, const double* B, double* out,
                             const int64_t* roff) {
            if (Gm.split64 > 1) {
                launch_gemm_f64(Gm.d_f64run.as<GemmTask>(), (int)Gm.f64run.size(), Gm.tiles64run, A, B,
                                P.part64.as<double>(), s);
                launch_splitk_reduce(Gm.d_reds64.as<SplitRed>(), Gm.d_red64_blocks.as<RedBlock>(),
                                     (int)Gm.red64_blocks.size(), P.part64.as<double>(), out, roff, s);
            } else {
                launch_gemm_f64(Gm.d_f64.as<GemmTask>(), ntasks, Gm.tiles64, A, B, out, s, roff);
            }
        };
        launch_gather(P.jX, P.oX.d_g64.as<OpGeom>(), x, P.opX.p, 0, s, "heff_pack_x");
        if (G) G->nx = last_node(s);
        f64_stage(P.g1, n1, P.L64.as<double>(), P.opX.as<double>(), P.t1.as<double>(), nullptr);
        launch_w12(P.jW, P.oT.d_g64.as<OpGeom>(), P.t1.as<double>(), P.opT64.p, 0, s);
        f64_stage(P.g4, n4, P.opT64.as<double>(), P.R64.as<double>(), y, P.row_off.as<int64_t>());
        if (G) {
            G->ny = last_node(s);
            G->iy = P.g4.split64 > 1 ? 3 : 4;
            G->ny_args = P.g4.split64 > 1 ? 5 : 6;
        }
    } else {
        launch_gather(P.jX, P.oX.d_gtc.as<OpGeom>(), x, P.opX.p, P.planes, s, "heff_pack_x");
        if (G) G->nx = last_node(s);
        launch_stage(P.g1, P, P.Ltc.as<uint16_t>(), P.opX.as<uint16_t>(), P.t1.p, nullptr, s);
        if (!P.fusedS4) launch_w12(P.jW, P.oT.d_gtc.as<OpGeom>(), P.t1.as<float>(), P.opTtc.p, P.planes, s);
        launch_stage(P.g4, P, P.opTtc.as<uint16_t>(), P.Rtc.as<uint16_t>(), y, P.row_off.as<int64_t>(), s,
                     P.fusedS4);
        if (G) {
            G->ny = last_node(s);
            G->iy = P.g4.split > 1 ? 3 : 5;
            G->ny_args = P.g4.split > 1 ? 5 : 12;
        }
    }
}

std::vector<void*> node_args(cudaGraphNode_t n, int count) {
    cudaKernelNodeParams p{};
    CUDA_CHECK(cudaGraphKernelNodeGetParams(n, &p));
    TNH_REQUIRE(p.kernelParams != nullptr, TNH_ERR_CUDA, "heff: captured kernel without argument array");
    return std::vector<void*>(p.kernelParams, p.kernelParams + count);
}

void patch(cudaGraphExec_t ex, cudaGraphNode_t n, std::vector<void*>& args, int idx, void* slot) {
    cudaKernelNodeParams p{};
    CUDA_CHECK(cudaGraphKernelNodeGetParams(n, &p));
    args[idx] = slot;
    p.kernelParams = args.data();
    p.extra = nullptr;
    CUDA_CHECK(cudaGraphExecKernelNodeSetParams(ex, n, &p));
}

// Capture the chain once (x and y of this call) on a stream of its own (the
// plan's stream may be the legacy default stream, which cannot be
// captured); the graph is replayed on the plan's stream, and later calls
// patch the two pointer arguments.
void capture(HeffPlan& P, HeffPlan::Graph& G, bool f64, const double* x, double* y) {
    cudaStream_t s = nullptr;
    CUDA_CHECK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    struct StreamGuard {
        cudaStream_t s;
        ~StreamGuard() { cudaStreamDestroy(s); }
    } sg{s};
    CUDA_CHECK(cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed));
    try {
        launch_chain(P, f64, x, y, s, &G);
    } catch (...) {
        cudaGraph_t g = nullptr;
        cudaStreamEndCapture(s, &g);
        if (g) cudaGraphDestroy(g);
        throw;
    }
    CUDA_CHECK(cudaStreamEndCapture(s, &G.graph));
    CUDA_CHECK(cudaGraphInstantiate(&G.exec, G.graph, 0));
    G.ix = 4;
    G.ax = node_args(G.nx, 6);
    G.ay = node_args(G.ny, G.ny_args);
    G.x = x;
    G.y = y;
}

// The MPO part of one application (graph replay after the first call).
void heff_chain(HeffPlan& P, tnh_precision prec, const double* x, double* y) {
    cudaStream_t s = P.stream;
    if (P.zero_y && P.n > 0) CUDA_CHECK(cudaMemsetAsync(y, 0, (size_t)P.n * sizeof(double), s));
    if (P.g1.f64.empty() || P.g4.f64.empty() || P.jX.ntiles == 0) {
        if (!P.zero_y && P.n > 0) CUDA_CHECK(cudaMemsetAsync(y, 0, (size_t)P.n * sizeof(double), s));
        return;
    }
    const bool f64 = prec == TNH_FP64;
    HeffPlan::Graph& G = P.graphs[f64 ? 0 : 1];
    Profiler* prof = active_profiler();
    // direct launches while profiling (per-kernel events) and on the first
    // call (kernel attributes are set outside any capture)
    if ((prof && prof->on) || G.calls++ == 0) {
        launch_chain(P, f64, x, y, s, nullptr);
        CUDA_CHECK(cudaGetLastError());
        return;
    }
    if (!G.exec) {
        capture(P, G, f64, x, y);
    } else {
        if (x != G.x) {
            G.x = x;
            patch(G.exec, G.nx, G.ax, G.ix, &G.x);
        }
        if (y != G.y) {
            G.y = y;
            patch(G.exec, G.ny, G.ay, G.iy, &G.y);
        }
    }
    CUDA_CHECK(cudaGraphLaunch(G.exec, s));
}

}  // namespace

void heff_apply(HeffPlan& P, tnh_precision prec, const double* x, double* y) {
    TNH_REQUIRE(prec == TNH_FP64 || prec == P.prec, TNH_ERR_ARG,
                "heff_apply: precision %d not prepared by this plan", (int)prec);
    heff_chain(P, prec, x, y);
    add_projectors(P, x, y);
}

const double* heff_diag(HeffPlan& P) {
    if (P.diag.p) return P.diag.as<double>();
    cudaStream_t s = P.stream;
    P.diag.alloc((size_t)std::max<int64_t>(P.n, 1) * sizeof(double));
    CUDA_CHECK(cudaMemsetAsync(P.diag.p, 0, P.diag.bytes, s));
    if (P.dg_nblocks > 0) {
        const unsigned gx = (unsigned)std::min<int64_t>(std::max<int64_t>(1, (P.dg_maxblock + 255) / 256), 64);
        KScope ks("heff_diag", s);
        heff_diag_kernel<<<dim3(gx, (unsigned)P.dg_nblocks), 256, 0, s>>>(
            P.d_dblocks.as<DiagBlock>(), P.d_dstart.as<int>(), P.d_dterms.as<DiagTerm>(), P.Ld.as<double>(),
            P.Rd.as<double>(), P.dg_wdim, P.dg_zdim, P.dg_d2, P.diag.as<double>());
    }
    CUDA_CHECK(cudaGetLastError());
    return P.diag.as<double>();
}

}  // namespace tnh

using namespace tnh;

extern "C" {

tnh_status tnh_heff_plan(tnh_ctx* ctx, const tnh_tensor* L, const tnh_tensor* W1, const tnh_tensor* W2,
                         const tnh_tensor* R, const tnh_tensor* psi, tnh_precision prec, tnh_heff** plan) {
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    return guard(c, [&] {
        TNH_REQUIRE(c && plan, TNH_ERR_ARG, "tnh_heff_plan: NULL argument");
        CUDA_CHECK(cudaSetDevice(c->device));
        auto P = make_heff(c, parse_tensor(L, "L"), parse_tensor(W1, "W1"), parse_tensor(W2, "W2"),
                           parse_tensor(R, "R"), parse_tensor(psi, "psi", false), prec);
        *plan = reinterpret_cast<tnh_heff*>(P.release());
    });
}

tnh_status tnh_heff_plan_sum(tnh_ctx* ctx, int32_t nterm, const tnh_tensor* L, const tnh_tensor* W1,
                             const tnh_tensor* W2, const tnh_tensor* R, const tnh_tensor* psi, tnh_precision prec,
                             tnh_heff** plan) {
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    return guard(c, [&] {
        TNH_REQUIRE(c && plan && L && W1 && W2 && R && psi, TNH_ERR_ARG, "tnh_heff_plan_sum: NULL argument");
        TNH_REQUIRE(nterm >= 1, TNH_ERR_ARG, "tnh_heff_plan_sum: nterm = %d", nterm);
        CUDA_CHECK(cudaSetDevice(c->device));
        std::vector<Layout> l, w1, w2, r;
        for (int t = 0; t < nterm; ++t) {
            l.push_back(parse_tensor(&L[t], "L"));
            w1.push_back(parse_tensor(&W1[t], "W1"));
            w2.push_back(parse_tensor(&W2[t], "W2"));
            r.push_back(parse_tensor(&R[t], "R"));
            TNH_REQUIRE(l[t].rank() == 3 && r[t].rank() == 3 && w1[t].rank() == 4 && w2[t].rank() == 4,
                        TNH_ERR_ARG, "tnh_heff_plan_sum: ranks must be L 3, W 4, R 3");
        }
        // make_heff synchronises the stream before it returns, after which
        // the staged direct sums are no longer read
        DevBuf bl, bw1, bw2, br;
        Layout sl = direct_sum(l, {1}, bl, c->stream), sw1 = direct_sum(w1, {0, 1}, bw1, c->stream),
               sw2 = direct_sum(w2, {0, 1}, bw2, c->stream), sr = direct_sum(r, {1}, br, c->stream);
        auto P = make_heff(c, sl, sw1, sw2, sr, parse_tensor(psi, "psi", false), prec);
        *plan = reinterpret_cast<tnh_heff*>(P.release());
    });
}

tnh_status tnh_heff_set_projectors(tnh_heff* plan, int32_t k, const double* phi, double weight) {
    auto* P = reinterpret_cast<HeffPlan*>(plan);
    return guard(P ? P->ctx : nullptr, [&] {
        TNH_REQUIRE(P, TNH_ERR_ARG, "tnh_heff_set_projectors: NULL plan");
        set_projectors(*P, k, phi, weight);
        CUDA_CHECK(cudaStreamSynchronize(P->stream));
    });
}

tnh_status tnh_heff_apply(tnh_heff* plan, const double* x, double* y) {
    auto* P = reinterpret_cast<HeffPlan*>(plan);
    return guard(P ? P->ctx : nullptr, [&] {
        TNH_REQUIRE(P && x && y, TNH_ERR_ARG, "tnh_heff_apply: NULL argument");
        TNH_REQUIRE(x != y, TNH_ERR_ARG, "tnh_heff_apply: x and y alias");
        heff_apply(*P, P->prec, x, y);
    });
}

tnh_status tnh_heff_apply_prec(tnh_heff* plan, tnh_precision prec, const double* x, double* y) {
    auto* P = reinterpret_cast<HeffPlan*>(plan);
    return guard(P ? P->ctx : nullptr, [&] {
        TNH_REQUIRE(P && x && y, TNH_ERR_ARG, "tnh_heff_apply_prec: NULL argument");
        TNH_REQUIRE(x != y, TNH_ERR_ARG, "tnh_heff_apply_prec: x and y alias");
        heff_apply(*P, prec, x, y);
    });
}

tnh_status tnh_heff_apply_host(tnh_heff* plan, const double* x, double* y) {
    auto* P = reinterpret_cast<HeffPlan*>(plan);
    return guard(P ? P->ctx : nullptr, [&] {
        TNH_REQUIRE(P && x && y, TNH_ERR_ARG, "tnh_heff_apply_host: NULL argument");
        CUDA_CHECK(cudaSetDevice(P->ctx->device));
        const size_t bytes = (size_t)P->n * sizeof(double);
        if (P->n > 0 && !P->hx.p) {
            AllocScope scope(P->stream);
            P->hx.alloc(bytes);
            P->hy.alloc(bytes);
        }
        if (P->n > 0) {
            CUDA_CHECK(cudaMemcpyAsync(P->hx.p, x, bytes, cudaMemcpyHostToDevice, P->stream));
            heff_apply(*P, P->prec, P->hx.as<double>(), P->hy.as<double>());
            CUDA_CHECK(cudaMemcpyAsync(y, P->hy.p, bytes, cudaMemcpyDeviceToHost, P->stream));
        }
        // the plan's stream is the context's: reading the error flag after y
        // is the one synchronisation of the call
        check_device_flag(P->ctx);
    });
}

tnh_status tnh_heff_diag(tnh_heff* plan, double* d) {
    auto* P = reinterpret_cast<HeffPlan*>(plan);
    return guard(P ? P->ctx : nullptr, [&] {
        TNH_REQUIRE(P && d, TNH_ERR_ARG, "tnh_heff_diag: NULL argument");
        const double* src = heff_diag(*P);
        if (P->n > 0)
            CUDA_CHECK(cudaMemcpyAsync(d, src, (size_t)P->n * sizeof(double), cudaMemcpyDeviceToDevice, P->stream));
        CUDA_CHECK(cudaStreamSynchronize(P->stream));
    });
}

tnh_status tnh_heff_flops(const tnh_heff* plan, double* flops) {
    auto* P = reinterpret_cast<const HeffPlan*>(plan);
    return guard(nullptr, [&] {
        TNH_REQUIRE(P && flops, TNH_ERR_ARG, "tnh_heff_flops: NULL argument");
        *flops = P->flops;
    });
}

tnh_status tnh_heff_flops_detail(const tnh_heff* plan, double* s1, double* s23, double* s4) {
    auto* P = reinterpret_cast<const HeffPlan*>(plan);
    return guard(nullptr, [&] {
        TNH_REQUIRE(P && s1 && s23 && s4, TNH_ERR_ARG, "tnh_heff_flops_detail: NULL argument");
        *s1 = P->f_s1;
        *s23 = P->f_s23;
        *s4 = P->f_s4;
    });
}

tnh_status tnh_heff_tuning(const tnh_heff* plan, int32_t* choice) {
    auto* P = reinterpret_cast<const HeffPlan*>(plan);
    return guard(nullptr, [&] {
        TNH_REQUIRE(P && choice, TNH_ERR_ARG, "tnh_heff_tuning: NULL argument");
        for (int k = 0; k < 4; ++k) choice[k] = P->tune[k];
        choice[4] = P->tune_measured ? 1 : 0;
        choice[5] = P->strategy;
        choice[6] = P->strategy_measured ? 1 : 0;
        choice[7] = P->fusedS4 ? 1 : 0;
    });
}

tnh_status tnh_heff_size(const tnh_heff* plan, int64_t* n) {
    auto* P = reinterpret_cast<const HeffPlan*>(plan);
    return guard(nullptr, [&] {
        TNH_REQUIRE(P && n, TNH_ERR_ARG, "tnh_heff_size: NULL argument");
        *n = P->n;
    });
}

void tnh_heff_free(tnh_heff* plan) {
    auto* P = reinterpret_cast<HeffPlan*>(plan);
    if (!P) return;
    cudaStreamSynchronize(P->stream);
    delete P;
}

}  // extern "C"
