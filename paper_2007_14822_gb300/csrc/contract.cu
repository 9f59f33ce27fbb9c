// Labelled block-sparse contraction: planning (host) and execution (device).
//
// C = A * B sums every label that A and B share (Sec. 4, Sec. 9.1). For
// block-sparse storage the product is the set of dense block-pair products
// whose contracted sectors agree (Sec. 9.4). Pairs that land on the same C
// block are concatenated along K so one GEMM task owns each C block: the
// reduction is deterministic and needs no atomics.
//
// Execution is permute-into-GEMM-operands ("TTGT", Sec. 9.4) with the
// permutation fused into the operand packing pass, which also converts
// float64 into the split-bf16 tile format that the tcgen05 GEMM consumes.
#include <algorithm>
#include <map>

#include "tnh_guard.h"
#include "tnh_internal.h"

namespace tnh {

namespace {

std::vector<int64_t> row_major_strides(const Layout& T, int b) {
    int r = T.rank();
    std::vector<int64_t> s(r, 1);
    for (int i = r - 2; i >= 0; --i) s[i] = s[i + 1] * T.bdim(b, i + 1);
    return s;
}

int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

}  // namespace

std::unique_ptr<ContractPlan> plan_contract(const Layout& A, const Layout& B, const Layout& C,
                                            cudaStream_t s) {
    const int ra = A.rank(), rb = B.rank(), rc = C.rank();
    auto lab = [](const Layout& T) {
        std::vector<int64_t> l;
        for (auto& ix : T.inds) l.push_back(ix.label);
        return l;
    };
    auto la = lab(A), lb = lab(B), lc = lab(C);
    auto uniq = [](std::vector<int64_t> v) {
        std::sort(v.begin(), v.end());
        return std::adjacent_find(v.begin(), v.end()) == v.end();
    };
    TNH_REQUIRE(uniq(la) && uniq(lb) && uniq(lc), TNH_ERR_LABEL, "contract: repeated label in a tensor");
    std::vector<int> ia, ib, fa, fb;
    for (int i = 0; i < ra; ++i) {
        auto it = std::find(lb.begin(), lb.end(), la[i]);
        if (it != lb.end()) {
            ia.push_back(i);
            ib.push_back((int)(it - lb.begin()));
        } else {
            fa.push_back(i);
        }
    }
    for (int j = 0; j < rb; ++j)
        if (std::find(la.begin(), la.end(), lb[j]) == la.end()) fb.push_back(j);
    TNH_REQUIRE((int)(fa.size() + fb.size()) == rc, TNH_ERR_LABEL,
                "contract: C has %d indices, the product has %zu free ones", rc, fa.size() + fb.size());
    for (size_t k = 0; k < ia.size(); ++k) {
        const Index &x = A.inds[ia[k]], &y = B.inds[ib[k]];
        TNH_REQUIRE(x.same_space(y), TNH_ERR_SHAPE, "contract: label %lld has different sectors",
                    (long long)x.label);
        TNH_REQUIRE(x.arrow != y.arrow, TNH_ERR_ARROW,
                    "contract: contracted label %lld has equal arrows", (long long)x.label);
    }
    // position in C of every free index
    std::vector<int> ca(fa.size()), cb(fb.size());
    for (size_t k = 0; k < fa.size(); ++k) {
        auto it = std::find(lc.begin(), lc.end(), la[fa[k]]);
        TNH_REQUIRE(it != lc.end(), TNH_ERR_LABEL, "contract: free label %lld missing in C",
                    (long long)la[fa[k]]);
        ca[k] = (int)(it - lc.begin());
        TNH_REQUIRE(C.inds[ca[k]].same_space(A.inds[fa[k]]) && C.inds[ca[k]].arrow == A.inds[fa[k]].arrow,
                    TNH_ERR_SHAPE, "contract: C index for label %lld differs from A's", (long long)la[fa[k]]);
    }
    for (size_t k = 0; k < fb.size(); ++k) {
        auto it = std::find(lc.begin(), lc.end(), lb[fb[k]]);
        TNH_REQUIRE(it != lc.end(), TNH_ERR_LABEL, "contract: free label %lld missing in C",
                    (long long)lb[fb[k]]);
        cb[k] = (int)(it - lc.begin());
        TNH_REQUIRE(C.inds[cb[k]].same_space(B.inds[fb[k]]) && C.inds[cb[k]].arrow == B.inds[fb[k]].arrow,
                    TNH_ERR_SHAPE, "contract: C index for label %lld differs from B's", (long long)lb[fb[k]]);
    }
    const int nq = C.nq();
    if (C.nblocks() > 0 && A.nblocks() > 0 && B.nblocks() > 0) {
        std::vector<int> f(nq);
        for (int k = 0; k < nq; ++k) f[k] = A.flux[k] + B.flux[k];
        TNH_REQUIRE(f == C.flux, TNH_ERR_FLUX, "contract: C flux is not flux(A) + flux(B)");
    }
    TNH_REQUIRE(C.packed_total() <= C.size || C.nblocks() == 0, TNH_ERR_SHAPE, "contract: C too small");

    // B blocks keyed by their contracted sectors (in A's contracted order)
    std::map<std::vector<int>, std::vector<int>> bmap;
    for (int b = 0; b < B.nblocks(); ++b) {
        std::vector<int> k;
        for (int j : ib) k.push_back(B.sect[(size_t)b * rb + j]);
        bmap[k].push_back(b);
    }
    // pairs per C block
    std::vector<std::vector<std::pair<int, int>>> pairs(C.nblocks());
    for (int a = 0; a < A.nblocks(); ++a) {
        std::vector<int> k;
        for (int i : ia) k.push_back(A.sect[(size_t)a * ra + i]);
        auto it = bmap.find(k);
        if (it == bmap.end()) continue;
        for (int b : it->second) {
            std::vector<int> ck(rc);
            for (size_t q = 0; q < fa.size(); ++q) ck[ca[q]] = A.sect[(size_t)a * ra + fa[q]];
            for (size_t q = 0; q < fb.size(); ++q) ck[cb[q]] = B.sect[(size_t)b * rb + fb[q]];
            int c = C.find(ck);
            TNH_REQUIRE(c >= 0, TNH_ERR_FLUX, "contract: a block pair lands outside C's blocks");
            pairs[c].push_back({a, b});
        }
    }

    auto P = std::make_unique<ContractPlan>();
    P->c_total = C.size;
    int64_t a64 = 0, b64 = 0, atile = 0, btile = 0, cel = 0;
    int tf = 0, tt = 0;
    bool uncovered = false;
    for (int c = 0; c < C.nblocks(); ++c) {
        if (pairs[c].empty()) { uncovered = true; continue; }
        const int t = (int)P->tasks_f64.size();
        int a0 = pairs[c][0].first, b0 = pairs[c][0].second;
        auto sa0 = row_major_strides(A, a0);
        auto sb0 = row_major_strides(B, b0);
        int64_t M = 1, N = 1;
        for (int i : fa) M *= A.bdim(a0, i);
        for (int j : fb) N *= B.bdim(b0, j);
        int64_t K = 0;
        for (auto& pr : pairs[c]) {
            int a = pr.first, b = pr.second;
            auto sa = row_major_strides(A, a);
            auto sb = row_major_strides(B, b);
            Piece pa{}, pb{};
            pa.src_off = A.off[a];
            pa.nr = (int)fa.size();
            pa.nc = (int)ia.size();
            int64_t kp = 1;
            for (int q = 0; q < pa.nr; ++q) { pa.dims[q] = A.bdim(a, fa[q]); pa.strides[q] = sa[fa[q]]; }
            for (int q = 0; q < pa.nc; ++q) {
                pa.dims[pa.nr + q] = A.bdim(a, ia[q]);
                pa.strides[pa.nr + q] = sa[ia[q]];
                kp *= pa.dims[pa.nr + q];
            }
            pa.rows = (int)M;
            pa.cols = (int)kp;
            pa.task = t;
            pa.row0 = 0;
            pa.col0 = (int)K;
            pb.src_off = B.off[b];
            pb.nr = (int)fb.size();
            pb.nc = (int)ib.size();
            for (int q = 0; q < pb.nr; ++q) { pb.dims[q] = B.bdim(b, fb[q]); pb.strides[q] = sb[fb[q]]; }
            for (int q = 0; q < pb.nc; ++q) {
                pb.dims[pb.nr + q] = B.bdim(b, ib[q]);
                pb.strides[pb.nr + q] = sb[ib[q]];
            }
            pb.rows = (int)N;
            pb.cols = (int)kp;
            pb.task = t;
            pb.row0 = 0;
            pb.col0 = (int)K;
            P->packA.push_back(pa);
            P->packB.push_back(pb);
            K += kp;
        }
        (void)sa0;
        (void)sb0;
        TNH_REQUIRE(M < (1 << 30) && N < (1 << 30) && K < (1 << 30), TNH_ERR_SHAPE, "contract: block too large");
        // unpack piece: Ct[M][N] -> C block
        auto scs = row_major_strides(C, c);
        Piece pc{};
        pc.src_off = C.off[c];   // destination block offset
        pc.nr = (int)fa.size();
        pc.nc = (int)fb.size();
        for (int q = 0; q < pc.nr; ++q) { pc.dims[q] = C.bdim(c, ca[q]); pc.strides[q] = scs[ca[q]]; }
        for (int q = 0; q < pc.nc; ++q) { pc.dims[pc.nr + q] = C.bdim(c, cb[q]); pc.strides[pc.nr + q] = scs[cb[q]]; }
        pc.rows = (int)M;
        pc.cols = (int)N;
        pc.task = t;
        pc.row0 = 0;
        pc.col0 = 0;
        P->unpackC.push_back(pc);
        P->cbase.push_back(cel);
        P->ldc.push_back((int)N);

        GemmTask g{};
        g.M = (int)M; g.N = (int)N; g.K = (int)K;
        g.mt = (int)((M + kF64TileM - 1) / kF64TileM);
        g.nt = (int)((N + kF64TileN - 1) / kF64TileN);
        g.kt = (int)((K + kF64TileK - 1) / kF64TileK);
        g.lda = g.ldb = (int)round_up(K, kF64TileK);
        g.a_base = a64;
        g.b_base = b64;
        g.c_base = cel;
        g.ldc = (int)N;
        g.tile0 = tf;
        a64 += (int64_t)g.mt * kF64TileM * g.lda;
        b64 += (int64_t)g.nt * kF64TileN * g.ldb;
        tf += g.mt * g.nt;
        P->tasks_f64.push_back(g);

        GemmTask h = g;
        h.mt = (int)((M + kTcTileM - 1) / kTcTileM);
        h.nt = (int)((N + kTcTileN - 1) / kTcTileN);
        h.kt = (int)((K + kTcTileK - 1) / kTcTileK);
        h.a_base = atile;
        h.b_base = btile;
        h.tile0 = tt;
        atile += (int64_t)h.mt * h.kt;
        btile += (int64_t)h.nt * h.kt;
        tt += h.mt * h.nt;
        P->tasks_tc.push_back(h);

        cel += M * N;
        P->flops += 2.0 * (double)M * (double)N * (double)K;
    }
    P->ntiles_f64 = tf;
    P->ntiles_tc = tt;
    P->a_elems_f64 = a64;
    P->b_elems_f64 = b64;
    P->a_tiles = atile;
    P->b_tiles = btile;
    P->c_elems = cel;
    (void)uncovered;
    if (!uncovered) P->c_total = 0;   // every C block is written by a task

    std::vector<Chunk> ch;
    std::vector<OpGeom> gA64, gB64, gAtc, gBtc;
    for (auto& g : P->tasks_f64) {
        gA64.push_back(OpGeom{g.a_base, g.lda});
        gB64.push_back(OpGeom{g.b_base, g.ldb});
    }
    for (auto& g : P->tasks_tc) {
        gAtc.push_back(OpGeom{g.a_base, g.kt});
        gBtc.push_back(OpGeom{g.b_base, g.kt});
    }
    P->d_packA = upload(P->packA, s);
    P->d_packB = upload(P->packB, s);
    P->d_unpack = upload(P->unpackC, s);
    make_chunks(P->packA, ch);
    P->nchA = (int)ch.size();
    P->d_chA = upload(ch, s);
    make_chunks(P->packB, ch);
    P->nchB = (int)ch.size();
    P->d_chB = upload(ch, s);
    make_chunks(P->unpackC, ch);
    P->nchC = (int)ch.size();
    P->d_chC = upload(ch, s);
    P->d_geomA_f64 = upload(gA64, s);
    P->d_geomB_f64 = upload(gB64, s);
    P->d_geomA_tc = upload(gAtc, s);
    P->d_geomB_tc = upload(gBtc, s);
    P->d_tasks_f64 = upload(P->tasks_f64, s);
    P->d_tasks_tc = upload(P->tasks_tc, s);
    P->d_cbase = upload(P->cbase, s);
    P->d_ldc = upload(P->ldc, s);
    // the host vectors must stay alive until the async uploads have run
    CUDA_CHECK(cudaStreamSynchronize(s));
    return P;
}

double contract_flops(const Layout& A, const Layout& B) {
    // the block pairs plan_contract would form: contracted sectors equal
    std::vector<int> ia, ib;
    for (int i = 0; i < A.rank(); ++i)
        for (int j = 0; j < B.rank(); ++j)
            if (A.inds[i].label == B.inds[j].label) { ia.push_back(i); ib.push_back(j); }
    std::map<std::vector<int>, std::vector<int>> bmap;
    for (int b = 0; b < B.nblocks(); ++b) {
        std::vector<int> k;
        for (int j : ib) k.push_back(B.sect[(size_t)b * B.rank() + j]);
        bmap[k].push_back(b);
    }
    double f = 0.0;
    for (int a = 0; a < A.nblocks(); ++a) {
        std::vector<int> k;
        double K = 1.0;
        for (int i : ia) { k.push_back(A.sect[(size_t)a * A.rank() + i]); K *= A.bdim(a, i); }
        auto it = bmap.find(k);
        if (it == bmap.end()) continue;
        const double M = (double)A.belems(a) / K;
        for (int b : it->second) f += 2.0 * M * ((double)B.belems(b) / K) * K;
    }
    return f;
}

void run_contract(Ctx* ctx, const ContractPlan& P, const double* A, const double* B, double* C,
                  tnh_precision prec, Workspace& ws) {
    cudaStream_t s = ctx->stream;
    if (P.c_total > 0) CUDA_CHECK(cudaMemsetAsync(C, 0, (size_t)P.c_total * sizeof(double), s));
    if (P.tasks_f64.empty()) return;
    ws.ensure(ws.c, (size_t)P.c_elems * sizeof(double));
    const int ntask = (int)P.tasks_f64.size();
    if (prec == TNH_FP64) {
        size_t ab = (size_t)P.a_elems_f64 * sizeof(double), bb = (size_t)P.b_elems_f64 * sizeof(double);
        ws.ensure(ws.a, ab);
        ws.ensure(ws.b, bb);
        CUDA_CHECK(cudaMemsetAsync(ws.a.p, 0, ab, s));
        CUDA_CHECK(cudaMemsetAsync(ws.b.p, 0, bb, s));
        launch_pack_f64(P.d_packA.as<Piece>(), P.d_chA.as<Chunk>(), P.nchA, P.d_geomA_f64.as<OpGeom>(), A,
                        ws.a.as<double>(), s);
        launch_pack_f64(P.d_packB.as<Piece>(), P.d_chB.as<Chunk>(), P.nchB, P.d_geomB_f64.as<OpGeom>(), B,
                        ws.b.as<double>(), s);
        launch_gemm_f64(P.d_tasks_f64.as<GemmTask>(), ntask, P.ntiles_f64, ws.a.as<double>(),
                        ws.b.as<double>(), ws.c.as<double>(), s);
    } else {
        int planes = planes_of(prec);
        TNH_REQUIRE(planes > 0, TNH_ERR_ARG, "contract: unknown precision %d", (int)prec);
        size_t ab = (size_t)P.a_tiles * planes * kTcTileElems * 2;
        size_t bb = (size_t)P.b_tiles * planes * kTcTileElems * 2;
        ws.ensure(ws.a, ab);
        ws.ensure(ws.b, bb);
        CUDA_CHECK(cudaMemsetAsync(ws.a.p, 0, ab, s));
        CUDA_CHECK(cudaMemsetAsync(ws.b.p, 0, bb, s));
        launch_pack_bf16(P.d_packA.as<Piece>(), P.d_chA.as<Chunk>(), P.nchA, P.d_geomA_tc.as<OpGeom>(), A,
                         ws.a.as<uint16_t>(), planes, s);
        launch_pack_bf16(P.d_packB.as<Piece>(), P.d_chB.as<Chunk>(), P.nchB, P.d_geomB_tc.as<OpGeom>(), B,
                         ws.b.as<uint16_t>(), planes, s);
        launch_gemm_tc(P.d_tasks_tc.as<GemmTask>(), ntask, P.ntiles_tc, ws.a.as<uint16_t>(),
                       ws.b.as<uint16_t>(), ws.c.as<double>(), planes, ctx->num_sms,
                       ctx->d_flag.as<int>(), s);
    }
    launch_unpack(P.d_unpack.as<Piece>(), P.d_chC.as<Chunk>(), P.nchC, P.d_cbase.as<int64_t>(),
                  P.d_ldc.as<int>(), ws.c.as<double>(), C, s);
    CUDA_CHECK(cudaGetLastError());
}

}  // namespace tnh

using namespace tnh;

extern "C" tnh_status tnh_contract(tnh_ctx* ctx, const tnh_tensor* A, const tnh_tensor* B, tnh_tensor* C,
                                   tnh_precision prec) {
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    return guard(c, [&] {
        TNH_REQUIRE(c, TNH_ERR_ARG, "tnh_contract: ctx NULL");
        TNH_REQUIRE(prec == TNH_FP64 || planes_of(prec) > 0, TNH_ERR_ARG, "tnh_contract: bad precision");
        CUDA_CHECK(cudaSetDevice(c->device));
        Layout a = parse_tensor(A, "A"), b = parse_tensor(B, "B"), cc = parse_tensor(C, "C");
        auto P = plan_contract(a, b, cc, c->stream);
        Workspace ws;
        run_contract(c, *P, a.data, b.data, cc.data, prec, ws);
        // workspace and plan are freed on return: wait for the kernels using them
        CUDA_CHECK(cudaStreamSynchronize(c->stream));
        check_device_flag(c);
    });
}
