// Effective-Hamiltonian plan: y = H_eff . x for two-site DMRG (Sec. 7.2).
//
//   y[a',s1',s2',b'] = sum L[a,w,a'] W1[w,w1,s1,s1'] W2[w1,w2,s2,s2']
//                          R[b,w2,b'] x[a,s1,s2,b]
//
// evaluated as four labelled contractions S1 (sum a), S2 (sum w, s1),
// S3 (sum w1, s2), S4 (sum w2, b), each a grouped block-pair GEMM.
#include <algorithm>

#include "heff.h"
#include "tnh_guard.h"

namespace tnh {

namespace {

enum : int64_t { La = 1, Lw = 2, Lap = 3, Ls1 = 4, Ls2 = 5, Lb = 6, Lw1 = 7, Ls1p = 8, Lw2 = 9, Ls2p = 10, Lbp = 11 };

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

DevBuf copy_data(const Layout& T, cudaStream_t s) {
    DevBuf b((size_t)std::max<int64_t>(T.size, 1) * sizeof(double));
    if (T.size) CUDA_CHECK(cudaMemcpyAsync(b.p, T.data, (size_t)T.size * sizeof(double),
                                           cudaMemcpyDeviceToDevice, s));
    return b;
}

}  // namespace

HeffPlan::~HeffPlan() = default;

std::unique_ptr<HeffPlan> make_heff(Ctx* ctx, const Layout& L0, const Layout& W10, const Layout& W20,
                                    const Layout& R0, const Layout& psi0, tnh_precision prec, bool copy_inputs) {
    TNH_REQUIRE(L0.rank() == 3 && R0.rank() == 3 && W10.rank() == 4 && W20.rank() == 4 && psi0.rank() == 4,
                TNH_ERR_ARG, "heff_plan: ranks must be L 3, W 4, R 3, psi 4");
    TNH_REQUIRE(prec == TNH_FP64 || planes_of(prec) > 0, TNH_ERR_ARG, "heff_plan: bad precision");
    cudaStream_t s = ctx->stream;
    auto P = std::make_unique<HeffPlan>();
    P->ctx = ctx;
    P->stream = ctx->stream;
    P->prec = prec;
    Layout L = with_labels(L0, {La, Lw, Lap});
    Layout W1 = with_labels(W10, {Lw, Lw1, Ls1, Ls1p});
    Layout W2 = with_labels(W20, {Lw1, Lw2, Ls2, Ls2p});
    Layout R = with_labels(R0, {Lb, Lw2, Lbp});
    Layout X = with_labels(psi0, {La, Ls1, Ls2, Lb});
    // output layout: psi's blocks on the product's indices
    Layout Y = X;
    Y.inds = {L.inds[2], W1.inds[3], W2.inds[3], R.inds[2]};
    for (int i = 0; i < 4; ++i)
        TNH_REQUIRE(Y.inds[i].same_space(X.inds[i]) && Y.inds[i].arrow == X.inds[i].arrow, TNH_ERR_SHAPE,
                    "heff_plan: output index %d does not match psi's (sectors or arrow)", i);
    P->n = X.size;
    P->psi = X;
    // intermediates
    Layout T1 = make_layout({L.inds[1], L.inds[2], X.inds[1], X.inds[2], X.inds[3]}, add_flux(L.flux, X.flux));
    Layout T2 = make_layout({T1.inds[1], T1.inds[3], T1.inds[4], W1.inds[1], W1.inds[3]},
                            add_flux(T1.flux, W1.flux));
    Layout T3 = make_layout({T2.inds[0], T2.inds[2], T2.inds[4], W2.inds[1], W2.inds[3]},
                            add_flux(T2.flux, W2.flux));
    P->c1 = plan_contract(L, X, T1, s);
    P->c2 = plan_contract(T1, W1, T2, s);
    P->c3 = plan_contract(T2, W2, T3, s);
    P->c4 = plan_contract(T3, R, Y, s);
    P->t1.alloc((size_t)std::max<int64_t>(T1.size, 1) * 8);
    P->t2.alloc((size_t)std::max<int64_t>(T2.size, 1) * 8);
    P->t3.alloc((size_t)std::max<int64_t>(T3.size, 1) * 8);
    if (copy_inputs) {
        P->Ld = copy_data(L, s);
        P->Rd = copy_data(R, s);
        P->W1d = copy_data(W1, s);
        P->W2d = copy_data(W2, s);
        P->Lp = P->Ld.as<double>();
        P->Rp = P->Rd.as<double>();
        P->W1p = P->W1d.as<double>();
        P->W2p = P->W2d.as<double>();
    } else {
        P->Lp = L.data;
        P->Rp = R.data;
        P->W1p = W1.data;
        P->W2p = W2.data;
    }
    P->flops = P->c1->flops + P->c2->flops + P->c3->flops + P->c4->flops;
    CUDA_CHECK(cudaStreamSynchronize(s));
    return P;
}

void heff_apply(HeffPlan& P, tnh_precision prec, const double* x, double* y) {
    Ctx* ctx = P.ctx;
    TNH_REQUIRE(prec == TNH_FP64 || prec == P.prec, TNH_ERR_ARG,
                "heff_apply: precision %d not prepared by this plan", (int)prec);
    run_contract(ctx, *P.c1, P.Lp, x, P.t1.as<double>(), prec, P.ws);
    run_contract(ctx, *P.c2, P.t1.as<double>(), P.W1p, P.t2.as<double>(), prec, P.ws);
    run_contract(ctx, *P.c3, P.t2.as<double>(), P.W2p, P.t3.as<double>(), prec, P.ws);
    run_contract(ctx, *P.c4, P.t3.as<double>(), P.Rp, y, prec, P.ws);
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

tnh_status tnh_heff_flops(const tnh_heff* plan, double* flops) {
    auto* P = reinterpret_cast<const HeffPlan*>(plan);
    return guard(nullptr, [&] {
        TNH_REQUIRE(P && flops, TNH_ERR_ARG, "tnh_heff_flops: NULL argument");
        *flops = P->flops;
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
