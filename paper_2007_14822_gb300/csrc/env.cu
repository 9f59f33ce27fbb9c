// Environment update of two-site DMRG (the "forming the environment tensors"
// step of Sec. 7.2):
//   dir +1: L'[b,w',b'] = sum L[a,w,a'] A[a,s,b] W[w,w',s,s'] A[a',s',b']
//   dir -1: R'[a,w,a'] = sum A[a,s,b] W[w,w',s,s'] A[a',s',b'] R[b,w',b']
// as three labelled contractions; the bra tensor is A with its arrows
// reversed (real data, Sec. 8.3 dag).
#include "env.h"
#include "tnh_guard.h"

namespace tnh {

namespace {

enum : int64_t { Ea = 1, Ew = 2, Eap = 3, Es = 4, Eb = 5, Ewp = 6, Esp = 7, Ebp = 8 };

Layout lab(Layout T, std::initializer_list<int64_t> labels) {
    int i = 0;
    for (int64_t l : labels) T.inds[i++].label = l;
    return T;
}

Layout dagger(Layout T) {
    for (auto& ix : T.inds) ix.arrow = -ix.arrow;
    for (auto& f : T.flux) f = -f;
    return T;
}

std::vector<int> fsum(const std::vector<int>& a, const std::vector<int>& b) {
    std::vector<int> r(a.size());
    for (size_t k = 0; k < a.size(); ++k) r[k] = a[k] + b[k];
    return r;
}

}  // namespace

EnvPlan::~EnvPlan() = default;

std::unique_ptr<EnvPlan> make_env(Ctx* ctx, int dir, const Layout& E0, const Layout& A0, const Layout& W0,
                                  const Layout& O0) {
    TNH_REQUIRE(dir == 1 || dir == -1, TNH_ERR_ARG, "env_update: dir must be +1 or -1");
    TNH_REQUIRE(E0.rank() == 3 && A0.rank() == 3 && W0.rank() == 4 && O0.rank() == 3, TNH_ERR_ARG,
                "env_update: ranks must be E 3, A 3, W 4, E_out 3");
    cudaStream_t s = ctx->stream;
    auto P = std::make_unique<EnvPlan>();
    P->dir = dir;
    Layout A = lab(A0, {Ea, Es, Eb});
    Layout W = lab(W0, {Ew, Ewp, Es, Esp});
    Layout Ad = lab(dagger(A0), {Eap, Esp, Ebp});
    if (dir == 1) {
        Layout E = lab(E0, {Ea, Ew, Eap});
        Layout O = lab(O0, {Eb, Ewp, Ebp});
        Layout X = make_layout({E.inds[1], E.inds[2], A.inds[1], A.inds[2]}, fsum(E.flux, A.flux));
        Layout Y = make_layout({X.inds[1], X.inds[3], W.inds[1], W.inds[3]}, fsum(X.flux, W.flux));
        P->c1 = plan_contract(E, A, X, s);
        P->c2 = plan_contract(X, W, Y, s);
        P->c3 = plan_contract(Y, Ad, O, s);
        P->x.alloc((size_t)std::max<int64_t>(X.size, 1) * 8);
        P->y.alloc((size_t)std::max<int64_t>(Y.size, 1) * 8);
    } else {
        Layout E = lab(E0, {Eb, Ewp, Ebp});
        Layout O = lab(O0, {Ea, Ew, Eap});
        Layout X = make_layout({A.inds[0], A.inds[1], E.inds[1], E.inds[2]}, fsum(A.flux, E.flux));
        Layout Y = make_layout({X.inds[0], X.inds[3], W.inds[0], W.inds[3]}, fsum(X.flux, W.flux));
        P->c1 = plan_contract(A, E, X, s);
        P->c2 = plan_contract(X, W, Y, s);
        P->c3 = plan_contract(Y, Ad, O, s);
        P->x.alloc((size_t)std::max<int64_t>(X.size, 1) * 8);
        P->y.alloc((size_t)std::max<int64_t>(Y.size, 1) * 8);
    }
    P->flops = P->c1->flops + P->c2->flops + P->c3->flops;
    return P;
}

void run_env(Ctx* ctx, EnvPlan& P, const double* E, const double* A, const double* W, double* out,
             tnh_precision prec) {
    if (P.dir == 1) {
        run_contract(ctx, *P.c1, E, A, P.x.as<double>(), prec, P.ws);
    } else {
        run_contract(ctx, *P.c1, A, E, P.x.as<double>(), prec, P.ws);
    }
    run_contract(ctx, *P.c2, P.x.as<double>(), W, P.y.as<double>(), prec, P.ws);
    run_contract(ctx, *P.c3, P.y.as<double>(), A, out, prec, P.ws);
}

}  // namespace tnh

using namespace tnh;

extern "C" tnh_status tnh_env_update(tnh_ctx* ctx, int32_t dir, const tnh_tensor* E, const tnh_tensor* A,
                                     const tnh_tensor* W, tnh_tensor* E_out, tnh_precision prec) {
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    return guard(c, [&] {
        TNH_REQUIRE(c, TNH_ERR_ARG, "tnh_env_update: ctx NULL");
        TNH_REQUIRE(prec == TNH_FP64 || planes_of(prec) > 0, TNH_ERR_ARG, "tnh_env_update: bad precision");
        CUDA_CHECK(cudaSetDevice(c->device));
        Layout e = parse_tensor(E, "E"), a = parse_tensor(A, "A"), w = parse_tensor(W, "W"),
               o = parse_tensor(E_out, "E_out");
        auto P = make_env(c, dir, e, a, w, o);
        run_env(c, *P, e.data, a.data, w.data, o.data, prec);
        CUDA_CHECK(cudaStreamSynchronize(c->stream));
        check_device_flag(c);
    });
}
