// Two-site DMRG sweep driver (Sec. 7.2: dmrg(H, psi0, sweeps)).
//
// Host control, device compute. For every bond (j, j+1):
//   theta = A_j * A_{j+1}                         (labelled contraction)
//   E, theta = Lanczos(H_eff(L_j, W_j, W_{j+1}, R_{j+2}), theta)
//   U S V = truncated SVD of theta (rows a_j, s_j)  (cutoff, maxdim, Sec. 5)
//   left-to-right:  A_j = U,   A_{j+1} = S V,  L_{j+1} = update(L_j, A_j, W_j)
//   right-to-left:  A_j = U S, A_{j+1} = V,    R_{j+1} = update(R_{j+2}, A_{j+1}, W_{j+1})
// A sweep is the left-to-right pass over bonds (0,1)..(N-2,N-1) followed by
// the right-to-left pass in reverse (the paper does not define the
// schedule; this is the usual one). The reported energy is the eigenvalue
// at the last bond of the sweep.
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>

#include "env.h"
#include "heff.h"
#include "svd.h"
#include "tnh_guard.h"

namespace tnh {

namespace {

struct DTensor {
    Layout L;
    DevBuf buf;
};

DTensor new_tensor(const std::vector<Index>& inds, const std::vector<int>& flux, cudaStream_t s) {
    DTensor t;
    t.L = make_layout(inds, flux);
    t.buf.alloc((size_t)std::max<int64_t>(t.L.size, 1) * sizeof(double));
    t.L.data = t.buf.as<double>();
    CUDA_CHECK(cudaMemsetAsync(t.buf.p, 0, (size_t)std::max<int64_t>(t.L.size, 1) * sizeof(double), s));
    return t;
}

// element offset of the element (e0, e1, ...) of T (element numbers per index)
int64_t elem_offset(const Layout& T, const std::vector<int64_t>& el) {
    std::vector<int> key(T.rank());
    std::vector<int64_t> loc(T.rank());
    for (int i = 0; i < T.rank(); ++i) {
        int64_t e = el[i];
        int s = 0;
        while (s < T.inds[i].nsect && e >= T.inds[i].dim[s]) e -= T.inds[i].dim[s++];
        TNH_REQUIRE(s < T.inds[i].nsect, TNH_ERR_ARG, "dmrg: boundary element out of range");
        key[i] = s;
        loc[i] = e;
    }
    int b = T.find(key);
    TNH_REQUIRE(b >= 0, TNH_ERR_FLUX, "dmrg: boundary element lies in a forbidden block");
    int64_t off = 0;
    for (int i = 0; i < T.rank(); ++i) off = off * T.bdim(b, i) + loc[i];
    return T.off[b] + off;
}

void set_one(DTensor& t, const std::vector<int64_t>& el, cudaStream_t s) {
    static const double one = 1.0;
    int64_t o = elem_offset(t.L, el);
    CUDA_CHECK(cudaMemcpyAsync(t.L.data + o, &one, sizeof(double), cudaMemcpyHostToDevice, s));
}

Layout relabel(Layout T, std::initializer_list<int64_t> labels) {
    int i = 0;
    for (int64_t l : labels) T.inds[i++].label = l;
    return T;
}

std::vector<int> fsum(const std::vector<int>& a, const std::vector<int>& b) {
    std::vector<int> r(a.size());
    for (size_t k = 0; k < a.size(); ++k) r[k] = a[k] + b[k];
    return r;
}

}  // namespace

}  // namespace tnh

using namespace tnh;

extern "C" tnh_status tnh_dmrg(tnh_ctx* ctx, int32_t N, const tnh_tensor* mpo, int64_t start, int64_t done,
                               const tnh_tensor* mps, const tnh_sweep_params* p, double* energy,
                               tnh_sweep_stat* stats) {
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    return guard(c, [&] {
        TNH_REQUIRE(c && mpo && mps && p && energy, TNH_ERR_ARG, "tnh_dmrg: NULL argument");
        TNH_REQUIRE(N >= 2, TNH_ERR_ARG, "tnh_dmrg: N = %d < 2", N);
        TNH_REQUIRE(p->nsweep >= 1 && p->maxdim && p->cutoff, TNH_ERR_ARG, "tnh_dmrg: empty sweep schedule");
        const tnh_precision prec = (tnh_precision)p->precision;
        const tnh_precision eprec = (tnh_precision)p->env_precision;
        TNH_REQUIRE(prec == TNH_FP64 || planes_of(prec) > 0, TNH_ERR_ARG, "tnh_dmrg: bad precision");
        TNH_REQUIRE(eprec == TNH_FP64 || planes_of(eprec) > 0, TNH_ERR_ARG, "tnh_dmrg: bad env precision");
        CUDA_CHECK(cudaSetDevice(c->device));
        cudaStream_t s = c->stream;
        std::vector<Layout> W;
        std::vector<DTensor> A(N);
        for (int j = 0; j < N; ++j) {
            W.push_back(parse_tensor(&mpo[j], "mpo"));
            Layout a = parse_tensor(&mps[j], "mps");
            TNH_REQUIRE(a.rank() == 3 && W[j].rank() == 4, TNH_ERR_ARG, "tnh_dmrg: MPS rank 3, MPO rank 4");
            A[j] = new_tensor(a.inds, a.flux, s);
            for (int b = 0; b < a.nblocks(); ++b) {
                int d = A[j].L.find(a.key(b));
                CUDA_CHECK(cudaMemcpyAsync(A[j].L.data + A[j].L.off[d], a.data + a.off[b],
                                           (size_t)a.belems(b) * sizeof(double), cudaMemcpyDeviceToDevice, s));
            }
        }
        const int nq = A[0].L.nq();
        const std::vector<int> zero(nq, 0);
        std::vector<DTensor> Ls(N + 1), Rs(N + 1);
        {
            const Index& a0 = A[0].L.inds[0];
            Ls[0] = new_tensor({a0.dag(), W[0].inds[0].dag(), a0}, zero, s);
            set_one(Ls[0], {0, start, 0}, s);
            const Index& bN = A[N - 1].L.inds[2];
            Rs[N] = new_tensor({bN.dag(), W[N - 1].inds[1].dag(), bN}, zero, s);
            set_one(Rs[N], {0, done, 0}, s);
        }
        auto update_R = [&](int j) {   // R_j from R_{j+1}, A_j, W_j
            const Layout& a = A[j].L;
            Rs[j] = new_tensor({a.inds[0], W[j].inds[0], a.inds[0].dag()}, zero, s);
            auto P = make_env(c, -1, Rs[j + 1].L, a, W[j], Rs[j].L);
            run_env(c, *P, Rs[j + 1].L.data, a.data, W[j].data, Rs[j].L.data, eprec);
            CUDA_CHECK(cudaStreamSynchronize(s));
        };
        auto update_L = [&](int j) {   // L_{j+1} from L_j, A_j, W_j
            const Layout& a = A[j].L;
            Ls[j + 1] = new_tensor({a.inds[2], W[j].inds[1], a.inds[2].dag()}, zero, s);
            auto P = make_env(c, 1, Ls[j].L, a, W[j], Ls[j + 1].L);
            run_env(c, *P, Ls[j].L.data, a.data, W[j].data, Ls[j + 1].L.data, eprec);
            CUDA_CHECK(cudaStreamSynchronize(s));
        };
        for (int j = N - 1; j >= 2; --j) update_R(j);

        double E = 0.0;
        const bool dbg = std::getenv("TNH_DEBUG") != nullptr;
        using clk = std::chrono::steady_clock;
        auto since = [](clk::time_point a) { return std::chrono::duration<double>(clk::now() - a).count(); };
        for (int sw = 0; sw < p->nsweep; ++sw) {
            auto t0 = std::chrono::steady_clock::now();
            double ph[6] = {0, 0, 0, 0, 0, 0};   // theta, plan, eigsolve, svd, factors, environment (s)
            double maxerr = 0.0, resid = 0.0;
            int64_t nmv = 0;
            for (int pass = 0; pass < 2; ++pass) {
                for (int step = 0; step < N - 1; ++step) {
                    const int j = pass == 0 ? step : N - 2 - step;
                    const int dir = pass == 0 ? 1 : -1;
                    // theta = A_j * A_{j+1}
                    Layout a1 = relabel(A[j].L, {1, 2, 3});
                    Layout a2 = relabel(A[j + 1].L, {3, 4, 5});
                    DTensor th = new_tensor({a1.inds[0], a1.inds[1], a2.inds[1], a2.inds[2]},
                                            fsum(a1.flux, a2.flux), s);
                    th.L = relabel(th.L, {1, 2, 4, 5});
                    auto tp = clk::now();
                    {
                        auto cp = plan_contract(a1, a2, th.L, s);
                        Workspace ws;
                        run_contract(c, *cp, a1.data, a2.data, th.L.data, eprec, ws);
                        CUDA_CHECK(cudaStreamSynchronize(s));
                    }
                    ph[0] += since(tp);
                    // eigensolver
                    {
                        tp = clk::now();
                        auto P = make_heff(c, Ls[j].L, W[j], W[j + 1], Rs[j + 2].L, th.L, prec);
                        ph[1] += since(tp);
                        tp = clk::now();
                        EigResult r = eigsolve(*P, th.L.data, p->krylov_dim, p->lanczos_tol);
                        ph[2] += since(tp);
                        E = r.energy;
                        resid = r.resid;
                        nmv += r.matvecs;
                    }
                    // truncated SVD
                    tp = clk::now();
                    SvdResult* sv = svd_run(c, th.L, 2, p->cutoff[sw], p->maxdim[sw], p->mindim, dir > 0 ? 0 : 1);
                    ph[3] += since(tp);
                    tp = clk::now();
                    try {
                        SvdShape sh = svd_shape(sv);
                        maxerr = std::max(maxerr, sh.truncerr);
                        if (std::getenv("TNH_DEBUG")) {
                            int kept = 0;
                            for (int d : sh.dims) kept += d;
                            std::fprintf(stderr, "dmrg: sweep %d bond %d dir %+d E %.14f kept %d in %zu sectors truncerr %.3e\n",
                                         sw, j, dir, E, kept, sh.dims.size(), sh.truncerr);
                        }
                        Index link;
                        link.nsect = (int)sh.dims.size();
                        link.nq = nq;
                        link.arrow = 1;
                        for (auto& q : sh.qn) link.qn.insert(link.qn.end(), q.begin(), q.end());
                        link.dim = sh.dims;
                        link.finish();
                        DTensor U = new_tensor({th.L.inds[0], th.L.inds[1], link.dag()}, zero, s);
                        DTensor V = new_tensor({link, th.L.inds[2], th.L.inds[3]}, th.L.flux, s);
                        svd_fetch(sv, U.L, nullptr, V.L, dir > 0 ? 2 : 1);
                        A[j] = std::move(U);
                        A[j + 1] = std::move(V);
                    } catch (...) {
                        svd_delete(sv);
                        throw;
                    }
                    svd_delete(sv);
                    ph[4] += since(tp);
                    tp = clk::now();
                    if (dir > 0) update_L(j);
                    else update_R(j + 1);
                    ph[5] += since(tp);
                }
            }
            CUDA_CHECK(cudaStreamSynchronize(s));
            check_device_flag(c);
            double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
            if (dbg)
                std::fprintf(stderr,
                             "dmrg: sweep %d %.3f s: theta %.3f, H_eff plan %.3f, eigensolver %.3f, SVD %.3f, "
                             "factors %.3f, environment %.3f\n",
                             sw, secs, ph[0], ph[1], ph[2], ph[3], ph[4], ph[5]);
            if (stats) {
                tnh_sweep_stat& st = stats[sw];
                st.sweep = sw;
                st.energy = E;
                st.resid = resid;
                st.truncerr = maxerr;
                int ml = 0;
                for (int j = 0; j < N; ++j) ml = std::max<int>(ml, (int)A[j].L.inds[2].total);
                st.maxlink = ml;
                st.matvecs = nmv;
                st.seconds = secs;
            }
        }
        *energy = E;
    });
}
