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
//
// Sum of MPOs (Sec. 7.2): H = sum_t H_t is run as the direct sum of the
// terms' MPOs. Every MPO link index gets the sectors of all terms in turn,
// the site tensors are block diagonal (a block never joins two terms) and
// the boundary environments select every term's start / done state. The
// environments of all terms are then the sectors of one block-sparse
// environment, one H_eff plan covers every term in each grouped launch, and
// S4 sums the terms along its K dimension: the loop over terms is part of the
// grouped GEMMs, with no block of the explicitly summed MPO formed.
//
// Checkpoint and resume (the paper saves MPS to HDF5 files, Sec. 10; here a
// binary file): with a checkpoint path set on the context, the driver writes
// the MPS, the environments valid at that point (L_0..L_j and R_{j+2}..R_N
// for the next bond j), the position (sweep, pass, step) and the statistics
// so far after every `every` bonds and at the end of every sweep; a resumed
// run loads them and continues the schedule at that bond. The kernels are
// deterministic, so a resumed FP64 run reproduces the uninterrupted one.
//
// Excited states (Sec. 7.2): for every previous state P_i the driver keeps
// overlap environments LO_i (sites left of the bond) and RO_i (right of
// it); phi_i = LO_i P_i[j] P_i[j+1] RO_i is P_i in the current two-site
// basis, and weight * phi_i <phi_i, x> is added to every H_eff . x.
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <string>
#include <algorithm>

#include "env.h"
#include "heff.h"
#include "svd.h"
#include "tnh_guard.h"

namespace tnh {

namespace {

using DTensor = OwnedTensor;

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

// out = A * B in float64 (labels of A, B and out decide the contraction)
void contract64(Ctx* c, const Layout& A, const Layout& B, const Layout& out) {
    auto P = plan_contract(A, B, out, c->stream);
    Workspace ws;
    run_contract(c, *P, A.data, B.data, out.data, TNH_FP64, ws);
    CUDA_CHECK(cudaStreamSynchronize(c->stream));
}

// ---- overlap environments of a previous state P with the MPS A (real data:
// the bra is P with its arrows reversed). LO [p (Out), a (In)] covers the
// sites left of a link, RO [p (In), a (Out)] the sites right of it.
enum : int64_t { Opa = 1, Oa, Os, Opb, Ob, Os2, Opc };

// LO' [pb, b] = sum LO[pa, a] P[pa, s, pb] A[a, s, b]
DTensor overlap_left(Ctx* c, const Layout& LO, const Layout& P, const Layout& A) {
    cudaStream_t s = c->stream;
    Layout lo = relabel(LO, {Opa, Oa});
    Layout pb = relabel(dagger(P), {Opa, Os, Opb});
    Layout ak = relabel(A, {Oa, Os, Ob});
    DTensor X = new_tensor({lo.inds[1], pb.inds[1], pb.inds[2]}, fsum(lo.flux, pb.flux), s);
    X.L = relabel(X.L, {Oa, Os, Opb});
    contract64(c, lo, pb, X.L);
    DTensor out = new_tensor({pb.inds[2], A.inds[2]}, fsum(X.L.flux, A.flux), s);
    out.L = relabel(out.L, {Opb, Ob});
    contract64(c, X.L, ak, out.L);
    return out;
}

// RO' [pa, a] = sum P[pa, s, pb] A[a, s, b] RO[pb, b]
DTensor overlap_right(Ctx* c, const Layout& RO, const Layout& P, const Layout& A) {
    cudaStream_t s = c->stream;
    Layout ro = relabel(RO, {Opb, Ob});
    Layout pb = relabel(dagger(P), {Opa, Os, Opb});
    Layout ak = relabel(A, {Oa, Os, Ob});
    DTensor Y = new_tensor({pb.inds[0], pb.inds[1], ro.inds[1]}, fsum(pb.flux, ro.flux), s);
    Y.L = relabel(Y.L, {Opa, Os, Ob});
    contract64(c, pb, ro, Y.L);
    DTensor out = new_tensor({pb.inds[0], A.inds[0]}, fsum(Y.L.flux, A.flux), s);
    out.L = relabel(out.L, {Opa, Oa});
    contract64(c, Y.L, ak, out.L);
    return out;
}

// phi[a, s1, s2, b] = sum LO[pa, a] P1[pa, s1, pc] P2[pc, s2, pb] RO[pb, b],
// written into `out` (theta's layout). The contraction yields the bra, whose
// arrow-reversed layout has the same blocks and offsets as theta's.
void projected_state(Ctx* c, const Layout& LO, const Layout& P1, const Layout& P2, const Layout& RO,
                     const Layout& theta, double* out) {
    cudaStream_t s = c->stream;
    Layout lo = relabel(LO, {Opa, Oa});
    Layout p1 = relabel(dagger(P1), {Opa, Os, Opc});
    Layout p2 = relabel(dagger(P2), {Opc, Os2, Opb});
    Layout ro = relabel(RO, {Opb, Ob});
    DTensor Y1 = new_tensor({lo.inds[1], p1.inds[1], p1.inds[2]}, fsum(lo.flux, p1.flux), s);
    Y1.L = relabel(Y1.L, {Oa, Os, Opc});
    contract64(c, lo, p1, Y1.L);
    DTensor Y2 = new_tensor({Y1.L.inds[0], Y1.L.inds[1], p2.inds[1], p2.inds[2]}, fsum(Y1.L.flux, p2.flux), s);
    Y2.L = relabel(Y2.L, {Oa, Os, Os2, Opb});
    contract64(c, Y1.L, p2, Y2.L);
    Layout bra = relabel(dagger(theta), {Oa, Os, Os2, Ob});
    TNH_REQUIRE(bra.inds[0].same_space(Y2.L.inds[0]) && bra.inds[3].same_space(ro.inds[1]), TNH_ERR_SHAPE,
                "dmrg: previous state and MPS disagree on a link");
    bra.data = out;
    CUDA_CHECK(cudaMemsetAsync(out, 0, (size_t)std::max<int64_t>(theta.size, 1) * sizeof(double), s));
    contract64(c, Y2.L, ro, bra);
}

// ---- checkpoint file
//   "TNHCKPT1", int32 N, nq, sweep, pass, step, ndone
//   double energy, resid, maxerr, seconds; int64 matvecs
//   ndone x tnh_sweep_stat (the completed sweeps)
//   N tensors (the MPS), then for k = 0..N: int32 flag + tensor if set (L_k),
//   then the same for R_k
// tensor: int32 rank; per index int64 label, int32 nsect, nq, arrow, qn
// [nsect*nq], dim [nsect]; int32 flux [nq]; int64 size; float64 data [size].
constexpr char kCkptMagic[8] = {'T', 'N', 'H', 'C', 'K', 'P', 'T', '1'};

struct Ckpt {
    int N = 0, nq = 0, sweep = 0, pass = 0, step = 0;
    double energy = 0, resid = 0, maxerr = 0, seconds = 0;
    int64_t matvecs = 0;
    std::vector<tnh_sweep_stat> done;
};

struct File {
    FILE* f = nullptr;
    std::string path;
    File(const std::string& p, const char* mode) : path(p) {
        f = std::fopen(p.c_str(), mode);
        TNH_REQUIRE(f != nullptr, TNH_ERR_ARG, "dmrg checkpoint: cannot open %s", p.c_str());
    }
    ~File() { if (f) std::fclose(f); }
    void put(const void* p, size_t n) {
        TNH_REQUIRE(std::fwrite(p, 1, n, f) == n, TNH_ERR_ARG, "dmrg checkpoint: write to %s failed", path.c_str());
    }
    void get(void* p, size_t n) {
        TNH_REQUIRE(std::fread(p, 1, n, f) == n, TNH_ERR_ARG, "dmrg checkpoint: %s is truncated", path.c_str());
    }
    template <class T> void put(const T& v) { put(&v, sizeof v); }
    template <class T> T get() { T v; get(&v, sizeof v); return v; }
};

void put_tensor(File& F, const Layout& T, cudaStream_t s) {
    F.put<int32_t>(T.rank());
    for (const Index& ix : T.inds) {
        F.put<int64_t>(ix.label);
        F.put<int32_t>(ix.nsect);
        F.put<int32_t>(ix.nq);
        F.put<int32_t>(ix.arrow);
        F.put(ix.qn.data(), ix.qn.size() * sizeof(int));
        F.put(ix.dim.data(), ix.dim.size() * sizeof(int));
    }
    F.put(T.flux.data(), T.flux.size() * sizeof(int));
    F.put<int64_t>(T.size);
    std::vector<double> h((size_t)T.size);
    if (T.size) {
        CUDA_CHECK(cudaMemcpyAsync(h.data(), T.data, (size_t)T.size * sizeof(double), cudaMemcpyDeviceToHost, s));
        CUDA_CHECK(cudaStreamSynchronize(s));
    }
    F.put(h.data(), h.size() * sizeof(double));
}

DTensor get_tensor(File& F, int nq, cudaStream_t s) {
    const int rank = F.get<int32_t>();
    TNH_REQUIRE(rank >= 1 && rank <= kMaxDims, TNH_ERR_ARG, "dmrg checkpoint: %s: bad tensor rank", F.path.c_str());
    std::vector<Index> inds(rank);
    for (Index& ix : inds) {
        ix.label = F.get<int64_t>();
        ix.nsect = F.get<int32_t>();
        ix.nq = F.get<int32_t>();
        ix.arrow = F.get<int32_t>();
        TNH_REQUIRE(ix.nsect >= 1 && ix.nsect < (1 << 20) && ix.nq == nq && (ix.arrow == 1 || ix.arrow == -1),
                    TNH_ERR_ARG, "dmrg checkpoint: %s: bad index", F.path.c_str());
        ix.qn.resize((size_t)ix.nsect * nq);
        ix.dim.resize(ix.nsect);
        F.get(ix.qn.data(), ix.qn.size() * sizeof(int));
        F.get(ix.dim.data(), ix.dim.size() * sizeof(int));
        for (int d : ix.dim) TNH_REQUIRE(d >= 1, TNH_ERR_ARG, "dmrg checkpoint: %s: bad sector", F.path.c_str());
        ix.finish();
    }
    std::vector<int> flux(nq);
    F.get(flux.data(), flux.size() * sizeof(int));
    DTensor t = new_tensor(inds, flux, s);
    const int64_t n = F.get<int64_t>();
    TNH_REQUIRE(n == t.L.size, TNH_ERR_ARG, "dmrg checkpoint: %s: tensor size %lld, layout %lld", F.path.c_str(),
                (long long)n, (long long)t.L.size);
    std::vector<double> h((size_t)n);
    F.get(h.data(), h.size() * sizeof(double));
    if (n) {
        CUDA_CHECK(cudaMemcpyAsync(t.L.data, h.data(), (size_t)n * sizeof(double), cudaMemcpyHostToDevice, s));
        CUDA_CHECK(cudaStreamSynchronize(s));
    }
    return t;
}

// Write the state before bond `step` of `pass` in `sweep` (L_0..L_j and
// R_{j+2}..R_N valid, j that bond); written to path.tmp, then renamed.
void write_checkpoint(const std::string& path, const Ckpt& st, const std::vector<DTensor>& A,
                      const std::vector<DTensor>& Ls, const std::vector<DTensor>& Rs, cudaStream_t s) {
    const int N = st.N;
    const int j = st.pass == 0 ? st.step : N - 2 - st.step;
    const std::string tmp = path + ".tmp";
    {
        File F(tmp, "wb");
        F.put(kCkptMagic, sizeof kCkptMagic);
        for (int v : {st.N, st.nq, st.sweep, st.pass, st.step, (int)st.done.size()}) F.put<int32_t>(v);
        for (double v : {st.energy, st.resid, st.maxerr, st.seconds}) F.put<double>(v);
        F.put<int64_t>(st.matvecs);
        for (const tnh_sweep_stat& d : st.done) F.put(d);
        for (int k = 0; k < N; ++k) put_tensor(F, A[k].L, s);
        for (int k = 0; k <= N; ++k) {
            F.put<int32_t>(k <= j);
            if (k <= j) put_tensor(F, Ls[k].L, s);
        }
        for (int k = 0; k <= N; ++k) {
            F.put<int32_t>(k >= j + 2);
            if (k >= j + 2) put_tensor(F, Rs[k].L, s);
        }
        TNH_REQUIRE(std::fflush(F.f) == 0, TNH_ERR_ARG, "dmrg checkpoint: write to %s failed", tmp.c_str());
    }
    TNH_REQUIRE(std::rename(tmp.c_str(), path.c_str()) == 0, TNH_ERR_ARG, "dmrg checkpoint: cannot rename %s",
                tmp.c_str());
}

struct Loaded {
    Ckpt st;
    std::vector<DTensor> A, Ls, Rs;
};

Loaded read_checkpoint(const std::string& path, cudaStream_t s) {
    File F(path, "rb");
    char m[8];
    F.get(m, sizeof m);
    TNH_REQUIRE(std::equal(m, m + 8, kCkptMagic), TNH_ERR_ARG, "dmrg checkpoint: %s is not a checkpoint",
                path.c_str());
    Loaded r;
    Ckpt& st = r.st;
    st.N = F.get<int32_t>();
    st.nq = F.get<int32_t>();
    st.sweep = F.get<int32_t>();
    st.pass = F.get<int32_t>();
    st.step = F.get<int32_t>();
    const int ndone = F.get<int32_t>();
    TNH_REQUIRE(st.N >= 2 && st.nq >= 0 && st.nq <= 4 && st.sweep >= 0 && (st.pass == 0 || st.pass == 1) &&
                    st.step >= 0 && st.step < st.N - 1 && ndone == st.sweep,
                TNH_ERR_ARG, "dmrg checkpoint: %s: bad header", path.c_str());
    st.energy = F.get<double>();
    st.resid = F.get<double>();
    st.maxerr = F.get<double>();
    st.seconds = F.get<double>();
    st.matvecs = F.get<int64_t>();
    st.done.resize(ndone);
    for (auto& d : st.done) d = F.get<tnh_sweep_stat>();
    const int N = st.N, j = st.pass == 0 ? st.step : N - 2 - st.step;
    for (int k = 0; k < N; ++k) r.A.push_back(get_tensor(F, st.nq, s));
    r.Ls.resize(N + 1);
    r.Rs.resize(N + 1);
    for (int k = 0; k <= N; ++k) {
        const int has = F.get<int32_t>();
        TNH_REQUIRE(has == (k <= j), TNH_ERR_ARG, "dmrg checkpoint: %s: environment L%d", path.c_str(), k);
        if (has) r.Ls[k] = get_tensor(F, st.nq, s);
    }
    for (int k = 0; k <= N; ++k) {
        const int has = F.get<int32_t>();
        TNH_REQUIRE(has == (k >= j + 2), TNH_ERR_ARG, "dmrg checkpoint: %s: environment R%d", path.c_str(), k);
        if (has) r.Rs[k] = get_tensor(F, st.nq, s);
    }
    return r;
}

struct Problem {
    std::vector<std::vector<Layout>> W;   // [term][site]
    std::vector<int64_t> start, done;     // [term]
    std::vector<std::vector<Layout>> P;   // [previous state][site]
    double weight = 0.0;
};

void run_dmrg(Ctx* c, int N, const Problem& pr, const tnh_tensor* mps, const tnh_sweep_params* p, double* energy,
              tnh_sweep_stat* stats, Loaded* resume = nullptr) {
    TNH_REQUIRE(N >= 2, TNH_ERR_ARG, "tnh_dmrg: N = %d < 2", N);
    TNH_REQUIRE(p->nsweep >= 1 && p->maxdim && p->cutoff, TNH_ERR_ARG, "tnh_dmrg: empty sweep schedule");
    const tnh_precision prec = (tnh_precision)p->precision;
    const tnh_precision eprec = (tnh_precision)p->env_precision;
    TNH_REQUIRE(prec == TNH_FP64 || planes_of(prec) > 0, TNH_ERR_ARG, "tnh_dmrg: bad precision");
    TNH_REQUIRE(eprec == TNH_FP64 || planes_of(eprec) > 0, TNH_ERR_ARG, "tnh_dmrg: bad env precision");
    TNH_REQUIRE(p->eigensolver == 0 || p->eigensolver == 1, TNH_ERR_ARG, "tnh_dmrg: eigensolver %d", p->eigensolver);
    TNH_REQUIRE(p->energy_mode == 0 || p->energy_mode == 1, TNH_ERR_ARG, "tnh_dmrg: energy_mode %d", p->energy_mode);
    CUDA_CHECK(cudaSetDevice(c->device));
    cudaStream_t s = c->stream;
    const int T = (int)pr.W.size();
    // the MPO: one term as given, several as their direct sum
    std::vector<Layout> W(N);
    std::vector<DevBuf> Wbuf(T > 1 ? N : 0);
    for (int j = 0; j < N; ++j) {
        for (int t = 0; t < T; ++t)
            TNH_REQUIRE(pr.W[t][j].rank() == 4, TNH_ERR_ARG, "tnh_dmrg: MPO tensors have rank 4");
        if (T == 1) {
            W[j] = pr.W[0][j];
        } else {
            std::vector<Layout> terms;
            for (int t = 0; t < T; ++t) terms.push_back(pr.W[t][j]);
            W[j] = direct_sum(terms, {0, 1}, Wbuf[j], s);
        }
    }
    std::vector<DTensor> A(N);
    for (int j = 0; j < N && !resume; ++j) {
        Layout a = parse_tensor(&mps[j], "mps");
        TNH_REQUIRE(a.rank() == 3, TNH_ERR_ARG, "tnh_dmrg: MPS tensors have rank 3");
        A[j] = new_tensor(a.inds, a.flux, s);
        for (int b = 0; b < a.nblocks(); ++b) {
            int d = A[j].L.find(a.key(b));
            TNH_REQUIRE(d >= 0, TNH_ERR_FLUX, "tnh_dmrg: MPS site %d block %d has another flux", j, b);
            CUDA_CHECK(cudaMemcpyAsync(A[j].L.data + A[j].L.off[d], a.data + a.off[b],
                                       (size_t)a.belems(b) * sizeof(double), cudaMemcpyDeviceToDevice, s));
        }
    }
    std::vector<DTensor> Ls(N + 1), Rs(N + 1);
    if (resume) {
        TNH_REQUIRE(resume->st.N == N, TNH_ERR_SHAPE, "tnh_dmrg_resume: checkpoint of %d sites, problem of %d",
                    resume->st.N, N);
        TNH_REQUIRE(resume->st.sweep < p->nsweep, TNH_ERR_ARG,
                    "tnh_dmrg_resume: checkpoint at sweep %d, schedule of %d sweeps", resume->st.sweep, p->nsweep);
        A = std::move(resume->A);
        Ls = std::move(resume->Ls);
        Rs = std::move(resume->Rs);
        for (int j = 0; j < N; ++j)
            TNH_REQUIRE(A[j].L.rank() == 3 && A[j].L.inds[1].same_space(W[j].inds[3]) &&
                            A[j].L.inds[1].arrow == W[j].inds[3].arrow,
                        TNH_ERR_SHAPE, "tnh_dmrg_resume: site %d of the checkpoint does not match the MPO", j);
        for (int k = 0; k <= N; ++k) {
            if (Ls[k].L.rank())
                TNH_REQUIRE(Ls[k].L.rank() == 3 && Ls[k].L.inds[1].same_space(k < N ? W[k].inds[0] : W[N - 1].inds[1]),
                            TNH_ERR_SHAPE, "tnh_dmrg_resume: environment L%d does not match the MPO", k);
            if (Rs[k].L.rank())
                TNH_REQUIRE(Rs[k].L.rank() == 3 && Rs[k].L.inds[1].same_space(k > 0 ? W[k - 1].inds[1] : W[0].inds[0]),
                            TNH_ERR_SHAPE, "tnh_dmrg_resume: environment R%d does not match the MPO", k);
        }
    }
    const int nq = A[0].L.nq();
    const std::vector<int> zero(nq, 0);
    if (!resume) {
        const Index& a0 = A[0].L.inds[0];
        Ls[0] = new_tensor({a0.dag(), W[0].inds[0].dag(), a0}, zero, s);
        const Index& bN = A[N - 1].L.inds[2];
        Rs[N] = new_tensor({bN.dag(), W[N - 1].inds[1].dag(), bN}, zero, s);
        int64_t o0 = 0, oN = 0;
        for (int t = 0; t < T; ++t) {
            const int64_t w0 = pr.W[t][0].inds[0].total, wN = pr.W[t][N - 1].inds[1].total;
            TNH_REQUIRE(pr.start[t] >= 0 && pr.start[t] < w0 && pr.done[t] >= 0 && pr.done[t] < wN, TNH_ERR_ARG,
                        "tnh_dmrg: term %d boundary state out of range", t);
            set_one(Ls[0], {0, o0 + pr.start[t], 0}, s);
            set_one(Rs[N], {0, oN + pr.done[t], 0}, s);
            o0 += w0;
            oN += wN;
        }
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
    if (!resume)
        for (int j = N - 1; j >= 2; --j) update_R(j);
    // where the run starts: the checkpoint's next bond, else the beginning
    const int sw0 = resume ? resume->st.sweep : 0, pass0 = resume ? resume->st.pass : 0;
    const int step0 = resume ? resume->st.step : 0;
    const int jstart = pass0 == 0 ? step0 : N - 2 - step0;

    // overlap environments of the previous states
    const int K = (int)pr.P.size();
    std::vector<std::vector<DTensor>> LO(K), RO(K);
    for (int i = 0; i < K; ++i) {
        const std::vector<Layout>& P = pr.P[i];
        for (int j = 0; j < N; ++j)
            TNH_REQUIRE(P[j].rank() == 3 && P[j].inds[1].same_space(A[j].L.inds[1]) && P[j].nq() == nq,
                        TNH_ERR_SHAPE, "tnh_dmrg: previous state %d site %d does not match the MPS", i, j);
        LO[i].resize(N + 1);
        RO[i].resize(N + 1);
        LO[i][0] = new_tensor({P[0].inds[0], A[0].L.inds[0].dag()}, zero, s);
        RO[i][N] = new_tensor({P[N - 1].inds[2], A[N - 1].L.inds[2].dag()}, zero, s);
        // both boundary links have dimension 1; a missing block means the two
        // states carry different total charge (zero overlap)
        if (LO[i][0].L.nblocks()) set_one(LO[i][0], {0, 0}, s);
        if (RO[i][N].L.nblocks()) set_one(RO[i][N], {0, 0}, s);
        for (int j = N - 1; j >= jstart + 2; --j) RO[i][j] = overlap_right(c, RO[i][j + 1].L, P[j], A[j].L);
        for (int j = 0; j < jstart; ++j) LO[i][j + 1] = overlap_left(c, LO[i][j].L, P[j], A[j].L);
    }

    double E = resume ? resume->st.energy : 0.0;
    const bool dbg = std::getenv("TNH_DEBUG") != nullptr;
    using clk = std::chrono::steady_clock;
    auto since = [](clk::time_point a) { return std::chrono::duration<double>(clk::now() - a).count(); };
    // checkpoint state: completed sweeps' statistics and the bonds done by this call
    Ckpt ck;
    ck.N = N;
    ck.nq = nq;
    if (resume) {
        ck.done = resume->st.done;
        if (stats)
            for (size_t k = 0; k < ck.done.size(); ++k) stats[k] = ck.done[k];
    }
    const std::string ckpath = c->ckpt_path;
    int64_t bonds = 0;
    c->pos_finished = false;
    for (int sw = sw0; sw < p->nsweep; ++sw) {
        auto t0 = std::chrono::steady_clock::now();
        double ph[6] = {0, 0, 0, 0, 0, 0};   // theta, plan, eigsolve, svd, factors, environment (s)
        double maxerr = 0.0, resid = 0.0, prior = 0.0;
        int64_t nmv = 0;
        if (resume && sw == sw0) {
            maxerr = resume->st.maxerr;
            resid = resume->st.resid;
            nmv = resume->st.matvecs;
            prior = resume->st.seconds;
        }
        for (int pass = (sw == sw0 ? pass0 : 0); pass < 2; ++pass) {
            for (int step = (sw == sw0 && pass == pass0 ? step0 : 0); step < N - 1; ++step) {
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
                    if (K) {
                        DevBuf phi((size_t)K * std::max<int64_t>(th.L.size, 1) * sizeof(double));
                        for (int i = 0; i < K; ++i)
                            projected_state(c, LO[i][j].L, pr.P[i][j], pr.P[i][j + 1], RO[i][j + 2].L, th.L,
                                            phi.as<double>() + (int64_t)i * th.L.size);
                        set_projectors(*P, K, phi.as<double>(), pr.weight);
                        CUDA_CHECK(cudaStreamSynchronize(s));
                    }
                    ph[1] += since(tp);
                    tp = clk::now();
                    // the FP64 product for the energy: every bond, or the sweep's last one
                    const bool fp64e = p->energy_mode == 0 || (pass == 1 && step == N - 2);
                    EigResult r = p->eigensolver == 1
                                      ? davidson(*P, th.L.data, p->krylov_dim, p->lanczos_tol, fp64e)
                                      : eigsolve(*P, th.L.data, p->krylov_dim, p->lanczos_tol, fp64e);
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
                    if (dbg) {
                        int kept = 0;
                        for (int d : sh.dims) kept += d;
                        std::fprintf(stderr, "dmrg: sweep %d bond %d dir %+d E %.14f kept %d in %zu sectors truncerr %.3e "
                                     "(so far: theta %.3f plan %.3f eig %.3f svd %.3f s)\n",
                                     sw, j, dir, E, kept, sh.dims.size(), sh.truncerr, ph[0], ph[1], ph[2], ph[3]);
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
                if (dir > 0) {
                    update_L(j);
                    for (int i = 0; i < K; ++i) LO[i][j + 1] = overlap_left(c, LO[i][j].L, pr.P[i][j], A[j].L);
                } else {
                    update_R(j + 1);
                    for (int i = 0; i < K; ++i)
                        RO[i][j + 1] = overlap_right(c, RO[i][j + 2].L, pr.P[i][j + 1], A[j + 1].L);
                }
                ph[5] += since(tp);
                // checkpoint inside the sweep (the end of a sweep writes below)
                ++bonds;
                const bool last = pass == 1 && step == N - 2;
                const bool stop = c->ckpt_stop > 0 && bonds >= c->ckpt_stop;
                if (!last && (stop || (!ckpath.empty() && c->ckpt_every > 0 && bonds % c->ckpt_every == 0))) {
                    CUDA_CHECK(cudaStreamSynchronize(s));
                    check_device_flag(c);
                    ck.sweep = sw;
                    ck.pass = step + 1 < N - 1 ? pass : pass + 1;
                    ck.step = step + 1 < N - 1 ? step + 1 : 0;
                    ck.energy = E;
                    ck.resid = resid;
                    ck.maxerr = maxerr;
                    ck.matvecs = nmv;
                    ck.seconds = prior + std::chrono::duration<double>(clk::now() - t0).count();
                    if (!ckpath.empty()) write_checkpoint(ckpath, ck, A, Ls, Rs, s);
                    if (stop) {
                        c->pos_sweep = ck.sweep;
                        c->pos_pass = ck.pass;
                        c->pos_step = ck.step;
                        *energy = E;
                        c->mps = std::move(A);
                        return;
                    }
                }
            }
        }
        CUDA_CHECK(cudaStreamSynchronize(s));
        check_device_flag(c);
        double secs = prior + std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (dbg)
            std::fprintf(stderr,
                         "dmrg: sweep %d %.3f s: theta %.3f, H_eff plan %.3f, eigensolver %.3f, SVD %.3f, "
                         "factors %.3f, environment %.3f\n",
                         sw, secs, ph[0], ph[1], ph[2], ph[3], ph[4], ph[5]);
        tnh_sweep_stat st{};
        st.sweep = sw;
        st.energy = E;
        st.resid = resid;
        st.truncerr = maxerr;
        int ml = 0;
        for (int j = 0; j < N; ++j) ml = std::max<int>(ml, (int)A[j].L.inds[2].total);
        st.maxlink = ml;
        st.matvecs = nmv;
        st.seconds = secs;
        if (stats) stats[sw] = st;
        ck.done.push_back(st);
        const bool stop = c->ckpt_stop > 0 && bonds >= c->ckpt_stop;
        if (sw + 1 < p->nsweep && (!ckpath.empty() || stop)) {
            ck.sweep = sw + 1;
            ck.pass = ck.step = 0;
            ck.energy = E;
            ck.resid = ck.maxerr = ck.seconds = 0.0;
            ck.matvecs = 0;
            if (!ckpath.empty()) write_checkpoint(ckpath, ck, A, Ls, Rs, s);
            if (stop) {
                c->pos_sweep = ck.sweep;
                c->pos_pass = c->pos_step = 0;
                *energy = E;
                c->mps = std::move(A);
                return;
            }
        }
    }
    if (eprec != TNH_FP64) {
        // the final state's energy with FP64 environments: R_N-1 .. R_2 again
        // from the final MPS, then <theta|H_eff theta> / <theta|theta> at bond
        // (0, 1) in FP64 (theta = A_0 A_1, sites 2.. right-orthogonal)
        for (int j = N - 1; j >= 2; --j) {
            const Layout& a = A[j].L;
            Rs[j] = new_tensor({a.inds[0], W[j].inds[0], a.inds[0].dag()}, zero, s);
            auto P = make_env(c, -1, Rs[j + 1].L, a, W[j], Rs[j].L);
            run_env(c, *P, Rs[j + 1].L.data, a.data, W[j].data, Rs[j].L.data, TNH_FP64);
            CUDA_CHECK(cudaStreamSynchronize(s));
        }
        Layout a1 = relabel(A[0].L, {1, 2, 3});
        Layout a2 = relabel(A[1].L, {3, 4, 5});
        DTensor th = new_tensor({a1.inds[0], a1.inds[1], a2.inds[1], a2.inds[2]}, fsum(a1.flux, a2.flux), s);
        th.L = relabel(th.L, {1, 2, 4, 5});
        contract64(c, a1, a2, th.L);
        auto P = make_heff(c, Ls[0].L, W[0], W[1], Rs[2].L, th.L, TNH_FP64);
        if (K) {
            DevBuf phi((size_t)K * std::max<int64_t>(th.L.size, 1) * sizeof(double));
            for (int i = 0; i < K; ++i)
                projected_state(c, LO[i][0].L, pr.P[i][0], pr.P[i][1], RO[i][2].L, th.L,
                                phi.as<double>() + (int64_t)i * th.L.size);
            set_projectors(*P, K, phi.as<double>(), pr.weight);
        }
        const double ef = rayleigh_fp64(*P, th.L.data);
        E = ef;
        if (stats && p->nsweep > 0) stats[p->nsweep - 1].energy = ef;
    }
    c->pos_sweep = p->nsweep;
    c->pos_pass = c->pos_step = 0;
    c->pos_finished = true;
    *energy = E;
    c->mps = std::move(A);
}

}  // namespace

}  // namespace tnh

using namespace tnh;

extern "C" {

tnh_status tnh_dmrg(tnh_ctx* ctx, int32_t N, const tnh_tensor* mpo, int64_t start, int64_t done,
                    const tnh_tensor* mps, const tnh_sweep_params* p, double* energy, tnh_sweep_stat* stats) {
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    return guard(c, [&] {
        TNH_REQUIRE(c && mpo && mps && p && energy, TNH_ERR_ARG, "tnh_dmrg: NULL argument");
        TNH_REQUIRE(N >= 2, TNH_ERR_ARG, "tnh_dmrg: N = %d < 2", N);
        Problem pr;
        pr.W.resize(1);
        for (int j = 0; j < N; ++j) pr.W[0].push_back(parse_tensor(&mpo[j], "mpo"));
        pr.start = {start};
        pr.done = {done};
        run_dmrg(c, N, pr, mps, p, energy, stats);
    });
}

tnh_status tnh_dmrg_ex(tnh_ctx* ctx, int32_t N, const tnh_dmrg_problem* prob, const tnh_tensor* mps,
                       const tnh_sweep_params* p, double* energy, tnh_sweep_stat* stats) {
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    return guard(c, [&] {
        TNH_REQUIRE(c && prob && mps && p && energy, TNH_ERR_ARG, "tnh_dmrg_ex: NULL argument");
        TNH_REQUIRE(N >= 2, TNH_ERR_ARG, "tnh_dmrg_ex: N = %d < 2", N);
        TNH_REQUIRE(prob->nterm >= 1 && prob->mpo && prob->start && prob->done, TNH_ERR_ARG,
                    "tnh_dmrg_ex: need at least one MPO with its boundary states");
        TNH_REQUIRE(prob->northo >= 0 && (prob->northo == 0 || prob->ortho), TNH_ERR_ARG,
                    "tnh_dmrg_ex: previous states missing");
        Problem pr;
        pr.W.resize(prob->nterm);
        for (int t = 0; t < prob->nterm; ++t) {
            for (int j = 0; j < N; ++j) pr.W[t].push_back(parse_tensor(&prob->mpo[(size_t)t * N + j], "mpo"));
            pr.start.push_back(prob->start[t]);
            pr.done.push_back(prob->done[t]);
        }
        pr.P.resize(prob->northo);
        for (int i = 0; i < prob->northo; ++i)
            for (int j = 0; j < N; ++j) pr.P[i].push_back(parse_tensor(&prob->ortho[(size_t)i * N + j], "ortho"));
        pr.weight = prob->weight;
        run_dmrg(c, N, pr, mps, p, energy, stats);
    });
}

tnh_status tnh_dmrg_checkpoint(tnh_ctx* ctx, const char* path, int32_t every, int64_t stop_after) {
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    return guard(c, [&] {
        TNH_REQUIRE(c, TNH_ERR_ARG, "tnh_dmrg_checkpoint: ctx is NULL");
        TNH_REQUIRE(every >= 0 && stop_after >= 0, TNH_ERR_ARG, "tnh_dmrg_checkpoint: every %d, stop_after %lld",
                    every, (long long)stop_after);
        c->ckpt_path = path ? path : "";
        c->ckpt_every = every;
        c->ckpt_stop = stop_after;
    });
}

tnh_status tnh_dmrg_resume(tnh_ctx* ctx, int32_t N, const tnh_dmrg_problem* prob, const char* path,
                           const tnh_sweep_params* p, double* energy, tnh_sweep_stat* stats) {
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    return guard(c, [&] {
        TNH_REQUIRE(c && prob && path && p && energy, TNH_ERR_ARG, "tnh_dmrg_resume: NULL argument");
        TNH_REQUIRE(N >= 2, TNH_ERR_ARG, "tnh_dmrg_resume: N = %d < 2", N);
        TNH_REQUIRE(prob->nterm >= 1 && prob->mpo && prob->start && prob->done, TNH_ERR_ARG,
                    "tnh_dmrg_resume: need at least one MPO with its boundary states");
        TNH_REQUIRE(prob->northo >= 0 && (prob->northo == 0 || prob->ortho), TNH_ERR_ARG,
                    "tnh_dmrg_resume: previous states missing");
        CUDA_CHECK(cudaSetDevice(c->device));
        Problem pr;
        pr.W.resize(prob->nterm);
        for (int t = 0; t < prob->nterm; ++t) {
            for (int j = 0; j < N; ++j) pr.W[t].push_back(parse_tensor(&prob->mpo[(size_t)t * N + j], "mpo"));
            pr.start.push_back(prob->start[t]);
            pr.done.push_back(prob->done[t]);
        }
        pr.P.resize(prob->northo);
        for (int i = 0; i < prob->northo; ++i)
            for (int j = 0; j < N; ++j) pr.P[i].push_back(parse_tensor(&prob->ortho[(size_t)i * N + j], "ortho"));
        pr.weight = prob->weight;
        Loaded ld = read_checkpoint(path, c->stream);
        run_dmrg(c, N, pr, nullptr, p, energy, stats, &ld);
    });
}

tnh_status tnh_dmrg_position(tnh_ctx* ctx, int32_t* sweep, int32_t* pass, int32_t* step, int32_t* finished) {
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    return guard(c, [&] {
        TNH_REQUIRE(c && sweep && pass && step && finished, TNH_ERR_ARG, "tnh_dmrg_position: NULL argument");
        *sweep = c->pos_sweep;
        *pass = c->pos_pass;
        *step = c->pos_step;
        *finished = c->pos_finished ? 1 : 0;
    });
}

tnh_status tnh_dmrg_mps_size(tnh_ctx* ctx, int32_t* N) {
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    return guard(c, [&] {
        TNH_REQUIRE(c && N, TNH_ERR_ARG, "tnh_dmrg_mps_size: NULL argument");
        *N = (int32_t)c->mps.size();
    });
}

tnh_status tnh_dmrg_mps_link(tnh_ctx* ctx, int32_t j, int32_t* nsect, int32_t* nq, int32_t* qn, int32_t* sect_dim) {
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    return guard(c, [&] {
        TNH_REQUIRE(c && nsect, TNH_ERR_ARG, "tnh_dmrg_mps_link: NULL argument");
        const int N = (int)c->mps.size();
        TNH_REQUIRE(N > 0, TNH_ERR_ARG, "tnh_dmrg_mps_link: no DMRG run on this context");
        TNH_REQUIRE(j >= 0 && j <= N, TNH_ERR_ARG, "tnh_dmrg_mps_link: link %d out of 0..%d", j, N);
        const Index& ix = j < N ? c->mps[j].L.inds[0] : c->mps[N - 1].L.inds[2];
        *nsect = ix.nsect;
        if (nq) *nq = ix.nq;
        if (qn) std::copy(ix.qn.begin(), ix.qn.end(), qn);
        if (sect_dim) std::copy(ix.dim.begin(), ix.dim.end(), sect_dim);
    });
}

tnh_status tnh_dmrg_mps_get(tnh_ctx* ctx, int32_t j, tnh_tensor* A) {
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    return guard(c, [&] {
        TNH_REQUIRE(c && A, TNH_ERR_ARG, "tnh_dmrg_mps_get: NULL argument");
        const int N = (int)c->mps.size();
        TNH_REQUIRE(j >= 0 && j < N, TNH_ERR_ARG, "tnh_dmrg_mps_get: site %d out of 0..%d", j, N - 1);
        CUDA_CHECK(cudaSetDevice(c->device));
        const Layout& src = c->mps[j].L;
        Layout dst = parse_tensor(A, "A");
        TNH_REQUIRE(dst.rank() == 3, TNH_ERR_SHAPE, "tnh_dmrg_mps_get: A must have rank 3");
        for (int i = 0; i < 3; ++i)
            TNH_REQUIRE(dst.inds[i].same_space(src.inds[i]) && dst.inds[i].arrow == src.inds[i].arrow, TNH_ERR_SHAPE,
                        "tnh_dmrg_mps_get: index %d of A differs from the stored site %d", i, j);
        cudaStream_t s = c->stream;
        for (int b = 0; b < src.nblocks(); ++b)
            TNH_REQUIRE(dst.find(src.key(b)) >= 0, TNH_ERR_SHAPE, "tnh_dmrg_mps_get: A lacks stored block %d", b);
        for (int b = 0; b < dst.nblocks(); ++b) {
            const int d = src.find(dst.key(b));
            const size_t bytes = (size_t)dst.belems(b) * sizeof(double);
            if (d >= 0)
                CUDA_CHECK(cudaMemcpyAsync(dst.data + dst.off[b], src.data + src.off[d], bytes,
                                           cudaMemcpyDeviceToDevice, s));
            else
                CUDA_CHECK(cudaMemsetAsync(dst.data + dst.off[b], 0, bytes, s));
        }
        CUDA_CHECK(cudaStreamSynchronize(s));
    });
}

}  // extern "C"
