// Device Lanczos eigensolver for the lowest eigenpair of H_eff.
//
// The paper (Sec. 7.2, Sec. 12.2) only says that DMRG finds the dominant
// eigenvector of H_eff with a few Krylov steps per bond. This is the
// textbook Lanczos iteration with full reorthogonalisation:
//   q_0 = psi / |psi|;  w = H q_j;  alpha_j = q_j . w;
//   w -= alpha_j q_j + beta_{j-1} q_{j-1};
//   twice: h = Q^T w, w -= Q h      (classical Gram-Schmidt, applied twice)
//   beta_j = |w|;  q_{j+1} = w / beta_j.
// After every step the lowest eigenvalue of the tridiagonal matrix T_j is
// found by multisection on its Sturm sequence (division-free minors) and its
// eigenvector by one twisted factorization of T_j - theta, refined by the
// Rayleigh quotient; the Ritz residual estimate is beta_j |s_j|. Every
// vector operation is float64 with a fixed-order (deterministic) reduction.
#include <cmath>

#include "heff.h"
#include "prof.h"
#include "tnh_guard.h"

namespace tnh {

namespace {

constexpr int kRedThreads = 256;

// partial[j * G + block] = sum over this block's elements of Q_j . w
__global__ void multidot_partial(const double* __restrict__ Q, int64_t ldq, const double* __restrict__ w,
                                 int64_t n, double* __restrict__ partial) {
    __shared__ double red[kRedThreads];
    const int j = blockIdx.y;
    const double* q = Q + (int64_t)j * ldq;
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        s = fma(q[i], w[i], s);
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = kRedThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[(int64_t)j * gridDim.x + blockIdx.x] = red[0];
}

// out[j] = sum_b partial[j * G + b], fixed order
__global__ void reduce_partials(const double* __restrict__ partial, int G, double* __restrict__ out) {
    __shared__ double red[kRedThreads];
    const int j = blockIdx.x;
    double s = 0.0;
    for (int b = threadIdx.x; b < G; b += blockDim.x) s += partial[(int64_t)j * G + b];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = kRedThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[j] = red[0];
}

// w -= alpha q_j + beta q_{j-1}   (qm may be null)
__global__ void lanczos_three_term(double* __restrict__ w, const double* __restrict__ qj,
                                   const double* __restrict__ qm, const double* __restrict__ alpha,
                                   const double* __restrict__ beta, int64_t n) {
    const double a = *alpha, b = qm ? *beta : 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double v = w[i] - a * qj[i];
        if (qm) v -= b * qm[i];
        w[i] = v;
    }
}

// w += sign * sum_j c_j Q_j   (k vectors); if overwrite, w = sum_j c_j Q_j
__global__ void multi_axpy(double* __restrict__ w, const double* __restrict__ Q, int64_t ldq, int k,
                           const double* __restrict__ c, double sign, int overwrite, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int j = 0; j < k; ++j) s = fma(c[j], Q[(int64_t)j * ldq + i], s);
        w[i] = overwrite ? s : w[i] + sign * s;
    }
}

// y = x * num / sqrt(den) (mode 0), y = x / sqrt(den) (mode 1), y = x / den (mode 2)
__global__ void scale_copy(const double* __restrict__ x, double* __restrict__ y, int64_t n,
                           const double* __restrict__ num, const double* __restrict__ den, int mode) {
    double f;
    if (mode == 0) f = *num / sqrt(*den);
    else if (mode == 1) f = 1.0 / sqrt(*den);
    else f = 1.0 / *den;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = x[i] * f;
}

// y -= e * x
__global__ void axpy_dev(double* __restrict__ y, const double* __restrict__ x, const double* __restrict__ e,
                         int64_t n) {
    const double a = *e;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] -= a * x[i];
}

// Number of eigenvalues of the symmetric tridiagonal (a, b) below x: the
// number of negative pivots d_i = p_{i+1} / p_i of T - x = L D L^T
// (Sylvester's inertia), read off the signs of the leading minors
//   p_0 = 1, p_1 = a_0 - x, p_{i+1} = (a_i - x) p_i - b_{i-1}^2 p_{i-1}
// without a division (float64 division is slow on this GPU). An exactly
// zero pivot is taken as a tiny positive one (p_{i+1} = 2^-200 p_i), and the
// pair (p_{i-1}, p_i) is rescaled by an exact power of two when it leaves
// [2^-500, 2^500].
__device__ int sturm_count(const double* a, const double* b2, int k, double x) {
    int c = 0;
    double pm = 1.0, p = a[0] - x;
    if (p == 0.0) p = 0x1p-200;
    if (p < 0.0) ++c;
    for (int i = 1; i < k; ++i) {
        double pn = (a[i] - x) * p - b2[i - 1] * pm;
        if (pn == 0.0) pn = p * 0x1p-200;
        if ((pn < 0.0) != (p < 0.0)) ++c;
        pm = p;
        p = pn;
        const double ap = fabs(p);
        if (ap > 0x1p500) { p *= 0x1p-500; pm *= 0x1p-500; }
        else if (ap < 0x1p-500 && fabs(pm) < 0x1p-500) { p *= 0x1p500; pm *= 0x1p500; }
    }
    return c;
}

constexpr int kMaxKrylov = 256;

// Lowest eigenpair of T_k (alpha[0..k), beta[0..k-1)); beta2_last = |w|^2 of
// the current step. out[0] = theta, out[1] = beta_k |s_k|, out[2] = beta_k,
// beta[k-1] = beta_k is written, s[0..k) = normalised eigenvector.
__global__ void tridiag_lowest(const double* __restrict__ alpha, double* __restrict__ beta, int k,
                               const double* __restrict__ beta2_last, double* __restrict__ out,
                               double* __restrict__ s) {
    __shared__ double a[kMaxKrylov], b[kMaxKrylov], b2[kMaxKrylov];
    __shared__ double lo_s, hi_s, tiny_s;
    __shared__ int first_s;
    __shared__ double dd[kMaxKrylov], dl[kMaxKrylov], v[kMaxKrylov];
    const int t = threadIdx.x, nt = blockDim.x;
    for (int i = t; i < k; i += nt) a[i] = alpha[i];
    for (int i = t; i + 1 < k; i += nt) { b[i] = beta[i]; b2[i] = beta[i] * beta[i]; }
    __syncthreads();
    if (t == 0) {
        double lo = a[0], hi = a[0];
        for (int i = 0; i < k; ++i) {
            double r = (i > 0 ? fabs(b[i - 1]) : 0.0) + (i + 1 < k ? fabs(b[i]) : 0.0);
            lo = fmin(lo, a[i] - r);
            hi = fmax(hi, a[i] + r);
        }
        double pad = 1e-12 * fmax(1.0, fmax(fabs(lo), fabs(hi)));
        lo_s = lo - pad;
        hi_s = hi + pad;
    }
    __syncthreads();
    // multisection: 32 probes per round, by the first warp only (float64
    // throughput of one SM bounds many probes; 5 bits per round suffice)
    if (t < 32) {
        double lo = lo_s, hi = hi_s;
        for (int round = 0; round < 24; ++round) {
            if (hi - lo <= 2e-16 * fmax(fabs(lo), fabs(hi))) break;
            const double x = lo + (hi - lo) * (double)(t + 1) / 33.0;
            const unsigned below = __ballot_sync(0xffffffffu, sturm_count(a, b2, k, x) >= 1);
            const int f = below ? __ffs(below) - 1 : 32;   // first probe with an eigenvalue below it
            const double nlo = f == 0 ? lo : lo + (hi - lo) * (double)f / 33.0;
            const double nhi = f == 32 ? hi : lo + (hi - lo) * (double)(f + 1) / 33.0;
            lo = nlo;
            hi = nhi;
        }
        if (t == 0) {
            lo_s = lo;
            hi_s = hi;
        }
    }
    __syncthreads();
    if (k == 1) {   // uniform branch: the other one has barriers
        if (t == 0) {
            double bk = sqrt(fmax(*beta2_last, 0.0));
            beta[0] = bk;
            out[0] = a[0];
            out[1] = bk;
            out[2] = bk;
            s[0] = 1.0;
        }
    } else {
        // eigenvector for theta by one twisted factorization of T - theta:
        // D+ from the top (thread 0) and D- from the bottom (thread 1) run
        // concurrently; the twist r minimises |gamma_r|, v_r = 1, and v is
        // recurred outwards (threads 0 and 1 again)
        const double theta = 0.5 * (lo_s + hi_s);
        if (t == 0) {
            double tn = 1e-300;
            for (int i = 0; i < k; ++i)
                tn = fmax(tn, fabs(a[i]) + (i + 1 < k ? fabs(b[i]) : 0.0) + (i > 0 ? fabs(b[i - 1]) : 0.0));
            tiny_s = fmax(1e-15 * tn, 1e-200);
        }
        __syncthreads();
        const double tiny = tiny_s;
        if (t == 0) {
            double d = a[0] - theta;
            for (int i = 0; i < k; ++i) {
                if (i > 0) d = (a[i] - theta) - b2[i - 1] / d;
                if (fabs(d) < tiny) d = d < 0.0 ? -tiny : tiny;
                dd[i] = d;   // D+
            }
        } else if (t == 1) {
            double d = a[k - 1] - theta;
            for (int i = k - 1; i >= 0; --i) {
                if (i < k - 1) d = (a[i] - theta) - b2[i] / d;
                if (fabs(d) < tiny) d = d < 0.0 ? -tiny : tiny;
                dl[i] = d;   // D-
            }
        }
        __syncthreads();
        if (t == 0) {
            int r = 0;
            double gbest = INFINITY;
            for (int i = 0; i < k; ++i) {
                const double g = fabs(dd[i] + dl[i] - (a[i] - theta));
                if (g < gbest) { gbest = g; r = i; }
            }
            first_s = r;
        }
        __syncthreads();
        const int r = first_s;
        if (t == 0) {   // v_r = 1 and the part above the twist
            double vi = 1.0;
            v[r] = 1.0;
            for (int i = r - 1; i >= 0; --i) {
                vi = -(b[i] / dd[i]) * vi;
                v[i] = vi;
            }
        } else if (t == 1) {   // the part below the twist (starts from v_r = 1 itself)
            double vi = 1.0;
            for (int i = r + 1; i < k; ++i) {
                vi = -(b[i - 1] / dl[i]) * vi;
                v[i] = vi;
            }
        }
        __syncthreads();
        if (t == 0) {
            double nrm = 0.0;
            for (int i = 0; i < k; ++i) nrm = fma(v[i], v[i], nrm);
            const double inv = 1.0 / sqrt(nrm);
            for (int i = 0; i < k; ++i) v[i] *= inv;
            // Rayleigh quotient refines theta to machine precision
            double rq = 0.0;
            for (int i = 0; i < k; ++i) {
                double tv = a[i] * v[i];
                if (i > 0) tv += b[i - 1] * v[i - 1];
                if (i + 1 < k) tv += b[i] * v[i + 1];
                rq += v[i] * tv;
            }
            double bk = sqrt(fmax(*beta2_last, 0.0));
            beta[k - 1] = bk;
            out[0] = rq;
            out[1] = bk * fabs(v[k - 1]);
            out[2] = bk;
            for (int i = 0; i < k; ++i) s[i] = v[i];
        }
    }
}

// Fixed-length runs (tol <= 0) need the tridiagonal eigenpair only at the
// end: intermediate steps only record beta_j = |w| (and alpha_j as a scale
// for the breakdown test).
__global__ void set_beta(const double* __restrict__ alpha_j, const double* __restrict__ beta2_last,
                         double* __restrict__ beta_j, double* __restrict__ out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        const double bk = sqrt(fmax(*beta2_last, 0.0));
        *beta_j = bk;
        out[0] = *alpha_j;
        out[1] = bk;
        out[2] = bk;
    }
}

int grid_for(int64_t n, int nsms) {
    int64_t g = (n + 255) / 256;
    int64_t cap = (int64_t)nsms * 8;
    return (int)std::max<int64_t>(1, std::min(g, cap));
}

}  // namespace

void VecWork::ensure(int nsms) {
    if (blocks) return;
    blocks = std::max(1, nsms * 2);
    partial.alloc((size_t)blocks * kMaxKrylov * sizeof(double));
    scal.alloc(64 * sizeof(double));
}

void vdot(Ctx* ctx, VecWork& w, const double* x, const double* y, int64_t n, double* d_out) {
    w.ensure(ctx->num_sms);
    { KScope ks_("multidot_partial", ctx->stream);
    multidot_partial<<<dim3(w.blocks, 1), kRedThreads, 0, ctx->stream>>>(x, 0, y, n, w.partial.as<double>());
    }
    { KScope ks_("reduce_partials", ctx->stream);
    reduce_partials<<<1, kRedThreads, 0, ctx->stream>>>(w.partial.as<double>(), w.blocks, d_out);
    }
}

void vscale_copy(Ctx* ctx, const double* x, double* y, int64_t n, const double* d_num, const double* d_den,
                 int mode) {
    { KScope ks_("scale_copy", ctx->stream);
    scale_copy<<<grid_for(n, ctx->num_sms), 256, 0, ctx->stream>>>(x, y, n, d_num, d_den, mode);
    }
}

void set_projectors(HeffPlan& P, int k, const double* phi, double weight) {
    TNH_REQUIRE(k >= 0 && k <= kMaxKrylov, TNH_ERR_ARG, "projectors: %d vectors, at most %d", k, kMaxKrylov);
    TNH_REQUIRE(k == 0 || phi, TNH_ERR_ARG, "projectors: vectors are NULL");
    TNH_REQUIRE(std::isfinite(weight), TNH_ERR_ARG, "projectors: weight %g", weight);
    P.nproj = 0;
    P.pweight = weight;
    if (k == 0 || P.n == 0) return;
    const size_t bytes = (size_t)k * P.n * sizeof(double);
    if (P.proj.bytes < bytes) P.proj.alloc(bytes);
    if (P.pcoef.bytes < (size_t)k * sizeof(double)) P.pcoef.alloc((size_t)k * sizeof(double));
    CUDA_CHECK(cudaMemcpyAsync(P.proj.p, phi, bytes, cudaMemcpyDeviceToDevice, P.stream));
    P.pvw.ensure(P.ctx->num_sms);
    P.nproj = k;
}

void add_projectors(HeffPlan& P, const double* x, double* y) {
    if (P.nproj == 0 || P.n == 0) return;
    cudaStream_t s = P.stream;
    const int64_t n = P.n;
    const double* phi = P.proj.as<double>();
    { KScope ks_("multidot_partial", s);
    multidot_partial<<<dim3(P.pvw.blocks, P.nproj), kRedThreads, 0, s>>>(phi, n, x, n, P.pvw.partial.as<double>());
    }
    { KScope ks_("reduce_partials", s);
    reduce_partials<<<P.nproj, kRedThreads, 0, s>>>(P.pvw.partial.as<double>(), P.pvw.blocks, P.pcoef.as<double>());
    }
    { KScope ks_("multi_axpy", s);
    multi_axpy<<<grid_for(n, P.ctx->num_sms), 256, 0, s>>>(y, phi, n, P.nproj, P.pcoef.as<double>(), P.pweight, 0, n);
    }
}

EigResult eigsolve(HeffPlan& P, double* psi, int kmax, double tol) {
    Ctx* ctx = P.ctx;
    cudaStream_t s = ctx->stream;
    const int64_t n = P.n;
    TNH_REQUIRE(kmax >= 1 && kmax < kMaxKrylov, TNH_ERR_ARG, "eigsolve: krylov_dim %d out of 1..%d", kmax,
                kMaxKrylov - 1);
    EigResult res;
    if (n == 0) return res;
    VecWork vw;
    vw.ensure(ctx->num_sms);
    DevBuf Q((size_t)(kmax + 1) * n * sizeof(double));
    DevBuf wv((size_t)n * sizeof(double)), yv((size_t)n * sizeof(double));
    // scalars: alpha[kmax] beta[kmax] h[kmax+1] s[kmax] out[4] misc[8]
    DevBuf sc((size_t)(4 * kmax + 16) * sizeof(double));
    double* alpha = sc.as<double>();
    double* beta = alpha + kmax;
    double* h = beta + kmax;
    double* sv = h + kmax + 1;
    double* out = sv + kmax;
    double* misc = out + 4;
    double* q = Q.as<double>();
    double* w = wv.as<double>();
    const int g = grid_for(n, ctx->num_sms);
    // q0 = psi / |psi|
    vdot(ctx, vw, psi, psi, n, misc);
    double hn2 = 0;
    CUDA_CHECK(cudaMemcpyAsync(&hn2, misc, sizeof(double), cudaMemcpyDeviceToHost, s));
    CUDA_CHECK(cudaStreamSynchronize(s));
    TNH_REQUIRE(std::isfinite(hn2) && hn2 > 0.0, TNH_ERR_NUMERIC, "eigsolve: start vector has norm^2 %g", hn2);
    { KScope ks_("scale_copy", s);
    scale_copy<<<g, 256, 0, s>>>(psi, q, n, nullptr, misc, 1);
    }
    int k = 0;
    double host[3] = {0, 0, 0};
    for (int j = 0; j < kmax; ++j) {
        double* qj = q + (int64_t)j * n;
        heff_apply(P, P.prec, qj, w);
        vdot(ctx, vw, qj, w, n, alpha + j);
        { KScope ks_("lanczos_three_term", s);
        lanczos_three_term<<<g, 256, 0, s>>>(w, qj, j > 0 ? qj - n : nullptr, alpha + j,
                                            j > 0 ? beta + (j - 1) : alpha, n);
        }
        for (int rep = 0; rep < 2; ++rep) {
            { KScope ks_("multidot_partial", s);
            multidot_partial<<<dim3(vw.blocks, j + 1), kRedThreads, 0, s>>>(q, n, w, n, vw.partial.as<double>());
            }
            { KScope ks_("reduce_partials", s);
            reduce_partials<<<j + 1, kRedThreads, 0, s>>>(vw.partial.as<double>(), vw.blocks, h);
            }
            { KScope ks_("multi_axpy", s);
            multi_axpy<<<g, 256, 0, s>>>(w, q, n, j + 1, h, -1.0, 0, n);
            }
        }
        vdot(ctx, vw, w, w, n, misc + 1);
        if (tol > 0.0 || j + 1 == kmax) {
            KScope ks_("tridiag_lowest", s);
            tridiag_lowest<<<1, 256, 0, s>>>(alpha, beta, j + 1, misc + 1, out, sv);
        } else {
            KScope ks_("set_beta", s);
            set_beta<<<1, 32, 0, s>>>(alpha + j, misc + 1, beta + j, out);
        }
        CUDA_CHECK(cudaMemcpyAsync(host, out, 3 * sizeof(double), cudaMemcpyDeviceToHost, s));
        CUDA_CHECK(cudaStreamSynchronize(s));
        k = j + 1;
        TNH_REQUIRE(std::isfinite(host[0]) && std::isfinite(host[1]), TNH_ERR_NUMERIC,
                    "eigsolve: non-finite Ritz value at step %d", j);
        const double scale = std::max(1.0, std::fabs(host[0]));
        if (host[2] <= 1e-14 * scale || j + 1 == kmax) {
            if (!(tol > 0.0 || j + 1 == kmax)) {   // breakdown in a fixed-length run: T_k was not solved yet
                KScope ks_("tridiag_lowest", s);
                tridiag_lowest<<<1, 256, 0, s>>>(alpha, beta, j + 1, misc + 1, out, sv);
            }
            break;
        }
        if (tol > 0.0 && host[1] <= tol * scale) break;
        { KScope ks_("scale_copy", s);
        scale_copy<<<g, 256, 0, s>>>(w, q + (int64_t)(j + 1) * n, n, nullptr, beta + j, 2);
        }
    }
    // Ritz vector, normalised, into psi
    { KScope ks_("multi_axpy", s);
    multi_axpy<<<g, 256, 0, s>>>(psi, q, n, k, sv, 1.0, 1, n);
    }
    vdot(ctx, vw, psi, psi, n, misc);
    { KScope ks_("scale_copy", s);
    scale_copy<<<g, 256, 0, s>>>(psi, psi, n, nullptr, misc, 1);
    }
    // float64 energy and residual
    heff_apply(P, TNH_FP64, psi, yv.as<double>());
    vdot(ctx, vw, psi, yv.as<double>(), n, misc + 2);
    { KScope ks_("axpy_dev", s);
    axpy_dev<<<g, 256, 0, s>>>(yv.as<double>(), psi, misc + 2, n);
    }
    vdot(ctx, vw, yv.as<double>(), yv.as<double>(), n, misc + 3);
    double fin[2];
    CUDA_CHECK(cudaMemcpyAsync(fin, misc + 2, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    CUDA_CHECK(cudaStreamSynchronize(s));
    check_device_flag(ctx);
    res.energy = fin[0];
    res.resid = std::sqrt(std::max(fin[1], 0.0));
    res.matvecs = k;
    return res;
}

}  // namespace tnh

using namespace tnh;

extern "C" tnh_status tnh_eigsolve(tnh_heff* plan, double* psi, int32_t krylov_dim, double tol, double* energy,
                                   double* resid, int32_t* matvecs) {
    auto* P = reinterpret_cast<HeffPlan*>(plan);
    return guard(P ? P->ctx : nullptr, [&] {
        TNH_REQUIRE(P && psi, TNH_ERR_ARG, "tnh_eigsolve: NULL argument");
        EigResult r = eigsolve(*P, psi, krylov_dim, tol);
        if (energy) *energy = r.energy;
        if (resid) *resid = r.resid;
        if (matvecs) *matvecs = r.matvecs;
    });
}
