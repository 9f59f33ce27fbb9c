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

// The same count in float32 (the float64 units of this GPU run at 1/64 of
// the float32 rate), rescaling at 2^+-60: exact up to float32 rounding of
// the minors, i.e. it may miscount only for x within float32 resolution of
// an eigenvalue.
__device__ int sturm_count_f32(const float* a, const float* b2, int k, float x) {
    int c = 0;
    float pm = 1.0f, p = a[0] - x;
    if (p == 0.0f) p = 0x1p-100f;
    if (p < 0.0f) ++c;
    for (int i = 1; i < k; ++i) {
        float pn = fmaf(a[i] - x, p, -b2[i - 1] * pm);
        if (pn == 0.0f) pn = p * 0x1p-100f;
        if ((pn < 0.0f) != (p < 0.0f)) ++c;
        pm = p;
        p = pn;
        const float ap = fabsf(p);
        if (ap > 0x1p60f) { p *= 0x1p-60f; pm *= 0x1p-60f; }
        else if (ap < 0x1p-60f && fabsf(pm) < 0x1p-60f) { p *= 0x1p60f; pm *= 0x1p60f; }
    }
    return c;
}

// Eigenvector for theta by one twisted factorization of T - theta (the
// twist r minimises |gamma_r|, v_r = 1, v recurred outwards), normalised;
// returns the Rayleigh quotient v^T T v. T = (a, b), b2 = b^2, in type R for
// the factorization; v and the quotient in float64. Called by the whole
// block (uniform); threads 0 and 32 run the two directions concurrently.
template <class R>
__device__ double twisted_rq(const double* a, const double* b, const double* b2, int k, double theta, double tiny,
                             R* dd, R* dl, double* v, int* twist) {
    const int t = threadIdx.x;
    if (t == 0) {
        R d = (R)(a[0] - theta);
        for (int i = 0; i < k; ++i) {
            if (i > 0) d = (R)(a[i] - theta) - (R)b2[i - 1] / d;
            if (fabs((double)d) < tiny) d = d < (R)0 ? (R)-tiny : (R)tiny;
            dd[i] = d;   // D+
        }
    } else if (t == 32) {
        R d = (R)(a[k - 1] - theta);
        for (int i = k - 1; i >= 0; --i) {
            if (i < k - 1) d = (R)(a[i] - theta) - (R)b2[i] / d;
            if (fabs((double)d) < tiny) d = d < (R)0 ? (R)-tiny : (R)tiny;
            dl[i] = d;   // D-
        }
    }
    __syncthreads();
    if (t == 0) {
        int r = 0;
        double gbest = INFINITY;
        for (int i = 0; i < k; ++i) {
            const double g = fabs((double)dd[i] + (double)dl[i] - (a[i] - theta));
            if (g < gbest) { gbest = g; r = i; }
        }
        *twist = r;
    }
    __syncthreads();
    const int r = *twist;
    if (t == 0) {   // v_r = 1 and the part above the twist
        R vi = (R)1;
        v[r] = 1.0;
        for (int i = r - 1; i >= 0; --i) {
            vi = -((R)b[i] / dd[i]) * vi;
            v[i] = (double)vi;
        }
    } else if (t == 32) {   // the part below the twist (starts from v_r = 1 itself)
        R vi = (R)1;
        for (int i = r + 1; i < k; ++i) {
            vi = -((R)b[i - 1] / dl[i]) * vi;
            v[i] = (double)vi;
        }
    }
    __syncthreads();
    __shared__ double rq_s;
    if (t == 0) {
        double nrm = 0.0;
        for (int i = 0; i < k; ++i) nrm = fma(v[i], v[i], nrm);
        const double inv = 1.0 / sqrt(nrm);
        for (int i = 0; i < k; ++i) v[i] *= inv;
        double rq = 0.0;
        for (int i = 0; i < k; ++i) {
            double tv = a[i] * v[i];
            if (i > 0) tv += b[i - 1] * v[i - 1];
            if (i + 1 < k) tv += b[i] * v[i + 1];
            rq += v[i] * tv;
        }
        rq_s = rq;
    }
    __syncthreads();
    return rq_s;
}

// Lowest eigenpair of T_k (alpha[0..k), beta[0..k-1)); beta2_last = |w|^2 of
// the current step. out[0] = theta, out[1] = beta_k |s_k|, out[2] = beta_k,
// beta[k-1] = beta_k is written, s[0..k) = normalised eigenvector.
//   1. float32 multisection (32 Sturm probes per round, one warp) brackets
//      the lowest eigenvalue to float32 resolution;
//   2. a float32 twisted factorization at the bracket's midpoint gives an
//      eigenvector accurate to about float32 precision; its float64
//      Rayleigh quotient is then accurate to about its square;
//   3. one float64 twisted factorization at that quotient and its Rayleigh
//      quotient give the pair to float64 accuracy (Rayleigh quotient
//      iteration, cubic convergence);
//   4. a float64 Sturm count just below the result confirms that no
//      eigenvalue lies below it; if one does (the float32 bracket missed a
//      close pair) the float64 multisection of the whole spectrum's bottom
//      decides instead, followed by one float64 twisted factorization.
__global__ void tridiag_lowest(const double* __restrict__ alpha, double* __restrict__ beta, int k,
                               const double* __restrict__ beta2_last, double* __restrict__ out,
                               double* __restrict__ s) {
    __shared__ double a[kMaxKrylov], b[kMaxKrylov], b2[kMaxKrylov];
    __shared__ float af[kMaxKrylov], b2f[kMaxKrylov];
    __shared__ double lo_s, hi_s, tiny_s, th_s;
    __shared__ int twist_s, bad_s;
    __shared__ double dd[kMaxKrylov], dl[kMaxKrylov], v[kMaxKrylov];
    __shared__ float ddf[kMaxKrylov], dlf[kMaxKrylov];
    const int t = threadIdx.x, nt = blockDim.x;
    for (int i = t; i < k; i += nt) { a[i] = alpha[i]; af[i] = (float)alpha[i]; }
    for (int i = t; i + 1 < k; i += nt) {
        b[i] = beta[i];
        b2[i] = beta[i] * beta[i];
        b2f[i] = (float)b2[i];
    }
    __syncthreads();
    if (t == 0) {
        double lo = a[0], hi = a[0], tn = 1e-300;
        for (int i = 0; i < k; ++i) {
            double r = (i > 0 ? fabs(b[i - 1]) : 0.0) + (i + 1 < k ? fabs(b[i]) : 0.0);
            lo = fmin(lo, a[i] - r);
            hi = fmax(hi, a[i] + r);
            tn = fmax(tn, fabs(a[i]) + r);
        }
        double pad = 1e-12 * fmax(1.0, fmax(fabs(lo), fabs(hi)));
        lo_s = lo - pad;
        hi_s = hi + pad;
        tiny_s = fmax(1e-15 * tn, 1e-200);
        bad_s = 0;
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
        return;
    }
    const double tiny = tiny_s;
    // 1. float32 multisection
    if (t < 32) {
        float lo = (float)lo_s, hi = (float)hi_s;
        lo = nextafterf(lo, -INFINITY);
        hi = nextafterf(hi, INFINITY);
        for (int round = 0; round < 8; ++round) {
            if (hi - lo <= 4e-7f * fmaxf(fabsf(lo), fabsf(hi))) break;
            const float x = lo + (hi - lo) * (float)(t + 1) / 33.0f;
            const unsigned below = __ballot_sync(0xffffffffu, sturm_count_f32(af, b2f, k, x) >= 1);
            const int f = below ? __ffs(below) - 1 : 32;
            const float nlo = f == 0 ? lo : lo + (hi - lo) * (float)f / 33.0f;
            const float nhi = f == 32 ? hi : lo + (hi - lo) * (float)(f + 1) / 33.0f;
            lo = nlo;
            hi = nhi;
        }
        if (t == 0) th_s = 0.5 * ((double)lo + (double)hi);
    }
    __syncthreads();
    // 2. float32 twisted factorization, float64 Rayleigh quotient
    const double tiny32 = fmax(1e-6 * (tiny * 1e15), 1e-30);
    double theta = twisted_rq<float>(a, b, b2, k, th_s, tiny32, ddf, dlf, v, &twist_s);
    // 3. float64 Rayleigh quotient iteration step
    theta = twisted_rq<double>(a, b, b2, k, theta, tiny, dd, dl, v, &twist_s);
    // 4. nothing below it
    if (t == 0) {
        const double delta = 1e-13 * fmax(1.0, tiny * 1e15);
        bad_s = sturm_count(a, b2, k, theta - delta) > 0;
    }
    __syncthreads();
    if (bad_s) {   // uniform: float64 multisection, then one twisted factorization
        if (t < 32) {
            double lo = lo_s, hi = hi_s;
            for (int round = 0; round < 24; ++round) {
                if (hi - lo <= 2e-16 * fmax(fabs(lo), fabs(hi))) break;
                const double x = lo + (hi - lo) * (double)(t + 1) / 33.0;
                const unsigned below = __ballot_sync(0xffffffffu, sturm_count(a, b2, k, x) >= 1);
                const int f = below ? __ffs(below) - 1 : 32;
                const double nlo = f == 0 ? lo : lo + (hi - lo) * (double)f / 33.0;
                const double nhi = f == 32 ? hi : lo + (hi - lo) * (double)(f + 1) / 33.0;
                lo = nlo;
                hi = nhi;
            }
            if (t == 0) th_s = 0.5 * (lo + hi);
        }
        __syncthreads();
        theta = twisted_rq<double>(a, b, b2, k, th_s, tiny, dd, dl, v, &twist_s);
    }
    if (t == 0) {
        double bk = sqrt(fmax(*beta2_last, 0.0));
        beta[k - 1] = bk;
        out[0] = theta;
        out[1] = bk * fabs(v[k - 1]);
        out[2] = bk;
        for (int i = 0; i < k; ++i) s[i] = v[i];
    }
}

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

// ---- Davidson helpers
constexpr int kDavMax = 48;   // largest subspace of the Davidson eigensolver

// T[i][j] = T[j][i] = h[i] for i <= j (new column of the projected matrix)
__global__ void set_column(double* __restrict__ T, int ld, int j, const double* __restrict__ h) {
    for (int i = threadIdx.x; i <= j; i += blockDim.x) {
        T[(int64_t)i * ld + j] = h[i];
        T[(int64_t)j * ld + i] = h[i];
    }
}

// Lowest eigenpair of the symmetric k x k matrix T (row pitch ld) by cyclic
// two-sided Jacobi in float64 (one CTA): the pairs of one step are disjoint,
// so all their column rotations run together, then all row rotations.
// out[0] = lowest eigenvalue, s[0..k) its unit eigenvector.
__global__ void __launch_bounds__(256) small_eigh_lowest(const double* __restrict__ T, int k, int ld,
                                                         double* __restrict__ out, double* __restrict__ s) {
    __shared__ double A[kDavMax][kDavMax + 1], V[kDavMax][kDavMax + 1];
    __shared__ double cs[kDavMax / 2], sn[kDavMax / 2];
    __shared__ int pp[kDavMax / 2], qq[kDavMax / 2];
    __shared__ double red[256];
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int e = tid; e < k * k; e += nt) {
        const int i = e / k, j = e - i * k;
        A[i][j] = T[(int64_t)i * ld + j];
        V[i][j] = i == j ? 1.0 : 0.0;
    }
    __syncthreads();
    const int ke = k + (k & 1), R = ke - 1, np = ke / 2;
    for (int sweep = 0; sweep < 30 && k > 1; ++sweep) {
        // off-diagonal and total Frobenius weight (fixed-order reduction)
        double off = 0.0, tot = 0.0;
        for (int e = tid; e < k * k; e += nt) {
            const int i = e / k, j = e - i * k;
            const double a2 = A[i][j] * A[i][j];
            tot += a2;
            if (i != j) off += a2;
        }
        red[tid] = off;
        __syncthreads();
        for (int o = nt / 2; o > 0; o >>= 1) {
            if (tid < o) red[tid] += red[tid + o];
            __syncthreads();
        }
        const double offs = red[0];
        __syncthreads();
        red[tid] = tot;
        __syncthreads();
        for (int o = nt / 2; o > 0; o >>= 1) {
            if (tid < o) red[tid] += red[tid + o];
            __syncthreads();
        }
        const double tots = red[0];
        __syncthreads();
        if (!(offs > 1e-30 * tots)) break;
        for (int st = 0; st < R; ++st) {
            if (tid < np) {
                const int a = tid == 0 ? 0 : 1 + (tid - 1 + st) % R;
                const int b = (ke - 1 - tid) == 0 ? 0 : 1 + (ke - 1 - tid - 1 + st) % R;
                const int p = min(a, b), q = max(a, b);
                double c = 1.0, sv = 0.0;
                if (q < k && A[p][q] != 0.0) {
                    const double tau = (A[q][q] - A[p][p]) / (2.0 * A[p][q]);
                    const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                    c = 1.0 / sqrt(1.0 + t * t);
                    sv = t * c;
                }
                pp[tid] = p;
                qq[tid] = q < k ? q : p;
                cs[tid] = c;
                sn[tid] = q < k ? sv : 0.0;
            }
            __syncthreads();
            // columns: A <- A J, V <- V J
            for (int e = tid; e < np * k; e += nt) {
                const int r = e / k, i = e - r * k;
                const int p = pp[r], q = qq[r];
                if (p == q) continue;
                const double c = cs[r], sv = sn[r];
                const double ap = A[i][p], aq = A[i][q];
                A[i][p] = c * ap - sv * aq;
                A[i][q] = sv * ap + c * aq;
                const double vp = V[i][p], vq = V[i][q];
                V[i][p] = c * vp - sv * vq;
                V[i][q] = sv * vp + c * vq;
            }
            __syncthreads();
            // rows: A <- J^T A
            for (int e = tid; e < np * k; e += nt) {
                const int r = e / k, j = e - r * k;
                const int p = pp[r], q = qq[r];
                if (p == q) continue;
                const double c = cs[r], sv = sn[r];
                const double ap = A[p][j], aq = A[q][j];
                A[p][j] = c * ap - sv * aq;
                A[q][j] = sv * ap + c * aq;
            }
            __syncthreads();
        }
    }
    if (tid == 0) {
        int m = 0;
        for (int i = 1; i < k; ++i)
            if (A[i][i] < A[m][m]) m = i;
        out[0] = A[m][m];
        red[0] = (double)m;
    }
    __syncthreads();
    const int m = (int)red[0];
    for (int i = tid; i < k; i += nt) s[i] = V[i][m];
}

// t = r / (theta - d), the denominator kept away from zero
__global__ void davidson_precondition(const double* __restrict__ r, const double* __restrict__ d,
                                      const double* __restrict__ theta, double* __restrict__ t, int64_t n) {
    const double th = *theta, floor = 1e-8 * fmax(1.0, fabs(th));
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double den = th - d[i];
        if (fabs(den) < floor) den = den < 0.0 ? -floor : floor;
        t[i] = r[i] / den;
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

EigResult eigsolve(HeffPlan& P, double* psi, int kmax, double tol, bool fp64_energy) {
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
    res.matvecs = k;
    if (!fp64_energy) {
        // the Ritz value and its residual estimate (of the last solve)
        CUDA_CHECK(cudaStreamSynchronize(s));
        check_device_flag(ctx);
        res.energy = host[0];
        res.resid = host[1];
        return res;
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

double rayleigh_fp64(HeffPlan& P, const double* x) {
    Ctx* ctx = P.ctx;
    cudaStream_t s = ctx->stream;
    const int64_t n = P.n;
    if (n == 0) return 0.0;
    VecWork vw;
    vw.ensure(ctx->num_sms);
    DevBuf yv((size_t)n * sizeof(double)), sc(4 * sizeof(double));
    heff_apply(P, TNH_FP64, x, yv.as<double>());
    vdot(ctx, vw, x, yv.as<double>(), n, sc.as<double>());
    vdot(ctx, vw, x, x, n, sc.as<double>() + 1);
    double h[2];
    CUDA_CHECK(cudaMemcpyAsync(h, sc.p, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    CUDA_CHECK(cudaStreamSynchronize(s));
    check_device_flag(ctx);
    TNH_REQUIRE(std::isfinite(h[0]) && h[1] > 0.0, TNH_ERR_NUMERIC, "rayleigh quotient of a zero or non-finite vector");
    return h[0] / h[1];
}

EigResult davidson(HeffPlan& P, double* psi, int kmax, double tol, bool fp64_energy) {
    Ctx* ctx = P.ctx;
    cudaStream_t s = ctx->stream;
    const int64_t n = P.n;
    TNH_REQUIRE(kmax >= 1 && kmax <= kDavMax, TNH_ERR_ARG, "davidson: krylov_dim %d out of 1..%d", kmax, kDavMax);
    EigResult res;
    if (n == 0) return res;
    const double* diag = heff_diag(P);
    VecWork vw;
    vw.ensure(ctx->num_sms);
    DevBuf Q((size_t)kmax * n * sizeof(double)), HQ((size_t)kmax * n * sizeof(double));
    DevBuf rv((size_t)n * sizeof(double)), tv((size_t)n * sizeof(double)), yv((size_t)n * sizeof(double));
    DevBuf Tm((size_t)kmax * kmax * sizeof(double));
    // scalars: h[kmax] sv[kmax] theta, |r|^2, |t|^2, misc
    DevBuf sc((size_t)(2 * kmax + 16) * sizeof(double));
    double* h = sc.as<double>();
    double* sv = h + kmax;
    double* misc = sv + kmax;   // [0] theta [1] |r|^2 [2] |t|^2 [3] |psi|^2 [4] E [5] |res|^2 [6] |t0|^2
    double* q = Q.as<double>();
    double* hq = HQ.as<double>();
    double* r = rv.as<double>();
    double* t = tv.as<double>();
    const int g = grid_for(n, ctx->num_sms);
    auto norm2 = [&](const double* x, double* out) { vdot(ctx, vw, x, x, n, out); };
    auto dots = [&](const double* basis, int k, const double* x, double* out) {
        { KScope ks_("multidot_partial", s);
        multidot_partial<<<dim3(vw.blocks, k), kRedThreads, 0, s>>>(basis, n, x, n, vw.partial.as<double>());
        }
        { KScope ks_("reduce_partials", s);
        reduce_partials<<<k, kRedThreads, 0, s>>>(vw.partial.as<double>(), vw.blocks, out);
        }
    };
    auto combine = [&](double* out, const double* basis, int k, const double* c, double sign, int overwrite) {
        KScope ks_("multi_axpy", s);
        multi_axpy<<<g, 256, 0, s>>>(out, basis, n, k, c, sign, overwrite, n);
    };
    norm2(psi, misc + 3);
    double hn2 = 0;
    CUDA_CHECK(cudaMemcpyAsync(&hn2, misc + 3, sizeof(double), cudaMemcpyDeviceToHost, s));
    CUDA_CHECK(cudaStreamSynchronize(s));
    TNH_REQUIRE(std::isfinite(hn2) && hn2 > 0.0, TNH_ERR_NUMERIC, "davidson: start vector has norm^2 %g", hn2);
    { KScope ks_("scale_copy", s);
    scale_copy<<<g, 256, 0, s>>>(psi, q, n, nullptr, misc + 3, 1);
    }
    int k = 0;
    for (int j = 0; j < kmax; ++j) {
        double* qj = q + (int64_t)j * n;
        heff_apply(P, P.prec, qj, hq + (int64_t)j * n);
        k = j + 1;
        // new column of T = Q^T H Q, lowest Ritz pair (theta, s)
        dots(q, k, hq + (int64_t)j * n, h);
        { KScope ks_("davidson_set_column", s);
        set_column<<<1, 64, 0, s>>>(Tm.as<double>(), kmax, j, h);
        }
        { KScope ks_("davidson_small_eigh", s);
        small_eigh_lowest<<<1, 256, 0, s>>>(Tm.as<double>(), k, kmax, misc, sv);
        }
        // u = Q s (into psi), r = H Q s - theta u
        combine(psi, q, k, sv, 1.0, 1);
        combine(r, hq, k, sv, 1.0, 1);
        { KScope ks_("axpy_dev", s);
        axpy_dev<<<g, 256, 0, s>>>(r, psi, misc, n);
        }
        norm2(r, misc + 1);
        double host[2];
        CUDA_CHECK(cudaMemcpyAsync(host, misc, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
        CUDA_CHECK(cudaStreamSynchronize(s));
        TNH_REQUIRE(std::isfinite(host[0]) && std::isfinite(host[1]), TNH_ERR_NUMERIC,
                    "davidson: non-finite Ritz value at step %d", j);
        const double scale = std::max(1.0, std::fabs(host[0]));
        if (j + 1 == kmax || (tol > 0.0 && std::sqrt(std::max(host[1], 0.0)) <= tol * scale)) break;
        // correction t = (theta - D)^-1 r, orthogonalised twice against Q
        { KScope ks_("davidson_precondition", s);
        davidson_precondition<<<g, 256, 0, s>>>(r, diag, misc, t, n);
        }
        norm2(t, misc + 6);
        for (int rep = 0; rep < 2; ++rep) {
            dots(q, k, t, h);
            combine(t, q, k, h, -1.0, 0);
        }
        norm2(t, misc + 2);
        double tn[5];
        CUDA_CHECK(cudaMemcpyAsync(tn, misc + 2, 5 * sizeof(double), cudaMemcpyDeviceToHost, s));
        CUDA_CHECK(cudaStreamSynchronize(s));
        // no new direction: the correction lies in the subspace to rounding
        if (!(tn[0] > 1e-24 * tn[4]) || !(tn[0] > 0.0)) break;
        { KScope ks_("scale_copy", s);
        scale_copy<<<g, 256, 0, s>>>(t, q + (int64_t)(j + 1) * n, n, nullptr, misc + 2, 1);
        }
    }
    // normalised Ritz vector in psi, float64 energy and residual
    norm2(psi, misc + 3);
    { KScope ks_("scale_copy", s);
    scale_copy<<<g, 256, 0, s>>>(psi, psi, n, nullptr, misc + 3, 1);
    }
    res.matvecs = k;
    if (!fp64_energy) {
        // the Ritz value and residual of the last projected solve
        double rr[2];
        CUDA_CHECK(cudaMemcpyAsync(rr, misc, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
        CUDA_CHECK(cudaStreamSynchronize(s));
        check_device_flag(ctx);
        res.energy = rr[0];
        res.resid = std::sqrt(std::max(rr[1], 0.0));
        return res;
    }
    double* y = yv.as<double>();
    heff_apply(P, TNH_FP64, psi, y);
    vdot(ctx, vw, psi, y, n, misc + 4);
    { KScope ks_("axpy_dev", s);
    axpy_dev<<<g, 256, 0, s>>>(y, psi, misc + 4, n);
    }
    vdot(ctx, vw, y, y, n, misc + 5);
    double fin[2];
    CUDA_CHECK(cudaMemcpyAsync(fin, misc + 4, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    CUDA_CHECK(cudaStreamSynchronize(s));
    check_device_flag(ctx);
    res.energy = fin[0];
    res.resid = std::sqrt(std::max(fin[1], 0.0));
    res.matvecs = k;
    return res;
}

}  // namespace tnh

using namespace tnh;

extern "C" tnh_status tnh_eigsolve_davidson(tnh_heff* plan, double* psi, int32_t krylov_dim, double tol,
                                            double* energy, double* resid, int32_t* matvecs) {
    auto* P = reinterpret_cast<HeffPlan*>(plan);
    return guard(P ? P->ctx : nullptr, [&] {
        TNH_REQUIRE(P && psi, TNH_ERR_ARG, "tnh_eigsolve_davidson: NULL argument");
        EigResult r = davidson(*P, psi, krylov_dim, tol);
        if (energy) *energy = r.energy;
        if (resid) *resid = r.resid;
        if (matvecs) *matvecs = r.matvecs;
    });
}

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

extern "C" tnh_status tnh_tridiag_lowest(tnh_ctx* ctx, int32_t k, const double* alpha, const double* beta,
                                         double* theta, double* v) {
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    return guard(c, [&] {
        TNH_REQUIRE(c && alpha && theta && v && (k == 1 || beta), TNH_ERR_ARG, "tnh_tridiag_lowest: NULL argument");
        TNH_REQUIRE(k >= 1 && k < kMaxKrylov, TNH_ERR_ARG, "tnh_tridiag_lowest: k = %d out of 1..%d", k,
                    kMaxKrylov - 1);
        for (int i = 0; i < k; ++i) TNH_REQUIRE(std::isfinite(alpha[i]), TNH_ERR_NUMERIC, "tnh_tridiag_lowest: alpha");
        for (int i = 0; i + 1 < k; ++i) TNH_REQUIRE(std::isfinite(beta[i]), TNH_ERR_NUMERIC, "tnh_tridiag_lowest: beta");
        CUDA_CHECK(cudaSetDevice(c->device));
        cudaStream_t s = c->stream;
        // device copies: alpha [k], beta [k] (beta[k-1] receives beta_k = 0), beta2_last, out[3], s[k]
        DevBuf d((size_t)(3 * k + 4) * sizeof(double));
        double* da = d.as<double>();
        double* db = da + k;
        double* dout = db + k;   // [0..2]
        double* dz = dout + 3;   // beta2_last = 0
        double* ds = dz + 1;
        CUDA_CHECK(cudaMemsetAsync(d.p, 0, d.bytes, s));
        CUDA_CHECK(cudaMemcpyAsync(da, alpha, (size_t)k * sizeof(double), cudaMemcpyHostToDevice, s));
        if (k > 1) CUDA_CHECK(cudaMemcpyAsync(db, beta, (size_t)(k - 1) * sizeof(double), cudaMemcpyHostToDevice, s));
        {
            KScope ks_("tridiag_lowest", s);
            tridiag_lowest<<<1, 256, 0, s>>>(da, db, k, dz, dout, ds);
        }
        CUDA_CHECK(cudaGetLastError());
        CUDA_CHECK(cudaMemcpyAsync(theta, dout, sizeof(double), cudaMemcpyDeviceToHost, s));
        CUDA_CHECK(cudaMemcpyAsync(v, ds, (size_t)k * sizeof(double), cudaMemcpyDeviceToHost, s));
        CUDA_CHECK(cudaStreamSynchronize(s));
    });
}
