// Effective-Hamiltonian plan and the device Lanczos eigensolver.
#pragma once

#include "tnh_internal.h"

namespace tnh {

struct HeffPlan {
    Ctx* ctx = nullptr;
    cudaStream_t stream = nullptr;   // copy: freeing a plan never touches ctx
    tnh_precision prec = TNH_FP64;
    int64_t n = 0;          // elements of the two-site state
    Layout psi;             // its layout
    double flops = 0.0;
    std::unique_ptr<ContractPlan> c1, c2, c3, c4;
    DevBuf t1, t2, t3, Ld, Rd, W1d, W2d;     // owned copies (public entry point)
    const double *Lp = nullptr, *Rp = nullptr, *W1p = nullptr, *W2p = nullptr;
    Workspace ws;
    ~HeffPlan();
};

// copy_inputs: keep private copies of L, W1, W2, R (else reference the
// caller's device data, which must outlive the plan)
std::unique_ptr<HeffPlan> make_heff(Ctx* ctx, const Layout& L, const Layout& W1, const Layout& W2,
                                    const Layout& R, const Layout& psi, tnh_precision prec,
                                    bool copy_inputs = true);
void heff_apply(HeffPlan& P, tnh_precision prec, const double* x, double* y);

struct EigResult {
    double energy = 0, resid = 0;
    int matvecs = 0;
};
// Lanczos on the plan; psi (device, length P.n) in/out.
EigResult eigsolve(HeffPlan& P, double* psi, int krylov_dim, double tol);

// ---- device vector helpers (float64, deterministic reductions) -----------
struct VecWork {
    DevBuf partial, scal;   // reduction partials, device scalars
    int blocks = 0;
    void ensure(int nsms);
};
void vdot(Ctx* ctx, VecWork& w, const double* x, const double* y, int64_t n, double* d_out);
void vscale_copy(Ctx* ctx, const double* x, double* y, int64_t n, const double* d_num, const double* d_den,
                 int mode);

}  // namespace tnh
