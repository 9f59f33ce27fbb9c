// Effective-Hamiltonian plan and the device Lanczos eigensolver.
#pragma once

#include <array>

#include "gather.h"
#include "tnh_internal.h"

namespace tnh {

// One GEMM operand of the plan in both formats (float64 rows for the FP64
// GEMM, split-bfloat16 tiles for the tcgen05 GEMM), per task.
struct HeffOperand {
    std::vector<OpGeom> g64, gtc;
    int64_t elems64 = 0, tiles = 0;
    DevBuf d_g64, d_gtc;
    void add_task(int64_t rows, int64_t K);
    int count() const { return (int)gtc.size(); }
};
// One GEMM of the plan. The tcgen05 tasks are launched as given in tc: the
// block tasks of tc_base, or, with split > 1, every block task cut into up
// to split K ranges that write float32 partials, summed by one reduction
// launch (reds) into the real output.
struct HeffGemm {
    std::vector<GemmTask> f64, tc, tc_base;
    int tiles64 = 0, tilestc = 0;
    int split = 1;
    int tile_policy = 0;   // N tile widths of the tcgen05 tasks (see tile_width)
    std::vector<SplitRed> reds;
    std::vector<RedBlock> red_blocks;
    int64_t red_total = 0, part_elems = 0;
    DevBuf d_f64, d_tc, d_reds, d_red_blocks;
    // the FP64 GEMM: with split64 > 1 the tasks of f64run write float64
    // partial slabs (K slices of 16-multiples), summed by reds64 in order
    int split64 = 1, tiles64run = 0;
    std::vector<GemmTask> f64run;
    std::vector<SplitRed> reds64;
    std::vector<RedBlock> red64_blocks;
    int64_t red64_total = 0, part64_elems = 0;
    DevBuf d_f64run, d_reds64, d_red64_blocks;
};

// ---- device vector helpers (float64, deterministic reductions) -----------
struct VecWork {
    DevBuf partial, scal;   // reduction partials, device scalars
    int blocks = 0;
    void ensure(int nsms);
};

struct HeffPlan {
    Ctx* ctx = nullptr;
    cudaStream_t stream = nullptr;   // copy: freeing a plan never touches ctx
    tnh_precision prec = TNH_FP64;
    int planes = 0;         // split-bfloat16 planes of prec (0 for FP64)
    int64_t n = 0;          // elements of the two-site state
    Layout psi;             // its layout
    double flops = 0.0;     // method flops of one application (S1..S4)
    double f_s1 = 0.0, f_s23 = 0.0, f_s4 = 0.0;
    // operands: S1 = L (A) x psi (B), S4 = T3 (A) x R (B)
    HeffOperand oL, oX, oT, oR;
    GatherJob jX;           // per application: pack psi
    W12Job jW;              // per application: fused S2+S3
    GatherJob jT;           // the same step as segments of S4's operand A tiles, formed inside S4 (three planes)
    bool fusedS4 = false;   // S4 forms its operand A from T1 itself (no separate W1.W2 pass)
    HeffGemm g1, g4;
    DevBuf L64, Ltc, R64, Rtc;   // L and R packed once
    DevBuf opX;             // operand B of S1 (either format)
    DevBuf opT64, opTtc;    // operand A of S4, one per format
    DevBuf t1;              // S1 result (float32 in the split modes)
    DevBuf row_off;         // S4 output row -> element offset in psi's layout
    DevBuf part;            // float32 partial slabs of K-split GEMMs
    DevBuf part64;          // float64 partial slabs of K-split FP64 GEMMs
    int64_t t1_elems = 0;
    bool zero_y = false;    // some output rows are written by no S4 task
    std::array<int, 5> tune{0, 1, 0, 1, 0};   // tile policy / K split of S1, then of S4; S4 fused
    bool tune_measured = false;            // chosen by timing in this plan (not cached or forced)
    int strategy = 0;                      // 0: combine, then contract; 1: block pairs (make_heff)
    bool strategy_measured = false;        // both strategies were timed for this plan
    float strategy_ms[2] = {0.f, 0.f};     // their times per product when measured
    // one CUDA graph per format (float64, split): the four launches of an
    // application, replayed with the x and y arguments patched in
    struct Graph {
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        cudaGraphNode_t nx = nullptr, ny = nullptr;   // the kernel nodes reading x / writing y
        std::vector<void*> ax, ay;                    // their argument pointer arrays
        int ix = 0, iy = 0;                           // index of x / y among the arguments
        int ny_args = 0;                              // argument count of the y node's kernel
        const double* x = nullptr;
        double* y = nullptr;
        int calls = 0;
    } graphs[2];
    // previous-state projectors (excited-state DMRG, Sec. 7.2): every
    // application adds weight * phi_i <phi_i, x> for the nproj vectors phi_i
    int nproj = 0;
    double pweight = 0.0;
    DevBuf proj;            // [nproj][n]
    DevBuf pcoef;           // [nproj] device scalars
    VecWork pvw;
    // diagonal of H_eff (Davidson preconditioner): environment diagonals
    // Ld [a][w], Rd [b][w2] taken when the plan is made, per-block and
    // per-(s1, s2) tables; the diagonal itself is formed on first use
    DevBuf Ld, Rd, d_dblocks, d_dstart, d_dterms, diag;
    int dg_wdim = 0, dg_zdim = 0, dg_d2 = 0, dg_nblocks = 0;
    int64_t dg_maxblock = 0;
    DevBuf hx, hy;          // device vectors of tnh_heff_apply_host (made on its first call)
    ~HeffPlan();
};

// L, W1, W2, R are read while the plan is made and not referenced after.
// strategy 0: combine the blocks of a contracted sector into one GEMM task
// (S1 per a-sector, S4 per b'-sector); 1: one task per block pair (S1) or
// per output block (S4).
std::unique_ptr<HeffPlan> make_heff_strategy(Ctx* ctx, const Layout& L, const Layout& W1, const Layout& W2,
                                             const Layout& R, const Layout& psi, tnh_precision prec, int strategy);
// The same with the strategy chosen per shape by timing both (cached in the
// context), or forced by TNH_HEFF_STRATEGY.
std::unique_ptr<HeffPlan> make_heff(Ctx* ctx, const Layout& L, const Layout& W1, const Layout& W2,
                                    const Layout& R, const Layout& psi, tnh_precision prec);
// H_eff (of the plan's MPO terms) plus the projectors, if any.
void heff_apply(HeffPlan& P, tnh_precision prec, const double* x, double* y);
// Diagonal of the MPO part of H_eff (device [P.n], float64), formed once.
const double* heff_diag(HeffPlan& P);
// Replace the projectors: phi is DEVICE [k][P.n] (copied), weight the penalty.
void set_projectors(HeffPlan& P, int k, const double* phi, double weight);
// y += P.pweight * sum_i phi_i <phi_i, x> (float64, deterministic).
void add_projectors(HeffPlan& P, const double* x, double* y);

struct EigResult {
    double energy = 0, resid = 0;
    int matvecs = 0;
};
// Lanczos on the plan; psi (device, length P.n) in/out. With fp64_energy
// the energy and residual come from a final FP64 product with the Ritz
// vector, else they are the Ritz value and residual estimate of the run.
EigResult eigsolve(HeffPlan& P, double* psi, int krylov_dim, double tol, bool fp64_energy = true);
// Davidson with the diagonal preconditioner; same contract as eigsolve.
EigResult davidson(HeffPlan& P, double* psi, int krylov_dim, double tol, bool fp64_energy = true);

void vdot(Ctx* ctx, VecWork& w, const double* x, const double* y, int64_t n, double* d_out);
// <x|H x> / <x|x> with the plan's FP64 product (x device, length P.n).
double rayleigh_fp64(HeffPlan& P, const double* x);
void vscale_copy(Ctx* ctx, const double* x, double* y, int64_t n, const double* d_num, const double* d_den,
                 int mode);

}  // namespace tnh
