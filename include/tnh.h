/*
 * tnh.h -- C ABI of the GB300 two-site DMRG effective-Hamiltonian library.
 *
 * The library computes the hot path of two-site DMRG as described in the
 * ITensor paper (arXiv:2007.14822): the labelled tensor contraction over
 * shared indices (Sec. 4, Sec. 9.1), on dense and QN block-sparse storage
 * (Sec. 6, Sec. 8, Sec. 9.2), the effective-Hamiltonian product H_eff . psi
 * that the eigensolver applies at every bond (Sec. 7.2), the environment
 * update, the truncated SVD with cutoff and maxdim (Sec. 5) and the sweep
 * driver dmrg(H, psi0, sweeps) (Sec. 7.2).
 *
 * Conventions shared by every entry point
 *   - Real float64 data, row-major, rightmost index fastest.
 *   - Tensor data pointers are DEVICE pointers owned by the caller; all
 *     metadata (indices, block lists) are HOST pointers read during the call
 *     and not retained.
 *   - Every call is asynchronous on the context's stream unless documented
 *     otherwise; calls that must read a result on the host (a kept dimension,
 *     an energy) synchronise that stream and say so.
 *   - No exception crosses the ABI. Every call returns a tnh_status; the text
 *     of the last error of a context is returned by tnh_last_error().
 *   - Nothing falls back to the CPU: when the device or the kernels are not
 *     usable the call fails with TNH_ERR_CUDA.
 *   - Errors any call may return besides those listed with it: TNH_ERR_ARG
 *     for a NULL handle or output pointer, a negative size or an unknown
 *     enum value; TNH_ERR_OOM when a device allocation fails (everything the
 *     call had allocated is released first); TNH_ERR_TIMEOUT when a bounded
 *     device wait gave up (the call that finds the context's device error
 *     flag set reports it and clears it; the context stays usable);
 *     TNH_ERR_CUDA for a failed CUDA call, named in tnh_last_error(). The
 *     functions that free a handle accept NULL and do nothing.
 */
#ifndef TNH_H
#define TNH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    TNH_OK = 0,
    TNH_ERR_ARG = 1,        /* null pointer, bad enum, bad size            */
    TNH_ERR_LABEL = 2,      /* labels do not pair up as a contraction needs */
    TNH_ERR_ARROW = 3,      /* contracted QN indices with equal arrows     */
    TNH_ERR_FLUX = 4,       /* a stored block violates the tensor's flux   */
    TNH_ERR_SHAPE = 5,      /* sector dims / block offsets inconsistent    */
    TNH_ERR_OOM = 6,        /* device allocation failed                    */
    TNH_ERR_CUDA = 7,       /* CUDA runtime / launch error                 */
    TNH_ERR_TIMEOUT = 8,    /* a bounded device wait gave up               */
    TNH_ERR_NUMERIC = 9,    /* NaN/Inf or Lanczos breakdown at start       */
    TNH_ERR_NOT_CONVERGED = 10
} tnh_status;

/* Arithmetic used by the contractions.
 *   TNH_FP64    plain float64 on the CUDA cores (the reference GPU path).
 *   TNH_BF16x6  each float64 operand split into three bfloat16 parts
 *               x = hi + mid + lo; six tensor-core products (hh, hm, mh,
 *               hl, lh, mm) accumulated in float32 (tcgen05, sm_103a).
 *   TNH_BF16x3  two-part split, three products (hh, hm, mh).
 *   TNH_BF16    one bfloat16 part, one product.
 * The split modes are the "lower precision" storage the paper mentions in
 * Sec. 6; their measured error against float64 is reported by the tests. */
typedef enum {
    TNH_FP64 = 0,
    TNH_BF16x6 = 1,
    TNH_BF16x3 = 2,
    TNH_BF16 = 3
} tnh_precision;

typedef struct tnh_ctx tnh_ctx;
typedef struct tnh_heff tnh_heff;
typedef struct tnh_svd tnh_svd;

/* A QN index (Sec. 3, Sec. 8.2).
 *   label     integer the contraction matches; equal labels are summed
 *             (it stands for the Index id + prime level of Sec. 3).
 *   nsect     number of sectors (>= 1); a dense index has one sector.
 *   nq        number of integer charges in a QN (0..4).
 *   qn        host [nsect * nq] charges, sector-major.
 *   sect_dim  host [nsect] sector dimensions (>= 1).
 *   arrow     +1 Out (charges added to the flux), -1 In (subtracted). */
typedef struct {
    int64_t label;
    int32_t nsect;
    int32_t nq;
    const int32_t* qn;
    const int32_t* sect_dim;
    int32_t arrow;
} tnh_index;

/* A block-sparse tensor (Sec. 6 "Block sparse storage", Sec. 9.2).
 *   rank        number of indices (0..8).
 *   inds        host [rank].
 *   nblocks     number of stored blocks; each block is a dense row-major
 *               array of the sector dimensions it selects.
 *   block_sect  host [nblocks * rank] sector number of each index.
 *   block_off   host [nblocks] element offset of each block in data.
 *   data        DEVICE float64 pointer (caller-owned).
 *   size        number of float64 elements behind data (bounds check).
 * A dense tensor is one block with one sector per index. Every block must
 * have the same flux (sum of arrow * charge); otherwise TNH_ERR_FLUX. */
typedef struct {
    int32_t rank;
    const tnh_index* inds;
    int32_t nblocks;
    const int32_t* block_sect;
    const int64_t* block_off;
    double* data;
    int64_t size;
} tnh_tensor;

/* ---- context ----------------------------------------------------------- */

/* Create a context on CUDA device `device` using `stream` (a cudaStream_t,
 * NULL for the legacy default stream). The library keeps the stream handle;
 * the caller keeps ownership of the stream. TNH_ERR_ARG for a device index
 * out of range; TNH_ERR_CUDA when there is no device or it is not an sm_103
 * GPU (the library is built for sm_103a only). */
tnh_status tnh_create(tnh_ctx** ctx, int device, void* stream);
/* Synchronise the context's stream and free the context. Plans and SVD
 * results made on it must not be used afterwards (they refer to it); they
 * may still be freed. NULL does nothing. */
void tnh_destroy(tnh_ctx* ctx);
/* Text of the last error raised on `ctx` (or of the last context-free error
 * when ctx is NULL). Valid until the next call on the same context. */
const char* tnh_last_error(const tnh_ctx* ctx);
/* Block until all work queued by the context has finished; reports a
 * bounded device wait that gave up in that work (TNH_ERR_TIMEOUT). */
tnh_status tnh_sync(tnh_ctx* ctx);

/* Kernel profiling (no counterpart in the paper; measurement support).
 * Between tnh_profile_begin and tnh_profile_end every kernel the library
 * launches for this context on the calling thread is bracketed by CUDA
 * events on its stream. tnh_profile_end synchronises the stream and returns,
 * per kernel name (at most max_kinds; *nkinds is the number found):
 * names [max_kinds * 64] NUL-terminated, launches, and summed device time
 * in milliseconds. Any output array may be NULL. */
tnh_status tnh_profile_begin(tnh_ctx* ctx);
tnh_status tnh_profile_end(tnh_ctx* ctx, int32_t max_kinds, int32_t* nkinds, char* names,
                           int64_t* launches, double* ms);

/* ---- failure injection (test support; no counterpart in the paper) ------
 * The library turns failures into status codes and keeps the context usable.
 * These calls make failures happen on purpose, without faulting a device.
 *
 * tnh_debug_fail_alloc: the k-th device allocation the library makes from
 * now on (k = 1: the next one; any context, any thread) fails as if the
 * device were out of memory, so the call making it returns TNH_ERR_OOM after
 * releasing everything it had allocated. k = 0 disarms. Process-wide.
 * TNH_ERR_ARG for k < 0.
 *
 * tnh_debug_pool_used: synchronises the context's stream, then writes the
 * bytes of the library's device memory pool (on the context's device) held
 * by live allocations: equal before and after a failed call means nothing
 * leaked.
 *
 * tnh_debug_wait_timeout: launches one thread that waits on a barrier
 * nothing ever completes, with the bounded wait the GEMM pipelines use; it
 * gives up after limit_ns (1 us .. 1 s), records the site in the context's
 * device error flag and returns. The call then returns TNH_ERR_TIMEOUT (as
 * any call that finds the flag set) and clears the flag; the context stays
 * usable. TNH_ERR_ARG for a limit outside the range. */
tnh_status tnh_debug_fail_alloc(int64_t k);
tnh_status tnh_debug_pool_used(tnh_ctx* ctx, uint64_t* bytes);
tnh_status tnh_debug_wait_timeout(tnh_ctx* ctx, uint64_t limit_ns);

/* tnh_debug_convert_check (test support): the packers round float64 inputs to
 * float32, and the epilogues widen float32 results to float64, with integer
 * operations (IEEE 754 binary32/binary64 formats; round to nearest, ties to
 * even) instead of the float64 pipe. This call runs both on n bit patterns
 * from a SplitMix64 counter generator seeded with seed (uniform patterns,
 * exponents across and beyond the float32 range, exact ties, the top binade)
 * and writes to *mismatches how many results differ in their bits from the
 * GPU's own conversion (NaN equals NaN). Synchronises the stream. */
tnh_status tnh_debug_convert_check(tnh_ctx* ctx, uint64_t n, uint64_t seed, uint64_t* mismatches);

/* ---- layout helper (host only, no device work) ------------------------- */

/* Enumerate the blocks of a tensor with the given indices and flux (Sec. 8.3:
 * only blocks whose flux equals the tensor's flux are stored), in
 * lexicographic order of the sector tuple, packed contiguously.
 *   flux        host [nq] (ignored when nq == 0).
 *   nblocks     out: number of allowed blocks.
 *   block_sect  out host [*nblocks * rank] or NULL to only count.
 *   block_off   out host [*nblocks] or NULL.
 *   total       out: number of elements of the packed storage.
 * Call once with NULL buffers to size them, then again to fill them. */
tnh_status tnh_layout(int32_t rank, const tnh_index* inds, const int32_t* flux,
                      int32_t* nblocks, int32_t* block_sect, int64_t* block_off,
                      int64_t* total);

/* ---- labelled contraction (Sec. 4, Sec. 9.1, Sec. 9.4) ------------------ */

/* C = A * B. Indices of A and B with equal labels are summed; they must
 * have the same sectors and opposite arrows (TNH_ERR_ARROW, Sec. 8.3). Every
 * other label must appear exactly once in C (TNH_ERR_LABEL), in any order;
 * C's blocks are given by the caller (tnh_layout) and every C block not
 * reached by a block pair is set to zero. A block-sparse product is the set
 * of dense block-pair products whose contracted sectors agree; pairs landing
 * on the same C block are summed (Sec. 9.4). Synchronises the stream (the
 * temporary plan and workspace are freed on return). */
tnh_status tnh_contract(tnh_ctx* ctx, const tnh_tensor* A, const tnh_tensor* B,
                        tnh_tensor* C, tnh_precision prec);

/* C = A * B for DENSE float64 tensors (one block, one sector per index),
 * with the same label rules and the same kernels as tnh_contract in
 * TNH_FP64, but allocating nothing, on the device or the host, when it
 * succeeds. The paper has no counterpart: this is for callers that must not
 * allocate while they work -- a process that reserved all device memory at
 * start-up, a latency-bound loop where cudaMalloc/cudaFree would stall the
 * device, a framework that only hands out memory from its own pool. Its
 * scratch (packed operands, GEMM result, launch descriptors) lives in one
 * static device array of 16 MiB that every GPU loading the library holds
 * until the process exits; a contraction needing more than that is refused
 * with TNH_ERR_ARG (use tnh_contract). The launch descriptors are written
 * into that array by a kernel that gets them as launch arguments: no host
 * buffer is copied. The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress) and caches it. Every call reuses the same
 * array, so calls whose work overlaps on the GPU (other streams, other
 * contexts on the same device) race and must be serialised by the caller. Asynchronous on the context's
 * stream. Errors, all raised before anything is launched: TNH_ERR_LABEL for
 * a label repeated within A, B or C, or a free label missing in C;
 * TNH_ERR_SHAPE when a C index differs from the A or B index of its label
 * in dimension or arrow; TNH_ERR_ARROW for a contracted pair with equal
 * arrows; TNH_ERR_ARG for a tensor that is not dense or too large. */
tnh_status tnh_contract_dense_noalloc(tnh_ctx* ctx, const tnh_tensor* A, const tnh_tensor* B,
                                      tnh_tensor* C);

/* ---- effective Hamiltonian (Sec. 7.2) ---------------------------------- */

/* Plan y = H_eff . psi with
 *   y[a',s1',s2',b'] = sum L[a,w,a'] W1[w,w1,s1,s1'] W2[w1,w2,s2,s2']
 *                          R[b,w2,b'] psi[a,s1,s2,b]
 *   L   [a, w, a']        left environment  (a In, w Out, a' Out)
 *   W1  [w, w1, s1, s1']  MPO tensor of site 1 (w In, w1 Out, s In, s' Out)
 *   W2  [w1, w2, s2, s2'] MPO tensor of site 2
 *   R   [b, w2, b']       right environment (b Out, w In, b' In)
 *   psi [a, s1, s2, b]    layout of the two-site state (data ignored).
 * Labels are taken from the position, not from the index labels. L, R and
 * the W's are read during the call (the plan keeps packed copies; the
 * caller may free them afterwards). Synchronises the context's stream.
 * Errors: TNH_ERR_ARG for other ranks or an unknown precision;
 * TNH_ERR_SHAPE when two contracted indices have different sectors, an
 * output index differs from psi's, or psi's storage is smaller than its
 * blocks; TNH_ERR_ARROW for contracted indices with equal arrows;
 * TNH_ERR_FLUX when L, W1, W2 and R together do not conserve psi's flux. */
tnh_status tnh_heff_plan(tnh_ctx* ctx, const tnh_tensor* L, const tnh_tensor* W1,
                         const tnh_tensor* W2, const tnh_tensor* R,
                         const tnh_tensor* psi, tnh_precision prec, tnh_heff** plan);
/* H_eff of a sum of MPOs, H = sum_t H_t (Sec. 7.2): nterm environments and
 * MPO tensors L[t], W1[t], W2[t], R[t] as for tnh_heff_plan, every term with
 * its own w, w1, w2 link indices (the a, s and b indices agree). The plan is
 * the one of the terms' direct sum: the w links are joined sector by sector,
 * term after term, so every grouped GEMM covers all terms and S4 sums them
 * along its K dimension. Same ownership as tnh_heff_plan; TNH_ERR_SHAPE if
 * the terms' shared indices differ. */
tnh_status tnh_heff_plan_sum(tnh_ctx* ctx, int32_t nterm, const tnh_tensor* L, const tnh_tensor* W1,
                             const tnh_tensor* W2, const tnh_tensor* R, const tnh_tensor* psi,
                             tnh_precision prec, tnh_heff** plan);
/* Projectors added to the plan's product (excited-state DMRG, Sec. 7.2):
 * from now on every application also adds weight * phi_i <phi_i, x> for the
 * k vectors phi (DEVICE float64 [k][n] in the psi layout, copied; k = 0
 * removes them), in float64 with deterministic reductions. k <= 256. */
tnh_status tnh_heff_set_projectors(tnh_heff* plan, int32_t k, const double* phi, double weight);
/* y = H_eff . x; x and y are DEVICE float64 vectors in the psi layout of the
 * plan (they must not alias: TNH_ERR_ARG). Asynchronous on the plan's
 * context stream. */
tnh_status tnh_heff_apply(tnh_heff* plan, const double* x, double* y);
/* y = H_eff . x for HOST vectors (float64, n elements in the psi layout): x is
 * copied to the device, the product runs in the plan's precision, y is copied
 * back, and the call returns when y is on the host (it synchronises the
 * plan's stream). x and y may be the same array. Page-locked host memory
 * makes the copies asynchronous DMA; pageable memory works, slower. The
 * first call on a plan allocates the plan's two device vectors (freed with
 * the plan). */
tnh_status tnh_heff_apply_host(tnh_heff* plan, const double* x, double* y);
/* Same product in another precision than the plan's (FP64 is always
 * available; a split mode is available when the plan was made with it,
 * else TNH_ERR_ARG). x and y must not alias (TNH_ERR_ARG). */
tnh_status tnh_heff_apply_prec(tnh_heff* plan, tnh_precision prec,
                               const double* x, double* y);
/* Algorithmic flops of one product: 2 M N K summed over every block GEMM of
 * the contraction chain (split-precision extra products not counted). */
tnh_status tnh_heff_flops(const tnh_heff* plan, double* flops);
/* The same flops split by step, for measurement: the S1 GEMM (sum over a of
 * L psi), the contractions with W1 and W2 (counted as the labelled chain
 * would, although the plan applies them fused in one pass) and the S4 GEMM
 * (sum over w2, b with R). s1 + s23 + s4 is tnh_heff_flops. */
tnh_status tnh_heff_flops_detail(const tnh_heff* plan, double* s1, double* s23, double* s4);
/* The choices made for the plan (choice [8]):
 * - choice[5]: the block-contraction strategy (Sec. 9.4: neither always
 *   wins): 0 combines the blocks of a contracted sector into one GEMM task
 *   (S1 one task per a-sector, S4 one per b'-sector), 1 contracts block pairs
 *   (S1 one task per (L block, psi block) pair, S4 one per output block);
 *   choice[6] = 1 when both were built and timed for this plan (0: the
 *   context had timed this shape before, or TNH_HEFF_STRATEGY forced it);
 * - for the two tcgen05 GEMMs (split-precision plans): choice[0] / choice[2]
 *   the N tile policy of S1 / S4 (0: 128-wide tiles; 1: widths 128, 64 or 32
 *   per output block, fewest operand bytes; 2: the same, fewest MMA
 *   columns), choice[1] / choice[3] their K-split factor (1, 2, 4, 8),
 *   choice[4] 1 when the plan timed the candidates itself (0: reused from
 *   the context or the TNH_TUNE_CACHE file, or forced by TNH_HEFF_SPLIT /
 *   TNH_HEFF_TILES). An FP64 plan reports 0 1 0 1 0 for these;
 * - choice[7]: 1 when the S4 GEMM forms its operand A itself from T1 (the
 *   W1.W2 step inside the GEMM, no separate pass; chosen by timing both, or
 *   forced by TNH_HEFF_FUSED=0/1), 0 otherwise. */
tnh_status tnh_heff_tuning(const tnh_heff* plan, int32_t* choice);
/* Diagonal of the MPO part of H_eff (the projectors excluded), DEVICE
 * float64 [n] in the psi layout:
 *   d[a,s1,s2,b] = sum L[a,w,a] W1[w,w1,s1,s1] W2[w1,w2,s2,s2] R[b,w2,b].
 * Synchronises the stream. */
tnh_status tnh_heff_diag(tnh_heff* plan, double* d);
/* Number of float64 elements of the psi layout. */
tnh_status tnh_heff_size(const tnh_heff* plan, int64_t* n);
void tnh_heff_free(tnh_heff* plan);

/* Lowest eigenpair of H_eff by Lanczos with full reorthogonalisation
 * (Gram-Schmidt applied twice), starting from psi (DEVICE, overwritten by the
 * normalised Ritz vector). Matvecs run in the plan's precision; the Krylov
 * vectors, dot products, tridiagonal eigensolve and the final energy
 * E = <psi|H psi> and residual |H psi - E psi| run in float64 on the device
 * (the final product is an FP64 H_eff). Stops when the Ritz residual
 * estimate falls below tol * max(1, |E|) or after krylov_dim matvecs
 * (1 <= krylov_dim <= 255, else TNH_ERR_ARG; a zero or non-finite start
 * vector is TNH_ERR_NUMERIC). Synchronises the context's stream once per
 * iteration. */
tnh_status tnh_eigsolve(tnh_heff* plan, double* psi, int32_t krylov_dim, double tol,
                        double* energy, double* resid, int32_t* matvecs);
/* Lowest eigenpair of H_eff by Davidson: the subspace grows by the
 * correction (theta - D)^-1 r of the Ritz pair (theta, u), r = H u - theta u,
 * D the diagonal of the MPO part of H_eff, orthogonalised twice against the
 * subspace. The projected matrix is solved by float64 Jacobi on the device.
 * Same arguments, stop rule (|r| <= tol * max(1, |E|)) and final float64
 * energy and residual as tnh_eigsolve; krylov_dim <= 48. */
tnh_status tnh_eigsolve_davidson(tnh_heff* plan, double* psi, int32_t krylov_dim, double tol,
                                 double* energy, double* resid, int32_t* matvecs);

/* Lowest eigenpair of the symmetric tridiagonal matrix with diagonal
 * alpha [k] and off-diagonal beta [k-1] (HOST arrays), by the kernel the
 * Lanczos eigensolver runs after each step: float32 Sturm multisection, one
 * float32 and one float64 twisted factorization with their Rayleigh
 * quotients, a float64 Sturm check that nothing lies below the result (else
 * float64 multisection). Writes theta and the normalised eigenvector v [k]
 * (HOST; its sign is arbitrary). For testing the eigensolver's inner step;
 * 1 <= k <= 255, TNH_ERR_NUMERIC for non-finite entries. Synchronous. */
tnh_status tnh_tridiag_lowest(tnh_ctx* ctx, int32_t k, const double* alpha, const double* beta,
                              double* theta, double* v);

/* ---- environment update ------------------------------------------------ */

/* dir = +1: E_out[b,w',b'] = sum E[a,w,a'] A[a,s,b] W[w,w',s,s'] A[a',s',b']
 * dir = -1: E_out[a,w,a'] = sum A[a,s,b] W[w,w',s,s'] A[a',s',b'] E[b,w',b']
 * A [a, s, b] is an MPS tensor (a Out, s Out, b In); its bra copy has the
 * arrows reversed (real data). E_out's blocks are given by the caller.
 * Synchronises the stream (temporary plan and workspace). */
tnh_status tnh_env_update(tnh_ctx* ctx, int32_t dir, const tnh_tensor* E,
                          const tnh_tensor* A, const tnh_tensor* W,
                          tnh_tensor* E_out, tnh_precision prec);

/* ---- truncated SVD (Sec. 5) --------------------------------------------- */

/* Factorise T with its first nrow indices as rows: blocks are grouped by
 * their row charge (each group is one dense matrix, as a combiner groups
 * equal-QN sectors, Sec. 4) and every group is factorised by one-sided
 * Jacobi on the device: float32 block sweeps find the dominant subspace,
 * float64 sweeps on the candidate columns give the result. The candidates
 * are the kept count k that the float32 values predict under the same
 * cutoff/maxdim rule, plus 16 + k/8, plus every column within 1e-4 of the
 * largest singular value, at most a group's row count per group. The
 * singular values of all groups are pooled and truncated in float64: the
 * squares are summed from the smallest upward while their share of the total
 * stays <= cutoff, at most maxdim and at least max(mindim, 1) values are kept
 * (Sec. 5); values with s^2 below 1e-16 of the total are float64 zeros and
 * are kept only if mindim asks for them. Ties are ordered by group, then position. exact_side = 0 makes U
 * orthonormal to float64 accuracy (a left-to-right move), 1 makes V so (a
 * right-to-left move); the other factor is the float64 product with T.
 * Synchronises the stream (the kept count sizes the results). */
tnh_status tnh_svd_trunc(tnh_ctx* ctx, const tnh_tensor* T, int32_t nrow, double cutoff,
                         int32_t maxdim, int32_t mindim, int32_t exact_side, tnh_svd** out);
/* Shape of the result: the new link index has nsect sectors (charges in
 * ascending order, qn [nsect * nq], sect_dim [nsect]); pass NULL arrays to
 * only read nsect. truncerr is the discarded share of sum s^2. */
tnh_status tnh_svd_info(const tnh_svd* svd, int32_t* nsect, int32_t* nq, int32_t* qn,
                        int32_t* sect_dim, double* truncerr);
/* Work of the two Jacobi stages, for measurement: rounds (grid-wide steps)
 * of the float32 and the float64 stage, and the floating-point operations
 * their rotations execute (per column pair and row: 6 for the three dot
 * products, 6 for the two rotated entries; every group counted in every
 * round, so an upper bound when groups converge at different rounds).
 * Any pointer may be NULL. */
tnh_status tnh_svd_stats(const tnh_svd* svd, int32_t* rounds32, int32_t* rounds64, double* flops32,
                         double* flops64);
/* Copy the factors: U [rows..., c] (c In) and V [c, cols...] (c Out) with
 * caller-given layouts (DEVICE data), S DEVICE [sum of sect_dim] in sector
 * order, descending inside a sector (S may be NULL). T = U diag(S) V up to
 * the truncation. absorb = 1 returns U diag(S) in U, absorb = 2 returns
 * diag(S) V in V (the two ways a two-site update moves the orthogonality
 * centre), absorb = 0 neither. Synchronises the stream. */
tnh_status tnh_svd_get(tnh_svd* svd, tnh_tensor* U, double* S, tnh_tensor* V, int32_t absorb);
void tnh_svd_free(tnh_svd* svd);

/* ---- two-site DMRG sweeps (Sec. 7.2) ------------------------------------ */

typedef struct {
    int32_t nsweep;
    const int32_t* maxdim;   /* host [nsweep] */
    const double* cutoff;    /* host [nsweep] */
    int32_t mindim;
    int32_t krylov_dim;      /* max Lanczos matvecs per bond */
    double lanczos_tol;
    int32_t precision;       /* tnh_precision of the Lanczos matvecs */
    int32_t env_precision;   /* tnh_precision of theta and the environments */
    int32_t eigensolver;     /* 0: Lanczos (tnh_eigsolve), 1: Davidson (tnh_eigsolve_davidson) */
    int32_t energy_mode;     /* 0: FP64 energy and residual (one FP64 H_eff product) at every bond;
                              * 1: at the last bond of each sweep only, the other bonds report
                              *    the eigensolver's Ritz value (the sweep statistics and the
                              *    returned energy are always FP64). */
} tnh_sweep_params;

typedef struct {
    int32_t sweep;
    double energy;           /* eigenvalue at the last bond of the sweep */
    double resid;            /* its FP64 residual */
    double truncerr;         /* largest truncation error of the sweep */
    int32_t maxlink;         /* largest MPS link dimension after the sweep */
    int64_t matvecs;
    double seconds;
} tnh_sweep_stat;

/* Run the sweeps on the MPS (right-orthogonal from site 1 on; a normalised
 * product state is) with MPO tensors W[j] [wl, wr, s, s'] (same arrows as
 * above). start/done are the MPO link states selected by the left and right
 * boundaries. A sweep is a left-to-right pass over the bonds followed by a
 * right-to-left pass; energy is the eigenvalue at the last bond. When the
 * environments are built in a split precision (env_precision), the energy of
 * the final sweep is evaluated again with FP64 environments rebuilt from the
 * final MPS (right-orthogonal from site 2 on): <theta|H_eff|theta> at bond
 * (0, 1) in FP64, the state's exact energy to float64 rounding. The final
 * MPS stays on the device inside the context (tnh_dmrg_mps_*). Synchronous.
 * Errors: TNH_ERR_ARG for N < 2, an empty schedule, an unknown precision,
 * eigensolver or energy mode, tensors of the wrong rank or start/done
 * outside the boundary links; TNH_ERR_FLUX for an MPS block with another
 * flux than its site's or a boundary state in a forbidden block;
 * TNH_ERR_SHAPE, TNH_ERR_ARROW as for the contractions of a bond;
 * TNH_ERR_NUMERIC when a start vector is zero or not finite. */
tnh_status tnh_dmrg(tnh_ctx* ctx, int32_t N, const tnh_tensor* mpo, int64_t start,
                    int64_t done, const tnh_tensor* mps, const tnh_sweep_params* p,
                    double* energy, tnh_sweep_stat* stats);

/* DMRG beyond one MPO (Sec. 7.2):
 * - H is the sum of nterm MPOs, run as if summed (each term keeps its own
 *   boundary states; the driver works on their direct sum, see
 *   tnh_heff_plan_sum);
 * - northo previous states (MPS of N sites each, e.g. read back with
 *   tnh_dmrg_mps_get) each add weight * |P_i><P_i| to H, so the run finds
 *   the lowest state above them (excited states). Their data is read during
 *   the call only. The reported energy includes the penalty terms. */
typedef struct {
    int32_t nterm;              /* MPOs summed, >= 1 */
    const tnh_tensor* mpo;      /* [nterm * N]: term t, site j at t * N + j */
    const int64_t* start;       /* [nterm] left boundary link state of each term */
    const int64_t* done;        /* [nterm] right boundary link state of each term */
    int32_t northo;             /* previous states, >= 0 */
    const tnh_tensor* ortho;    /* [northo * N]: state i, site j at i * N + j */
    double weight;              /* energy penalty of every previous state */
} tnh_dmrg_problem;
tnh_status tnh_dmrg_ex(tnh_ctx* ctx, int32_t N, const tnh_dmrg_problem* prob,
                       const tnh_tensor* mps, const tnh_sweep_params* p, double* energy,
                       tnh_sweep_stat* stats);

/* The MPS left by the last tnh_dmrg / tnh_dmrg_ex on this context. After a
 * full sweep it is right-orthogonal from site 1 on, so it can start another
 * run as it is (checkpoint and resume). N = 0 before any run.
 * tnh_dmrg_mps_link: link j in 0..N (link j is the left index of site j,
 * link N the right index of site N-1): sector count, nq, QNs [nsect * nq]
 * and sector dims [nsect] (nq, qn and sect_dim may be NULL, e.g. to learn
 * nsect first). tnh_dmrg_mps_get copies site j into A (DEVICE data), whose
 * indices must be [link j (Out), site (Out), link j+1 (In)] with these
 * sectors; blocks of A that are not stored are zeroed, a stored block that A
 * lacks is TNH_ERR_SHAPE. Synchronises the stream. */
/* Checkpoints of the runs on this context (the paper writes MPS to HDF5
 * files, Sec. 10; here one binary file with a header). With path non-NULL,
 * later tnh_dmrg / tnh_dmrg_ex / tnh_dmrg_resume runs write to path, after
 * every `every` bond updates (0: only at sweep ends) and at the end of every
 * sweep but the last: the MPS, the environments valid before the next bond
 * (left ones up to it, right ones after it), the position (sweep, pass
 * 0 = left-to-right / 1 = right-to-left, step within the pass), the energy
 * and statistics so far. The file is written to path.tmp and renamed, so a
 * crash never leaves a half-written checkpoint. With stop_after > 0 a run
 * returns TNH_OK after that many bond updates, right after writing its
 * checkpoint (e.g. a batch job whose time slot ends); tnh_dmrg_position
 * tells where it stopped. path NULL, every 0, stop_after 0 turn it off.
 * Settings stay until changed. TNH_ERR_ARG for negative values. */
tnh_status tnh_dmrg_checkpoint(tnh_ctx* ctx, const char* path, int32_t every, int64_t stop_after);
/* Continue the run saved in the checkpoint file `path`: prob must be the
 * problem of the run that wrote it (same MPO terms and boundary states, same
 * previous states) and p the same sweep schedule (TNH_ERR_SHAPE when the
 * stored MPS or environments do not fit the MPO, TNH_ERR_ARG for a file
 * that is not a checkpoint or a schedule that ended before it). The stored
 * MPS and environments are loaded, the overlap environments of previous
 * states recomputed, and the schedule continues at the stored bond; stats
 * [p->nsweep] gets the completed sweeps' statistics from the file and the
 * rest from this run. The kernels are deterministic: an FP64 run resumed
 * this way reproduces the uninterrupted run. Synchronous. */
tnh_status tnh_dmrg_resume(tnh_ctx* ctx, int32_t N, const tnh_dmrg_problem* prob, const char* path,
                           const tnh_sweep_params* p, double* energy, tnh_sweep_stat* stats);
/* Where the last run on this context ended: the next bond (sweep, pass,
 * step) and finished = 1 when the schedule completed (then sweep = nsweep). */
tnh_status tnh_dmrg_position(tnh_ctx* ctx, int32_t* sweep, int32_t* pass, int32_t* step, int32_t* finished);

tnh_status tnh_dmrg_mps_size(tnh_ctx* ctx, int32_t* N);
tnh_status tnh_dmrg_mps_link(tnh_ctx* ctx, int32_t j, int32_t* nsect, int32_t* nq, int32_t* qn,
                             int32_t* sect_dim);
tnh_status tnh_dmrg_mps_get(tnh_ctx* ctx, int32_t j, tnh_tensor* A);

#ifdef __cplusplus
}
#endif
#endif /* TNH_H */
