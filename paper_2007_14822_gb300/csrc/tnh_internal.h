// Internal declarations shared by the translation units of libtnh.so.
#pragma once

#include <cuda_runtime.h>

#include <array>
#include <cstdint>
#include <cstdio>
#include <map>
#include <memory>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/tnh.h"

namespace tnh {

// ------------------------------------------------------------------ errors
struct Error : public std::exception {
    tnh_status code;
    std::string msg;
    Error(tnh_status c, std::string m) : code(c), msg(std::move(m)) {}
    const char* what() const noexcept override { return msg.c_str(); }
};

std::string strf(const char* fmt, ...);

#define TNH_FAIL(code, ...) throw ::tnh::Error((code), ::tnh::strf(__VA_ARGS__))
#define TNH_REQUIRE(cond, code, ...) \
    do { if (!(cond)) TNH_FAIL(code, __VA_ARGS__); } while (0)
#define CUDA_CHECK(x)                                                              \
    do {                                                                           \
        cudaError_t e_ = (x);                                                      \
        if (e_ != cudaSuccess)                                                     \
            TNH_FAIL(e_ == cudaErrorMemoryAllocation ? TNH_ERR_OOM : TNH_ERR_CUDA, \
                     "%s: %s (%s:%d)", #x, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)

// ---------------------------------------------------------- device memory
// Owning device buffer, freed on destruction. Inside a library call on a
// context (AllocScope) it comes from a per-device stream-ordered pool that
// keeps freed memory for reuse: allocation and release are ordered on the
// context's stream (cudaMallocFromPoolAsync / cudaFreeAsync), so the many
// short-lived buffers of a DMRG step cost no device-wide synchronisation.
// Outside a call it is a plain cudaMalloc / cudaFree.
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    cudaStream_t stream = nullptr;   // stream of a pooled allocation
    bool pooled = false;
    DevBuf() = default;
    explicit DevBuf(size_t n) { alloc(n); }
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    DevBuf(DevBuf&& o) noexcept : p(o.p), bytes(o.bytes), stream(o.stream), pooled(o.pooled) {
        o.p = nullptr;
        o.bytes = 0;
        o.pooled = false;
    }
    DevBuf& operator=(DevBuf&& o) noexcept {
        if (this != &o) {
            release();
            p = o.p;
            bytes = o.bytes;
            stream = o.stream;
            pooled = o.pooled;
            o.p = nullptr;
            o.bytes = 0;
            o.pooled = false;
        }
        return *this;
    }
    ~DevBuf() { release(); }
    void alloc(size_t n);
    void release();
    template <class T> T* as() const { return static_cast<T*>(p); }
};
// Pooled allocations on stream s for the lifetime of the scope (per thread).
struct AllocScope {
    bool prev_on;
    cudaStream_t prev_s;
    explicit AllocScope(cudaStream_t s);
    ~AllocScope();
};
// Return the pool's cached memory of the current device to the driver.
void trim_pool();
// Bytes of the current device's pool held by live allocations.
uint64_t pool_used_bytes();
// Test support: true for the allocation that an armed countdown selects
// (tnh_debug_fail_alloc); that allocation then fails with TNH_ERR_OOM.
bool alloc_fault_injected();

template <class T>
DevBuf upload(const std::vector<T>& v, cudaStream_t s) {
    DevBuf b(std::max<size_t>(v.size() * sizeof(T), 16));
    if (!v.empty())
        CUDA_CHECK(cudaMemcpyAsync(b.p, v.data(), v.size() * sizeof(T),
                                   cudaMemcpyHostToDevice, s));
    return b;
}

// ------------------------------------------------------------- structures
struct Index {
    int64_t label = 0;
    int nsect = 0, nq = 0, arrow = 1;
    std::vector<int> qn;    // nsect * nq
    std::vector<int> dim;   // nsect
    std::vector<int64_t> off;
    int64_t total = 0;
    void finish();
    int q(int s, int k) const { return qn[(size_t)s * nq + k]; }
    bool same_space(const Index& o) const { return nq == o.nq && qn == o.qn && dim == o.dim; }
    Index dag() const { Index r = *this; r.arrow = -arrow; return r; }
    Index relabel(int64_t l) const { Index r = *this; r.label = l; return r; }
};

// Host view of a block-sparse tensor: indices + block table + device data.
struct Layout {
    std::vector<Index> inds;
    std::vector<int> sect;      // nblocks * rank
    std::vector<int64_t> off;   // nblocks
    std::vector<int> flux;      // nq
    double* data = nullptr;
    int64_t size = 0;
    std::map<std::vector<int>, int> lookup;
    int rank() const { return (int)inds.size(); }
    int nblocks() const { return (int)off.size(); }
    int nq() const { return inds.empty() ? (int)flux.size() : inds[0].nq; }
    std::vector<int> key(int b) const {
        return std::vector<int>(sect.begin() + (size_t)b * rank(), sect.begin() + (size_t)(b + 1) * rank());
    }
    int bdim(int b, int i) const { return inds[i].dim[sect[(size_t)b * rank() + i]]; }
    int64_t belems(int b) const {
        int64_t n = 1;
        for (int i = 0; i < rank(); ++i) n *= bdim(b, i);
        return n;
    }
    int64_t packed_total() const;
    void build_lookup();
    int find(const std::vector<int>& k) const {
        auto it = lookup.find(k);
        return it == lookup.end() ? -1 : it->second;
    }
};

// A tensor that owns its device data.
struct OwnedTensor {
    Layout L;
    DevBuf buf;
};

Index parse_index(const tnh_index& in, const char* what);
Layout parse_tensor(const tnh_tensor* t, const char* what, bool need_data = true);
// Allowed blocks of the given indices at the given flux, lexicographic, packed.
Layout make_layout(const std::vector<Index>& inds, const std::vector<int>& flux);
std::vector<int> block_flux(const std::vector<Index>& inds, const int* key, int nq);
// Direct sum of tensors along the index positions in cat: those indices
// get the sectors of every term in turn, the other indices must agree, and
// the blocks of term t keep their keys with the cat sectors shifted past the
// earlier terms' (no block mixes two terms). The data of the terms is copied
// one after the other into buf (stream-ordered on s).
Layout direct_sum(const std::vector<Layout>& T, const std::vector<int>& cat, DevBuf& buf, cudaStream_t s);

// ------------------------------------------------------------------ context
struct Profiler;
struct Ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int num_sms = 0;
    std::string err;
    DevBuf d_flag;    // int[4]: [0] device error code written by bounded waits
    std::unique_ptr<Profiler> prof;
    // H_eff GEMM choices of the plan autotuner (tile policy and K split of S1,
    // then of S4) by shape signature; loaded from TNH_TUNE_CACHE once
    std::map<std::vector<int>, std::array<int, 5>> heff_tune;
    bool tune_loaded = false;
    // H_eff block-contraction strategy (0 combine, 1 block pairs) by shape
    std::map<std::vector<int>, int> heff_strategy;
    // the MPS left by the last DMRG run
    std::vector<OwnedTensor> mps;
    // checkpointing of DMRG runs (tnh_dmrg_checkpoint) and where the last
    // run ended: next bond (sweep, pass, step) and whether it finished
    std::string ckpt_path;
    int ckpt_every = 0;
    int64_t ckpt_stop = 0;
    int pos_sweep = 0, pos_pass = 0, pos_step = 0;
    bool pos_finished = false;
    ~Ctx();
};

// Check the device error flag (synchronises); throws TNH_ERR_TIMEOUT if set.
void check_device_flag(Ctx* ctx);

// -------------------------------------------------------- pack / unpack
// A piece copies a strided sub-tensor (row dims then col dims) into a 2-D
// region of a task matrix, or back.
constexpr int kMaxDims = 8;
struct Piece {
    int64_t src_off;          // element offset in the strided tensor
    int64_t strides[kMaxDims];
    int dims[kMaxDims];
    int nr, nc;               // number of row / col dims
    int rows, cols;           // products of the dims
    int task;                 // task whose matrix receives / provides it
    int row0, col0;           // position inside that task matrix
};
struct Chunk {
    int piece;
    int start;                // first element (row-major over rows x cols)
    int count;
};
void make_chunks(const std::vector<Piece>& pieces, std::vector<Chunk>& chunks, int per_chunk = 4096);

// Operand formats
enum class Fmt { F64, BF16T };  // plain float64 [rows][ld] / bf16 split tiles

// Task geometry of one packed operand (per task).
struct OpGeom {
    int64_t base;   // F64: element offset; BF16T: tile offset
    int ld;         // F64: row pitch (padded K); BF16T: tiles along K
};

void launch_pack_f64(const Piece* d_pieces, const Chunk* d_chunks, int nchunks,
                     const OpGeom* d_geom, const double* src, double* dst, cudaStream_t s);
void launch_pack_bf16(const Piece* d_pieces, const Chunk* d_chunks, int nchunks,
                      const OpGeom* d_geom, const double* src, uint16_t* dst, int planes,
                      cudaStream_t s);
// Ct region of task -> strided destination (overwrite).
void launch_unpack(const Piece* d_pieces, const Chunk* d_chunks, int nchunks,
                   const int64_t* d_cbase, const int* d_ldc, const double* Ct, double* dst,
                   cudaStream_t s);

// ---------------------------------------------------------------- GEMMs
// C_t[M][ldc] = A_t[M][K] * B_t[N][K]^T for every task t (both K-major).
struct GemmTask {
    int M, N, K;
    int mt, nt, kt;          // tiles along M, N, K for the launch's tile shape
    int64_t a_base, b_base;  // F64: element offsets; BF16T: tile offsets
    int lda, ldb;            // F64 only: padded K pitch
    int64_t c_base;
    int ldc;
    int tile0;               // prefix sum of mt * nt
    int use_roff;            // 1: row m of C starts at row_off[roff + m] (scatter epilogue)
    int c_f32;               // tcgen05 GEMM only: C is float32 (else float64)
    int64_t roff;
    int kstride;             // tcgen05 GEMM: operand tiles per tile row (0: kt); a K-split sub-task
                             // covers kt k-blocks starting at its a_base / b_base
    int tn;                  // tcgen05 GEMM: N tile width 128, 64 or 32 (0: 128); B is packed in
                             // 128-row tiles, a narrower N tile reads a slice of one
};
void launch_gemm_f64(const GemmTask* d_tasks, int ntasks, int total_tiles, const double* A,
                     const double* B, double* C, cudaStream_t s, const int64_t* row_off = nullptr);
// tcgen05 split-bf16 GEMM; planes in {1,2,3}; err is a device int flag.
void launch_gemm_tc(const GemmTask* d_tasks, int ntasks, int total_tiles, const uint16_t* A,
                    const uint16_t* B, double* C, int planes, int num_sms, int* err,
                    cudaStream_t s, const int64_t* row_off = nullptr);
// K-split reduction: out = sum over S float32 partial slabs [S][M][N]
// (float32 partials summed in float32, float64 ones in float64, slab order),
// written to float32 or float64 rows.
struct SplitRed {
    int M, N, S;
    int use_roff, out_f32;
    int ldc;
    int64_t part;    // first element of the partial slabs
    int64_t roff;    // use_roff: row m starts at row_off[roff + m]
    int64_t c_base;  // else: row m starts at c_base + m * ldc
    int64_t e0;      // prefix of M * N over the reductions of one launch
};
// One block of the reduction launch: rows [m0, m1) of reduction red.
struct RedBlock { int red, m0, m1; };
// The blocks of a list of reductions, about 2048 elements each.
std::vector<RedBlock> reduction_blocks(const std::vector<SplitRed>& reds);
void launch_splitk_reduce(const SplitRed* d_reds, const RedBlock* d_blocks, int nblocks, const float* part,
                          void* out, const int64_t* row_off, cudaStream_t s);
// The same with float64 partial slabs (K-split FP64 GEMMs).
void launch_splitk_reduce(const SplitRed* d_reds, const RedBlock* d_blocks, int nblocks, const double* part,
                          void* out, const int64_t* row_off, cudaStream_t s);
constexpr int kF64TileM = 64, kF64TileN = 64, kF64TileK = 16;
constexpr int kTcTileM = 128, kTcTileN = 128, kTcTileK = 64;
constexpr int kTcTileElems = kTcTileM * kTcTileK;   // 8192 bf16 per plane tile

int planes_of(tnh_precision p);

// ------------------------------------------------------ contraction plan
struct ContractPlan {
    // host
    std::vector<GemmTask> tasks_f64, tasks_tc;
    std::vector<Piece> packA, packB, unpackC;
    std::vector<int64_t> cbase;
    std::vector<int> ldc;
    int ntiles_f64 = 0, ntiles_tc = 0;
    int64_t a_elems_f64 = 0, b_elems_f64 = 0, a_tiles = 0, b_tiles = 0, c_elems = 0;
    int64_t c_total = 0;  // elements of the output tensor
    double flops = 0.0;
    // device
    DevBuf d_packA, d_packB, d_unpack, d_chA, d_chB, d_chC;
    int nchA = 0, nchB = 0, nchC = 0;
    DevBuf d_geomA_f64, d_geomB_f64, d_geomA_tc, d_geomB_tc;
    DevBuf d_tasks_f64, d_tasks_tc, d_cbase, d_ldc;
};

// Label-matched plan for C = A * B (validates labels and arrows).
std::unique_ptr<ContractPlan> plan_contract(const Layout& A, const Layout& B, const Layout& C,
                                            cudaStream_t s);
// Flops (2 M N K summed over block pairs) of the contraction A * B.
double contract_flops(const Layout& A, const Layout& B);
// Workspace big enough for one execution of the plan in a precision.
struct Workspace {
    DevBuf a, b, c;
    void ensure(DevBuf& buf, size_t bytes);
};
// Execute: C.data = A.data * B.data (pack, GEMM, unpack).
void run_contract(Ctx* ctx, const ContractPlan& P, const double* A, const double* B, double* C,
                  tnh_precision prec, Workspace& ws);

}  // namespace tnh
