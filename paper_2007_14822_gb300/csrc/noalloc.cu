// Dense float64 contraction that allocates nothing.
//
// Some callers cannot allocate device memory during their work: code that
// runs with a memory budget fixed up front (a serving process that reserved
// all device memory at start-up, a real-time loop where cudaMalloc/cudaFree
// would stall or synchronise, or a framework that hands out memory only from
// its own pool). tnh_contract allocates its packing workspace on every call,
// so it does not suit them. This file gives them tnh_contract_dense_noalloc:
// the same labelled contraction for dense tensors, computed by the same
// kernels (operand packing, FP64 GEMM, result scatter), with every piece of
// scratch it needs -- the packed operands, the GEMM result and the launch
// descriptors -- taken from one static device array of fixed size. The
// descriptors are written into that array by a small kernel that receives
// them as launch arguments, so no host buffer is copied either.
//
// The array is a file-scope __device__ variable: every GPU that loads the
// library holds kScratchBytes of it until the process exits. Host code only
// sees a stand-in for its name, so the device address is looked up once per
// device with cudaGetSymbolAddress (with that device current) and cached.
#include <cstring>
#include <mutex>

#include "tnh_guard.h"
#include "tnh_internal.h"

// The scratch: 16 MiB of device memory per GPU, shared by every call.
static constexpr size_t kScratchBytes = size_t(16) << 20;
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

namespace tnh {

namespace {

constexpr int kMaxDevices = 64;
constexpr int kChunk = 8192;                        // elements per pack / unpack block
constexpr int kMaxChunks = 2048;                    // descriptor room per operand

__device__ __forceinline__ int nchunks_dev(int64_t n) { return (int)((n + kChunk - 1) / kChunk); }

std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of g_scratch on `device` (which must be current). The first
// call per device performs the lookup.
void* scratch_address(int device) {
    std::lock_guard<std::mutex> lock(g_mu);
    TNH_REQUIRE(device >= 0 && device < kMaxDevices, TNH_ERR_ARG, "noalloc: device %d out of range", device);
    if (!g_scratch_ptr[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        TNH_REQUIRE(e == cudaSuccess && p != nullptr, TNH_ERR_CUDA,
                    "noalloc: cudaGetSymbolAddress of the static scratch failed: %s", cudaGetErrorString(e));
        g_scratch_ptr[device] = p;
    }
    return g_scratch_ptr[device];
}

struct Dense {
    int rank;
    int64_t dim[kMaxDims], label[kMaxDims], stride[kMaxDims];
    int arrow[kMaxDims];
    double* data;
    int64_t off;
};

Dense view(const tnh_tensor* t, const char* what) {
    TNH_REQUIRE(t != nullptr, TNH_ERR_ARG, "noalloc: %s is NULL", what);
    TNH_REQUIRE(t->rank >= 0 && t->rank <= kMaxDims, TNH_ERR_ARG, "noalloc: %s rank %d", what, t->rank);
    TNH_REQUIRE(t->nblocks == 1 && t->block_off != nullptr, TNH_ERR_ARG,
                "noalloc: %s must be dense (exactly one stored block)", what);
    Dense d{};
    d.rank = t->rank;
    d.data = t->data;
    d.off = t->block_off[0];
    TNH_REQUIRE(d.data != nullptr, TNH_ERR_ARG, "noalloc: %s data is NULL", what);
    int64_t n = 1;
    for (int i = 0; i < t->rank; ++i) {
        const tnh_index& ix = t->inds[i];
        TNH_REQUIRE(ix.nsect == 1 && ix.sect_dim && ix.sect_dim[0] >= 1, TNH_ERR_ARG,
                    "noalloc: %s index %d must have one sector", what, i);
        TNH_REQUIRE(t->block_sect == nullptr || t->block_sect[i] == 0, TNH_ERR_SHAPE,
                    "noalloc: %s block sector out of range", what);
        d.dim[i] = ix.sect_dim[0];
        d.label[i] = ix.label;
        d.arrow[i] = ix.arrow;
        // every tensor that fits the scratch has far fewer elements than this
        TNH_REQUIRE(n <= (int64_t(1) << 40) / d.dim[i], TNH_ERR_ARG, "noalloc: %s has too many elements", what);
        n *= d.dim[i];
    }
    for (int i = 0; i < d.rank; ++i)
        for (int j = 0; j < i; ++j)
            TNH_REQUIRE(d.label[i] != d.label[j], TNH_ERR_LABEL, "noalloc: repeated label %lld in %s",
                        (long long)d.label[i], what);
    int64_t st = 1;
    for (int i = d.rank - 1; i >= 0; --i) {
        d.stride[i] = st;
        st *= d.dim[i];
    }
    TNH_REQUIRE(d.off >= 0 && d.off + n <= t->size, TNH_ERR_SHAPE, "noalloc: %s block outside its data", what);
    return d;
}

int find_label(const Dense& t, int64_t l) {
    for (int i = 0; i < t.rank; ++i)
        if (t.label[i] == l) return i;
    return -1;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

int nchunks(int64_t n) { return (int)((n + kChunk - 1) / kChunk); }

// Launch descriptors of one call: the fixed part travels as a kernel
// argument, the chunk lists (kChunk elements each) are generated here.
struct DescHead {
    Piece p[3];
    OpGeom ga, gb;
    GemmTask task;
    int64_t cbase;
    int ldc;
    int64_t n[3];   // elements of packed A, packed B, the result
};
struct Desc {
    DescHead h;
    Chunk ch[3][kMaxChunks];
};

__global__ void write_desc_kernel(DescHead h, Desc* __restrict__ d) {
    if (threadIdx.x == 0 && blockIdx.x == 0) d->h = h;
    for (int q = 0; q < 3; ++q) {
        const int nc = nchunks_dev(h.n[q]);
        for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += gridDim.x * blockDim.x) {
            const int64_t s0 = (int64_t)c * kChunk;
            d->ch[q][c] = Chunk{0, (int)s0, (int)(h.n[q] - s0 < kChunk ? h.n[q] - s0 : (int64_t)kChunk)};
        }
    }
}

}  // namespace

}  // namespace tnh

using namespace tnh;

extern "C" tnh_status tnh_contract_dense_noalloc(tnh_ctx* ctx, const tnh_tensor* A, const tnh_tensor* B,
                                                 tnh_tensor* C) {
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    return guard(c, [&] {
        TNH_REQUIRE(c, TNH_ERR_ARG, "noalloc: ctx is NULL");
        CUDA_CHECK(cudaSetDevice(c->device));
        unsigned char* base = static_cast<unsigned char*>(scratch_address(c->device));
        const Dense a = view(A, "A"), b = view(B, "B"), o = view(C, "C");
        // label matching: contracted = labels of A also in B
        int ia[kMaxDims], ib[kMaxDims], fa[kMaxDims], fb[kMaxDims];
        int nc = 0, nfa = 0, nfb = 0;
        for (int i = 0; i < a.rank; ++i) {
            int j = find_label(b, a.label[i]);
            if (j >= 0) {
                TNH_REQUIRE(a.dim[i] == b.dim[j], TNH_ERR_SHAPE, "noalloc: contracted label %lld dims differ",
                            (long long)a.label[i]);
                TNH_REQUIRE(a.arrow[i] != b.arrow[j], TNH_ERR_ARROW, "noalloc: contracted label %lld has equal arrows",
                            (long long)a.label[i]);
                ia[nc] = i;
                ib[nc++] = j;
            } else {
                fa[nfa++] = i;
            }
        }
        for (int j = 0; j < b.rank; ++j)
            if (find_label(a, b.label[j]) < 0) fb[nfb++] = j;
        TNH_REQUIRE(nfa + nfb == o.rank, TNH_ERR_LABEL, "noalloc: C has %d indices, the product %d", o.rank,
                    nfa + nfb);
        int64_t M = 1, N = 1, K = 1;
        Piece pa{}, pb{}, pc{};
        pa.src_off = a.off;
        pa.nr = nfa;
        pa.nc = nc;
        pb.src_off = b.off;
        pb.nr = nfb;
        pb.nc = nc;
        pc.src_off = o.off;
        pc.nr = nfa;
        pc.nc = nfb;
        for (int q = 0; q < nfa; ++q) {
            int k = find_label(o, a.label[fa[q]]);
            TNH_REQUIRE(k >= 0, TNH_ERR_LABEL, "noalloc: free label %lld of A not in C", (long long)a.label[fa[q]]);
            TNH_REQUIRE(o.dim[k] == a.dim[fa[q]] && o.arrow[k] == a.arrow[fa[q]], TNH_ERR_SHAPE,
                        "noalloc: C index for label %lld differs from A's (dimension or arrow)",
                        (long long)a.label[fa[q]]);
            pa.dims[q] = pc.dims[q] = (int)a.dim[fa[q]];
            pa.strides[q] = a.stride[fa[q]];
            pc.strides[q] = o.stride[k];
            M *= a.dim[fa[q]];
        }
        for (int q = 0; q < nfb; ++q) {
            int k = find_label(o, b.label[fb[q]]);
            TNH_REQUIRE(k >= 0, TNH_ERR_LABEL, "noalloc: free label %lld of B not in C", (long long)b.label[fb[q]]);
            TNH_REQUIRE(o.dim[k] == b.dim[fb[q]] && o.arrow[k] == b.arrow[fb[q]], TNH_ERR_SHAPE,
                        "noalloc: C index for label %lld differs from B's (dimension or arrow)",
                        (long long)b.label[fb[q]]);
            pb.dims[q] = pc.dims[nfa + q] = (int)b.dim[fb[q]];
            pb.strides[q] = b.stride[fb[q]];
            pc.strides[nfa + q] = o.stride[k];
            N *= b.dim[fb[q]];
        }
        for (int q = 0; q < nc; ++q) {
            pa.dims[nfa + q] = pb.dims[nfb + q] = (int)a.dim[ia[q]];
            pa.strides[nfa + q] = a.stride[ia[q]];
            pb.strides[nfb + q] = b.stride[ib[q]];
            K *= a.dim[ia[q]];
        }
        // the operands and the result must fit the scratch before any size is narrowed to int
        const int64_t lim = (int64_t)(kScratchBytes / sizeof(double));
        TNH_REQUIRE(M <= lim / K && N <= lim / K && M <= lim / N, TNH_ERR_ARG,
                    "noalloc: this contraction (M %lld, N %lld, K %lld) exceeds the static maximum of %zu bytes "
                    "of scratch (use tnh_contract for larger tensors)", (long long)M, (long long)N, (long long)K,
                    kScratchBytes);
        pa.rows = pc.rows = (int)M;
        pb.rows = pc.cols = (int)N;
        pa.cols = pb.cols = (int)K;
        GemmTask g{};
        g.M = (int)M;
        g.N = (int)N;
        g.K = (int)K;
        g.mt = (int)((M + kF64TileM - 1) / kF64TileM);
        g.nt = (int)((N + kF64TileN - 1) / kF64TileN);
        g.kt = (int)((K + kF64TileK - 1) / kF64TileK);
        g.lda = g.ldb = g.kt * kF64TileK;
        g.ldc = (int)N;
        // scratch layout: descriptors | packed A | packed B | GEMM result
        const size_t a_elems = (size_t)g.mt * kF64TileM * g.lda, b_elems = (size_t)g.nt * kF64TileN * g.ldb;
        const size_t c_elems = (size_t)M * N;
        const size_t desc_bytes = align256(sizeof(Desc));
        const size_t off_a = desc_bytes, off_b = off_a + align256(a_elems * 8), off_c = off_b + align256(b_elems * 8);
        const size_t need = off_c + align256(c_elems * 8);
        TNH_REQUIRE(need <= kScratchBytes, TNH_ERR_ARG,
                    "noalloc: this contraction needs %zu bytes of scratch; the static maximum is %zu bytes "
                    "(use tnh_contract for larger tensors)", need, kScratchBytes);
        const int64_t na = M * K, nb = N * K, ncc = M * N;
        TNH_REQUIRE((na + kChunk - 1) / kChunk <= kMaxChunks && (nb + kChunk - 1) / kChunk <= kMaxChunks &&
                        (ncc + kChunk - 1) / kChunk <= kMaxChunks, TNH_ERR_ARG,
                    "noalloc: operand too large for the static descriptor area");
        DescHead h{};
        h.p[0] = pa;
        h.p[1] = pb;
        h.p[2] = pc;
        h.ga = OpGeom{0, g.lda};
        h.gb = OpGeom{0, g.ldb};
        h.task = g;
        h.cbase = 0;
        h.ldc = (int)N;
        h.n[0] = na;
        h.n[1] = nb;
        h.n[2] = ncc;
        const int nca = nchunks(na), ncb = nchunks(nb), ncu = nchunks(ncc);
        Desc* d = reinterpret_cast<Desc*>(base);
        cudaStream_t s = c->stream;
        // the call reuses the array: write the descriptors, zero the padded operand space
        write_desc_kernel<<<8, 256, 0, s>>>(h, d);
        double* pA = reinterpret_cast<double*>(base + off_a);
        double* pB = reinterpret_cast<double*>(base + off_b);
        double* pC = reinterpret_cast<double*>(base + off_c);
        CUDA_CHECK(cudaMemsetAsync(pA, 0, a_elems * 8, s));
        CUDA_CHECK(cudaMemsetAsync(pB, 0, b_elems * 8, s));
        launch_pack_f64(&d->h.p[0], d->ch[0], nca, &d->h.ga, a.data, pA, s);
        launch_pack_f64(&d->h.p[1], d->ch[1], ncb, &d->h.gb, b.data, pB, s);
        launch_gemm_f64(&d->h.task, 1, g.mt * g.nt, pA, pB, pC, s);
        launch_unpack(&d->h.p[2], d->ch[2], ncu, &d->h.cbase, &d->h.ldc, pC, o.data, s);
        CUDA_CHECK(cudaGetLastError());
    });
}
