// Context, error handling, index/tensor parsing and the layout helper.
// Indices carry QN sectors and an arrow (Sec. 8.2); a tensor stores only
// the blocks whose flux matches its own (Sec. 8.3), packed one after the
// other in block-sparse storage (Sec. 6, Sec. 9.2).
#include <algorithm>
#include <cstdarg>
#include <cstring>
#include <map>
#include <mutex>
#include <numeric>

#include "prof.h"
#include "tnh_guard.h"
#include "tnh_internal.h"

namespace tnh {

std::string strf(const char* fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    return buf;
}

thread_local std::string g_last_error;

void set_error(Ctx* ctx, const std::string& m) {
    if (ctx) ctx->err = m;
    g_last_error = m;
}

namespace {

thread_local bool t_pool_on = false;
thread_local cudaStream_t t_pool_stream = nullptr;
std::mutex g_pool_mu;
std::map<int, cudaMemPool_t> g_pools;

// The library's pool on the current device: device memory, kept after
// release (release threshold: no limit) until trim_pool.
cudaMemPool_t device_pool() {
    int dev = 0;
    CUDA_CHECK(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_pool_mu);
    auto it = g_pools.find(dev);
    if (it != g_pools.end()) return it->second;
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    CUDA_CHECK(cudaMemPoolCreate(&pool, &props));
    uint64_t keep = ~0ull;
    CUDA_CHECK(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep));
    g_pools[dev] = pool;
    return pool;
}

}  // namespace

AllocScope::AllocScope(cudaStream_t s) : prev_on(t_pool_on), prev_s(t_pool_stream) {
    t_pool_on = true;
    t_pool_stream = s;
}

AllocScope::~AllocScope() {
    t_pool_on = prev_on;
    t_pool_stream = prev_s;
}

uint64_t pool_used_bytes() {
    uint64_t v = 0;
    CUDA_CHECK(cudaMemPoolGetAttribute(device_pool(), cudaMemPoolAttrUsedMemCurrent, &v));
    return v;
}

void trim_pool() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return;
    std::lock_guard<std::mutex> lk(g_pool_mu);
    auto it = g_pools.find(dev);
    if (it != g_pools.end()) cudaMemPoolTrimTo(it->second, 0);
}

void DevBuf::alloc(size_t n) {
    release();
    if (n == 0) n = 16;
    if (alloc_fault_injected())
        TNH_FAIL(TNH_ERR_OOM, "device allocation of %zu bytes: injected failure (tnh_debug_fail_alloc)", n);
    cudaError_t e;
    if (t_pool_on) {
        e = cudaMallocFromPoolAsync(&p, n, device_pool(), t_pool_stream);
        pooled = e == cudaSuccess;
        stream = t_pool_stream;
    } else {
        e = cudaMalloc(&p, n);
        pooled = false;
    }
    if (e != cudaSuccess) {
        p = nullptr;
        pooled = false;
        cudaGetLastError();
        TNH_FAIL(e == cudaErrorMemoryAllocation ? TNH_ERR_OOM : TNH_ERR_CUDA,
                 "device allocation of %zu bytes: %s", n, cudaGetErrorString(e));
    }
    bytes = n;
}

void DevBuf::release() {
    if (p) {
        if (pooled) cudaFreeAsync(p, stream);
        else cudaFree(p);
    }
    p = nullptr;
    bytes = 0;
    pooled = false;
}

void Workspace::ensure(DevBuf& buf, size_t bytes) {
    if (buf.bytes < bytes) buf.alloc(bytes);
}

int planes_of(tnh_precision p) {
    switch (p) {
        case TNH_BF16x6: return 3;
        case TNH_BF16x3: return 2;
        case TNH_BF16: return 1;
        default: return 0;
    }
}

void Index::finish() {
    off.assign(nsect, 0);
    total = 0;
    for (int s = 0; s < nsect; ++s) { off[s] = total; total += dim[s]; }
}

Index parse_index(const tnh_index& in, const char* what) {
    TNH_REQUIRE(in.nsect >= 1, TNH_ERR_ARG, "%s: index with nsect=%d", what, in.nsect);
    TNH_REQUIRE(in.nq >= 0 && in.nq <= 4, TNH_ERR_ARG, "%s: nq=%d out of 0..4", what, in.nq);
    TNH_REQUIRE(in.sect_dim != nullptr, TNH_ERR_ARG, "%s: sect_dim is NULL", what);
    TNH_REQUIRE(in.nq == 0 || in.qn != nullptr, TNH_ERR_ARG, "%s: qn is NULL", what);
    TNH_REQUIRE(in.arrow == 1 || in.arrow == -1, TNH_ERR_ARG, "%s: arrow must be +1/-1", what);
    Index r;
    r.label = in.label;
    r.nsect = in.nsect;
    r.nq = in.nq;
    r.arrow = in.arrow;
    r.dim.assign(in.sect_dim, in.sect_dim + in.nsect);
    if (in.nq) r.qn.assign(in.qn, in.qn + (size_t)in.nsect * in.nq);
    for (int d : r.dim) TNH_REQUIRE(d >= 1, TNH_ERR_SHAPE, "%s: sector dim %d < 1", what, d);
    r.finish();
    return r;
}

std::vector<int> block_flux(const std::vector<Index>& inds, const int* key, int nq) {
    std::vector<int> f(nq, 0);
    for (size_t i = 0; i < inds.size(); ++i)
        for (int k = 0; k < nq; ++k) f[k] += inds[i].arrow * inds[i].q(key[i], k);
    return f;
}

int64_t Layout::packed_total() const {
    int64_t t = 0;
    for (int b = 0; b < nblocks(); ++b) t += belems(b);
    return t;
}

void Layout::build_lookup() {
    lookup.clear();
    for (int b = 0; b < nblocks(); ++b) lookup[key(b)] = b;
}

Layout parse_tensor(const tnh_tensor* t, const char* what, bool need_data) {
    TNH_REQUIRE(t != nullptr, TNH_ERR_ARG, "%s: tensor is NULL", what);
    TNH_REQUIRE(t->rank >= 0 && t->rank <= kMaxDims, TNH_ERR_ARG, "%s: rank %d", what, t->rank);
    TNH_REQUIRE(t->rank == 0 || t->inds != nullptr, TNH_ERR_ARG, "%s: inds NULL", what);
    TNH_REQUIRE(t->nblocks >= 0, TNH_ERR_ARG, "%s: nblocks %d", what, t->nblocks);
    Layout L;
    for (int i = 0; i < t->rank; ++i) L.inds.push_back(parse_index(t->inds[i], what));
    int nq = L.inds.empty() ? 0 : L.inds[0].nq;
    for (auto& ix : L.inds)
        TNH_REQUIRE(ix.nq == nq, TNH_ERR_ARG, "%s: indices disagree on nq", what);
    if (t->nblocks) {
        TNH_REQUIRE(t->rank == 0 || t->block_sect, TNH_ERR_ARG, "%s: block_sect NULL", what);
        TNH_REQUIRE(t->block_off, TNH_ERR_ARG, "%s: block_off NULL", what);
    }
    L.sect.assign(t->block_sect, t->block_sect + (size_t)t->nblocks * t->rank);
    L.off.assign(t->block_off, t->block_off + t->nblocks);
    L.data = t->data;
    L.size = t->size;
    if (need_data) TNH_REQUIRE(L.data != nullptr || t->nblocks == 0, TNH_ERR_ARG, "%s: data NULL", what);
    L.flux.assign(nq, 0);
    for (int b = 0; b < t->nblocks; ++b) {
        for (int i = 0; i < t->rank; ++i) {
            int s = L.sect[(size_t)b * t->rank + i];
            TNH_REQUIRE(s >= 0 && s < L.inds[i].nsect, TNH_ERR_SHAPE,
                        "%s: block %d sector %d of index %d out of range", what, b, s, i);
        }
        auto f = block_flux(L.inds, &L.sect[(size_t)b * t->rank], nq);
        if (b == 0) L.flux = f;
        TNH_REQUIRE(f == L.flux, TNH_ERR_FLUX, "%s: block %d has a different flux", what, b);
        TNH_REQUIRE(L.off[b] >= 0 && L.off[b] + L.belems(b) <= t->size, TNH_ERR_SHAPE,
                    "%s: block %d [%lld, +%lld) outside size %lld", what, b,
                    (long long)L.off[b], (long long)L.belems(b), (long long)t->size);
    }
    L.build_lookup();
    TNH_REQUIRE((int)L.lookup.size() == t->nblocks, TNH_ERR_SHAPE, "%s: repeated block", what);
    return L;
}

Layout make_layout(const std::vector<Index>& inds, const std::vector<int>& flux) {
    Layout L;
    L.inds = inds;
    L.flux = flux;
    const int r = (int)inds.size();
    const int nq = (int)flux.size();
    int64_t off = 0;
    if (r == 0) {   // a scalar: one block when the flux is zero
        bool zero = true;
        for (int f : flux) zero &= f == 0;
        if (zero) {
            L.off.push_back(0);
            off = 1;
        }
        L.size = off;
        L.build_lookup();
        return L;
    }
    // Lexicographic tuples (last index fastest): an odometer over the first
    // r - 1 indices; for each prefix the flux rule fixes the charge the last
    // index must carry, and its sectors with that charge complete the tuple
    // in increasing order.
    const Index& last = inds[r - 1];
    std::map<std::vector<int>, std::vector<int>> by_q;
    for (int sct = 0; sct < last.nsect; ++sct) {
        std::vector<int> q(nq);
        for (int k = 0; k < nq; ++k) q[k] = last.q(sct, k);
        by_q[q].push_back(sct);
    }
    std::vector<int> key(r, 0), need(nq);
    while (true) {
        for (int k = 0; k < nq; ++k) {
            int f = 0;
            for (int i = 0; i < r - 1; ++i) f += inds[i].arrow * inds[i].q(key[i], k);
            need[k] = last.arrow * (flux[k] - f);
        }
        auto it = by_q.find(need);
        if (it != by_q.end()) {
            int64_t n0 = 1;
            for (int i = 0; i < r - 1; ++i) n0 *= inds[i].dim[key[i]];
            for (int sct : it->second) {
                key[r - 1] = sct;
                L.sect.insert(L.sect.end(), key.begin(), key.end());
                L.off.push_back(off);
                off += n0 * last.dim[sct];
            }
            key[r - 1] = 0;
        }
        int i = r - 2;
        while (i >= 0 && ++key[i] == inds[i].nsect) { key[i] = 0; --i; }
        if (i < 0) break;
    }
    L.size = off;
    L.build_lookup();
    return L;
}

Layout direct_sum(const std::vector<Layout>& T, const std::vector<int>& cat, DevBuf& buf, cudaStream_t s) {
    TNH_REQUIRE(!T.empty(), TNH_ERR_ARG, "direct sum: no terms");
    const int r = T[0].rank();
    std::vector<char> joined(r, 0);
    for (int i : cat) {
        TNH_REQUIRE(i >= 0 && i < r, TNH_ERR_ARG, "direct sum: index position %d out of range", i);
        joined[i] = 1;
    }
    Layout S;
    S.inds = T[0].inds;
    for (size_t t = 1; t < T.size(); ++t) {
        TNH_REQUIRE(T[t].rank() == r, TNH_ERR_SHAPE, "direct sum: term %zu has rank %d, not %d", t, T[t].rank(), r);
        for (int i = 0; i < r; ++i) {
            const Index& a = T[t].inds[i];
            Index& d = S.inds[i];
            TNH_REQUIRE(a.arrow == d.arrow, TNH_ERR_ARROW, "direct sum: term %zu index %d has another arrow", t, i);
            TNH_REQUIRE(a.nq == d.nq, TNH_ERR_SHAPE, "direct sum: term %zu index %d has another nq", t, i);
            if (joined[i]) {
                d.nsect += a.nsect;
                d.qn.insert(d.qn.end(), a.qn.begin(), a.qn.end());
                d.dim.insert(d.dim.end(), a.dim.begin(), a.dim.end());
            } else {
                TNH_REQUIRE(a.same_space(T[0].inds[i]), TNH_ERR_SHAPE,
                            "direct sum: term %zu index %d differs from term 0's", t, i);
            }
        }
    }
    for (auto& ix : S.inds) ix.finish();
    S.flux = T[0].flux;
    std::vector<int> shift(r, 0);
    std::vector<int64_t> base(T.size(), 0);
    int64_t total = 0;
    bool have_flux = false;
    for (size_t t = 0; t < T.size(); ++t) {
        const Layout& L = T[t];
        if (L.nblocks()) {
            if (have_flux)
                TNH_REQUIRE(L.flux == S.flux, TNH_ERR_FLUX, "direct sum: term %zu has another flux", t);
            S.flux = L.flux;
            have_flux = true;
        }
        base[t] = total;
        for (int b = 0; b < L.nblocks(); ++b) {
            std::vector<int> k = L.key(b);
            for (int i = 0; i < r; ++i) k[i] += shift[i];
            S.sect.insert(S.sect.end(), k.begin(), k.end());
            S.off.push_back(total + L.off[b]);
        }
        total += L.size;
        for (int i = 0; i < r; ++i)
            if (joined[i]) shift[i] += L.inds[i].nsect;
    }
    S.size = total;
    buf.alloc((size_t)std::max<int64_t>(total, 1) * sizeof(double));
    for (size_t t = 0; t < T.size(); ++t)
        if (T[t].size > 0 && T[t].data)
            CUDA_CHECK(cudaMemcpyAsync(buf.as<double>() + base[t], T[t].data, (size_t)T[t].size * sizeof(double),
                                       cudaMemcpyDeviceToDevice, s));
    S.data = buf.as<double>();
    S.build_lookup();
    return S;
}

void make_chunks(const std::vector<Piece>& pieces, std::vector<Chunk>& chunks, int per_chunk) {
    chunks.clear();
    for (int p = 0; p < (int)pieces.size(); ++p) {
        int64_t n = (int64_t)pieces[p].rows * pieces[p].cols;
        for (int64_t s = 0; s < n; s += per_chunk)
            chunks.push_back(Chunk{p, (int)s, (int)std::min<int64_t>(per_chunk, n - s)});
    }
}

Ctx::~Ctx() {
    if (prof && active_profiler() == prof.get()) set_active_profiler(nullptr);
}

void check_device_flag(Ctx* ctx) {
    int h[4] = {0, 0, 0, 0};
    CUDA_CHECK(cudaMemcpyAsync(h, ctx->d_flag.p, sizeof h, cudaMemcpyDeviceToHost, ctx->stream));
    CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
    if (h[0]) {
        CUDA_CHECK(cudaMemsetAsync(ctx->d_flag.p, 0, sizeof h, ctx->stream));
        TNH_FAIL(TNH_ERR_TIMEOUT, "device wait gave up (code %d, site %d, block %d)", h[0], h[1], h[2]);
    }
}

}  // namespace tnh

using namespace tnh;

extern "C" {

tnh_status tnh_create(tnh_ctx** out, int device, void* stream) {
    return guard(nullptr, [&] {
        TNH_REQUIRE(out != nullptr, TNH_ERR_ARG, "tnh_create: out is NULL");
        int n = 0;
        CUDA_CHECK(cudaGetDeviceCount(&n));
        TNH_REQUIRE(device >= 0 && device < n, TNH_ERR_ARG, "tnh_create: device %d of %d", device, n);
        CUDA_CHECK(cudaSetDevice(device));
        int major = 0, minor = 0;
        CUDA_CHECK(cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, device));
        CUDA_CHECK(cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, device));
        TNH_REQUIRE(major == 10 && minor == 3, TNH_ERR_CUDA,
                    "tnh_create: device %d is sm_%d%d; this library is built for sm_103a only",
                    device, major, minor);
        auto* c = new Ctx();
        c->device = device;
        c->stream = (cudaStream_t)stream;
        cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
        try {
            c->d_flag.alloc(16);
            CUDA_CHECK(cudaMemsetAsync(c->d_flag.p, 0, 16, c->stream));
        } catch (...) {
            delete c;
            throw;
        }
        *out = reinterpret_cast<tnh_ctx*>(c);
    });
}

void tnh_destroy(tnh_ctx* ctx) {
    if (!ctx) return;
    auto* c = reinterpret_cast<Ctx*>(ctx);
    cudaStreamSynchronize(c->stream);
    const int dev = c->device;
    cudaStream_t s = c->stream;
    delete c;
    // hand the pool's unused memory back (buffers of live plans stay)
    int cur = 0;
    if (cudaGetDevice(&cur) == cudaSuccess && cudaSetDevice(dev) == cudaSuccess) {
        cudaStreamSynchronize(s);
        trim_pool();
        cudaSetDevice(cur);
    }
}

const char* tnh_last_error(const tnh_ctx* ctx) {
    if (ctx) return reinterpret_cast<const Ctx*>(ctx)->err.c_str();
    return g_last_error.c_str();
}

tnh_status tnh_sync(tnh_ctx* ctx) {
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    return guard(c, [&] {
        TNH_REQUIRE(c, TNH_ERR_ARG, "tnh_sync: ctx NULL");
        CUDA_CHECK(cudaStreamSynchronize(c->stream));
        check_device_flag(c);
    });
}

tnh_status tnh_layout(int32_t rank, const tnh_index* inds, const int32_t* flux, int32_t* nblocks,
                      int32_t* block_sect, int64_t* block_off, int64_t* total) {
    return guard(nullptr, [&] {
        TNH_REQUIRE(rank >= 0 && rank <= kMaxDims, TNH_ERR_ARG, "tnh_layout: rank %d", rank);
        TNH_REQUIRE(nblocks && total, TNH_ERR_ARG, "tnh_layout: NULL output");
        std::vector<Index> ix;
        for (int i = 0; i < rank; ++i) ix.push_back(parse_index(inds[i], "tnh_layout"));
        int nq = ix.empty() ? 0 : ix[0].nq;
        std::vector<int> f(nq, 0);
        for (int k = 0; k < nq; ++k) f[k] = flux ? flux[k] : 0;
        Layout L = make_layout(ix, f);
        *nblocks = L.nblocks();
        *total = L.size;
        if (block_sect) std::copy(L.sect.begin(), L.sect.end(), block_sect);
        if (block_off) std::copy(L.off.begin(), L.off.end(), block_off);
    });
}

}  // extern "C"
