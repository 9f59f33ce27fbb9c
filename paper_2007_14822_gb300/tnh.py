"""Thin ctypes binding of ``libtnh.so`` (argument marshalling only).

Every computation runs in the CUDA library; this module only builds the
C structs of ``include/tnh.h`` from Python objects and passes device
pointers of float64 torch tensors. It raises if the library has not been
built (there is no CPU fallback).
"""
from __future__ import annotations

import ctypes as C
import os
import weakref

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libtnh.so")

OK = 0
STATUS = {0: "TNH_OK", 1: "TNH_ERR_ARG", 2: "TNH_ERR_LABEL", 3: "TNH_ERR_ARROW", 4: "TNH_ERR_FLUX",
          5: "TNH_ERR_SHAPE", 6: "TNH_ERR_OOM", 7: "TNH_ERR_CUDA", 8: "TNH_ERR_TIMEOUT",
          9: "TNH_ERR_NUMERIC", 10: "TNH_ERR_NOT_CONVERGED"}
FP64, BF16x6, BF16x3, BF16 = 0, 1, 2, 3
PRECISION = {"fp64": FP64, "bf16x6": BF16x6, "bf16x3": BF16x3, "bf16": BF16}

# exported symbols declared in include/tnh.h
SYMBOLS = ["tnh_create", "tnh_destroy", "tnh_last_error", "tnh_sync", "tnh_layout", "tnh_contract",
           "tnh_heff_plan", "tnh_heff_apply", "tnh_heff_apply_prec", "tnh_heff_flops", "tnh_heff_flops_detail", "tnh_heff_size",
           "tnh_heff_free", "tnh_eigsolve", "tnh_env_update", "tnh_svd_trunc", "tnh_svd_info",
           "tnh_svd_stats", "tnh_svd_get", "tnh_svd_free", "tnh_dmrg", "tnh_profile_begin", "tnh_profile_end",
           "tnh_contract_dense_noalloc", "tnh_heff_plan_sum", "tnh_heff_set_projectors", "tnh_dmrg_ex",
           "tnh_dmrg_mps_size", "tnh_dmrg_mps_link", "tnh_dmrg_mps_get", "tnh_eigsolve_davidson", "tnh_heff_diag",
           "tnh_debug_fail_alloc", "tnh_debug_pool_used", "tnh_debug_wait_timeout", "tnh_debug_convert_check",
           "tnh_heff_apply_host", "tnh_heff_tuning",
           "tnh_dmrg_checkpoint", "tnh_dmrg_resume", "tnh_dmrg_position", "tnh_tridiag_lowest"]


class TnhError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class tnh_index(C.Structure):
    _fields_ = [("label", C.c_int64), ("nsect", C.c_int32), ("nq", C.c_int32),
                ("qn", C.POINTER(C.c_int32)), ("sect_dim", C.POINTER(C.c_int32)), ("arrow", C.c_int32)]


class tnh_tensor(C.Structure):
    _fields_ = [("rank", C.c_int32), ("inds", C.POINTER(tnh_index)), ("nblocks", C.c_int32),
                ("block_sect", C.POINTER(C.c_int32)), ("block_off", C.POINTER(C.c_int64)),
                ("data", C.c_void_p), ("size", C.c_int64)]


class tnh_sweep_params(C.Structure):
    _fields_ = [("nsweep", C.c_int32), ("maxdim", C.POINTER(C.c_int32)), ("cutoff", C.POINTER(C.c_double)),
                ("mindim", C.c_int32), ("krylov_dim", C.c_int32), ("lanczos_tol", C.c_double),
                ("precision", C.c_int32), ("env_precision", C.c_int32), ("eigensolver", C.c_int32),
                ("energy_mode", C.c_int32)]


class tnh_sweep_stat(C.Structure):
    _fields_ = [("sweep", C.c_int32), ("energy", C.c_double), ("resid", C.c_double),
                ("truncerr", C.c_double), ("maxlink", C.c_int32), ("matvecs", C.c_int64),
                ("seconds", C.c_double)]


class tnh_dmrg_problem(C.Structure):
    _fields_ = [("nterm", C.c_int32), ("mpo", C.POINTER(tnh_tensor)), ("start", C.POINTER(C.c_int64)),
                ("done", C.POINTER(C.c_int64)), ("northo", C.c_int32), ("ortho", C.POINTER(tnh_tensor)),
                ("weight", C.c_double)]


_lib = None


def lib():
    """Load libtnh.so; raises when it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2007_14822_gb300.build.build() "
                           "(the CUDA library is required; there is no CPU fallback)")
    L = C.CDLL(LIB_PATH)
    vp, i32, i64, dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_double
    P = C.POINTER
    sig = {
        "tnh_create": (i32, [P(vp), C.c_int, vp]),
        "tnh_destroy": (None, [vp]),
        "tnh_last_error": (C.c_char_p, [vp]),
        "tnh_sync": (i32, [vp]),
        "tnh_layout": (i32, [i32, P(tnh_index), P(i32), P(i32), P(i32), P(i64), P(i64)]),
        "tnh_contract": (i32, [vp, P(tnh_tensor), P(tnh_tensor), P(tnh_tensor), C.c_int]),
        "tnh_heff_plan": (i32, [vp, P(tnh_tensor), P(tnh_tensor), P(tnh_tensor), P(tnh_tensor),
                                P(tnh_tensor), C.c_int, P(vp)]),
        "tnh_heff_apply": (i32, [vp, vp, vp]),
        "tnh_heff_apply_host": (i32, [vp, vp, vp]),
        "tnh_heff_apply_prec": (i32, [vp, C.c_int, vp, vp]),
        "tnh_heff_flops": (i32, [vp, P(dbl)]),
        "tnh_heff_flops_detail": (i32, [vp, P(dbl), P(dbl), P(dbl)]),
        "tnh_heff_size": (i32, [vp, P(i64)]),
        "tnh_heff_tuning": (i32, [vp, P(i32)]),
        "tnh_dmrg_checkpoint": (i32, [vp, C.c_char_p, i32, i64]),
        "tnh_dmrg_resume": (i32, [vp, i32, P(tnh_dmrg_problem), C.c_char_p, P(tnh_sweep_params), P(dbl),
                                  P(tnh_sweep_stat)]),
        "tnh_dmrg_position": (i32, [vp, P(i32), P(i32), P(i32), P(i32)]),
        "tnh_tridiag_lowest": (i32, [vp, i32, P(dbl), P(dbl), P(dbl), P(dbl)]),
        "tnh_heff_free": (None, [vp]),
        "tnh_eigsolve": (i32, [vp, vp, i32, dbl, P(dbl), P(dbl), P(i32)]),
        "tnh_eigsolve_davidson": (i32, [vp, vp, i32, dbl, P(dbl), P(dbl), P(i32)]),
        "tnh_heff_diag": (i32, [vp, vp]),
        "tnh_env_update": (i32, [vp, i32, P(tnh_tensor), P(tnh_tensor), P(tnh_tensor), P(tnh_tensor), C.c_int]),
        "tnh_svd_trunc": (i32, [vp, P(tnh_tensor), i32, dbl, i32, i32, i32, P(vp)]),
        "tnh_svd_info": (i32, [vp, P(i32), P(i32), P(i32), P(i32), P(dbl)]),
        "tnh_svd_stats": (i32, [vp, P(i32), P(i32), P(dbl), P(dbl)]),
        "tnh_svd_get": (i32, [vp, P(tnh_tensor), vp, P(tnh_tensor), i32]),
        "tnh_svd_free": (None, [vp]),
        "tnh_dmrg": (i32, [vp, i32, P(tnh_tensor), i64, i64, P(tnh_tensor), P(tnh_sweep_params), P(dbl),
                           P(tnh_sweep_stat)]),
        "tnh_contract_dense_noalloc": (i32, [vp, P(tnh_tensor), P(tnh_tensor), P(tnh_tensor)]),
        "tnh_heff_plan_sum": (i32, [vp, i32, P(tnh_tensor), P(tnh_tensor), P(tnh_tensor), P(tnh_tensor),
                                    P(tnh_tensor), C.c_int, P(vp)]),
        "tnh_heff_set_projectors": (i32, [vp, i32, vp, dbl]),
        "tnh_dmrg_ex": (i32, [vp, i32, P(tnh_dmrg_problem), P(tnh_tensor), P(tnh_sweep_params), P(dbl),
                              P(tnh_sweep_stat)]),
        "tnh_dmrg_mps_size": (i32, [vp, P(i32)]),
        "tnh_dmrg_mps_link": (i32, [vp, i32, P(i32), P(i32), P(i32), P(i32)]),
        "tnh_dmrg_mps_get": (i32, [vp, i32, P(tnh_tensor)]),
        "tnh_profile_begin": (i32, [vp]),
        "tnh_profile_end": (i32, [vp, i32, P(i32), C.c_char_p, P(i64), P(dbl)]),
        "tnh_debug_fail_alloc": (i32, [i64]),
        "tnh_debug_pool_used": (i32, [vp, P(C.c_uint64)]),
        "tnh_debug_wait_timeout": (i32, [vp, C.c_uint64]),
        "tnh_debug_convert_check": (i32, [vp, C.c_uint64, C.c_uint64, P(C.c_uint64)]),
    }
    for name, (res, args) in sig.items():
        if hasattr(L, name):
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
    _lib = L
    return L


def _check(code, ctx=None):
    if code != OK:
        msg = lib().tnh_last_error(ctx)
        raise TnhError(code, msg.decode() if msg else "")


# ------------------------------------------------------------- host objects
class Index:
    """A QN index: sectors [(qn tuple, dim)], arrow (+1 Out / -1 In), label."""

    def __init__(self, sectors, arrow=+1, label=0):
        self.sectors = [(tuple(int(x) for x in q), int(d)) for q, d in sectors]
        self.arrow = int(arrow)
        self.label = int(label)

    @staticmethod
    def dense(dim, arrow=+1, label=0, nq=1):
        return Index([((0,) * nq, dim)], arrow, label)

    @property
    def nq(self):
        return len(self.sectors[0][0])

    @property
    def dim(self):
        return sum(d for _, d in self.sectors)

    @property
    def nsect(self):
        return len(self.sectors)

    def dag(self):
        return Index(self.sectors, -self.arrow, self.label)

    def same_space(self, other):
        return self.sectors == other.sectors

    def _c(self, keep):
        qn = (C.c_int32 * max(1, self.nsect * self.nq))(*[x for q, _ in self.sectors for x in q])
        dims = (C.c_int32 * self.nsect)(*[d for _, d in self.sectors])
        keep += [qn, dims]
        return tnh_index(self.label, self.nsect, self.nq, C.cast(qn, C.POINTER(C.c_int32)),
                         C.cast(dims, C.POINTER(C.c_int32)), self.arrow)


def layout(inds, flux=None):
    """Allowed blocks (lexicographic) and packed offsets from the C library."""
    L = lib()
    keep = []
    arr = (tnh_index * max(1, len(inds)))(*[i._c(keep) for i in inds])
    nq = inds[0].nq if inds else 0
    fl = (C.c_int32 * max(1, nq))(*(flux or (0,) * nq))
    nb, tot = C.c_int32(0), C.c_int64(0)
    _check(L.tnh_layout(len(inds), arr, fl, C.byref(nb), None, None, C.byref(tot)))
    sect = (C.c_int32 * max(1, nb.value * len(inds)))()
    off = (C.c_int64 * max(1, nb.value))()
    _check(L.tnh_layout(len(inds), arr, fl, C.byref(nb), sect, off, C.byref(tot)))
    r = len(inds)
    blocks = [tuple(sect[b * r:(b + 1) * r]) for b in range(nb.value)]
    return blocks, [int(off[b]) for b in range(nb.value)], int(tot.value)


class Tensor:
    """Block-sparse float64 tensor whose data is a CUDA torch tensor.

    ``blocks`` are sector tuples and ``offsets`` their element offsets in
    ``data``; by default the allowed blocks of ``flux`` from ``layout()``.
    """

    def __init__(self, inds, flux=None, data=None, blocks=None, offsets=None, device="cuda"):
        import torch
        self.inds = list(inds)
        nq = self.inds[0].nq if self.inds else 0
        self.flux = tuple(flux) if flux is not None else (0,) * nq
        if blocks is None:
            blocks, offsets, total = layout(self.inds, self.flux)
        else:
            total = max([o + self.block_size(b) for b, o in zip(blocks, offsets)] or [0])
        self.blocks = [tuple(b) for b in blocks]
        self.offsets = list(offsets)
        if data is None:
            data = torch.zeros(max(total, 1), dtype=torch.float64, device=device)
        self.data = data

    def block_shape(self, key):
        return tuple(self.inds[i].sectors[s][1] for i, s in enumerate(key))

    def block_size(self, key):
        return int(np.prod(self.block_shape(key))) if len(key) else 1

    @property
    def rank(self):
        return len(self.inds)

    def with_inds(self, inds):
        return Tensor(inds, self.flux, self.data, self.blocks, self.offsets)

    def fill(self, fn):
        """Fill block ``key`` with ``fn(key, shape)`` (host numpy)."""
        import torch
        host = np.zeros(self.data.numel())
        for key, off in zip(self.blocks, self.offsets):
            shp = self.block_shape(key)
            host[off:off + self.block_size(key)] = np.asarray(fn(key, shp), dtype=np.float64).ravel()
        self.data.copy_(torch.from_numpy(host).to(self.data.device))
        return self

    def block_arrays(self):
        """Dict sector tuple -> numpy array (copied to the host)."""
        host = self.data.detach().cpu().numpy()
        out = {}
        for key, off in zip(self.blocks, self.offsets):
            out[key] = host[off:off + self.block_size(key)].reshape(self.block_shape(key)).copy()
        return out

    def _c(self, keep):
        r = self.rank
        inds = (tnh_index * max(1, r))(*[i._c(keep) for i in self.inds])
        sect = (C.c_int32 * max(1, len(self.blocks) * r))(*[s for b in self.blocks for s in b])
        off = (C.c_int64 * max(1, len(self.blocks)))(*self.offsets)
        keep += [inds, sect, off]
        return tnh_tensor(r, C.cast(inds, C.POINTER(tnh_index)), len(self.blocks),
                          C.cast(sect, C.POINTER(C.c_int32)), C.cast(off, C.POINTER(C.c_int64)),
                          C.c_void_p(self.data.data_ptr()), int(self.data.numel()))


def _ptr(t):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise TypeError("expected a contiguous float64 CUDA tensor")
    return C.c_void_p(t.data_ptr())


# ------------------------------------------------------------------ context
class Context:
    """A library context on one device and one CUDA stream."""

    def __init__(self, device=0, stream=None):
        import torch
        self._lib = lib()
        if stream is None:
            stream = torch.cuda.current_stream(device).cuda_stream
        self.stream = stream
        h = C.c_void_p()
        _check(self._lib.tnh_create(C.byref(h), int(device), C.c_void_p(stream)))
        self.h = h
        self._children = weakref.WeakSet()

    def close(self):
        """Free every plan / SVD result made by this context, then the context."""
        if getattr(self, "h", None):
            for ch in list(self._children):
                ch.free()
            self._lib.tnh_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def check(self, code):
        _check(code, self.h)

    def sync(self):
        self.check(self._lib.tnh_sync(self.h))

    # ---- failure injection (test support)
    def debug_fail_alloc(self, k):
        """The k-th device allocation from now fails with TNH_ERR_OOM (0 disarms)."""
        _check(self._lib.tnh_debug_fail_alloc(int(k)))

    def debug_pool_used(self):
        """Bytes of the library's device pool held by live allocations (syncs)."""
        v = C.c_uint64()
        self.check(self._lib.tnh_debug_pool_used(self.h, C.byref(v)))
        return v.value

    def debug_wait_timeout(self, limit_ns):
        """A bounded device wait that nothing completes: raises TNH_ERR_TIMEOUT."""
        self.check(self._lib.tnh_debug_wait_timeout(self.h, int(limit_ns)))

    def debug_convert_check(self, n, seed=0):
        """Mismatches of the integer-path float32/float64 conversions against
        the GPU's own conversion on n generated bit patterns (syncs)."""
        v = C.c_uint64()
        self.check(self._lib.tnh_debug_convert_check(self.h, int(n), int(seed), C.byref(v)))
        return v.value

    def profile_begin(self):
        self.check(self._lib.tnh_profile_begin(self.h))

    def profile_end(self):
        """{kernel name: (launches, device milliseconds)} since profile_begin."""
        mx = 64
        n = C.c_int32()
        names = C.create_string_buffer(64 * mx)
        launches = (C.c_int64 * mx)()
        ms = (C.c_double * mx)()
        self.check(self._lib.tnh_profile_end(self.h, mx, C.byref(n), names, launches, ms))
        out = {}
        for k in range(min(n.value, mx)):
            name = names.raw[64 * k:64 * (k + 1)].split(b"\0", 1)[0].decode()
            out[name] = (int(launches[k]), float(ms[k]))
        return out

    def contract(self, A, B, Cout, prec=FP64):
        keep = []
        a, b, c = A._c(keep), B._c(keep), Cout._c(keep)
        self.check(self._lib.tnh_contract(self.h, C.byref(a), C.byref(b), C.byref(c), int(prec)))
        return Cout

    def contract_dense_noalloc(self, A, B, Cout):
        """Dense FP64 C = A * B using only the library's static device scratch."""
        keep = []
        a, b, c = A._c(keep), B._c(keep), Cout._c(keep)
        self.check(self._lib.tnh_contract_dense_noalloc(self.h, C.byref(a), C.byref(b), C.byref(c)))
        return Cout

    def heff_plan(self, L, W1, W2, R, psi, prec=FP64):
        keep = []
        args = [t._c(keep) for t in (L, W1, W2, R, psi)]
        h = C.c_void_p()
        self.check(self._lib.tnh_heff_plan(self.h, *[C.byref(x) for x in args], int(prec), C.byref(h)))
        plan = Heff(self, h)
        self._children.add(plan)
        return plan

    def heff_plan_sum(self, Ls, W1s, W2s, Rs, psi, prec=FP64):
        """H_eff of a sum of MPOs: one (L, W1, W2, R) per term."""
        keep = []
        n = len(Ls)
        arrs = [(tnh_tensor * n)(*[t._c(keep) for t in ts]) for ts in (Ls, W1s, W2s, Rs)]
        p = psi._c(keep)
        h = C.c_void_p()
        self.check(self._lib.tnh_heff_plan_sum(self.h, n, *arrs, C.byref(p), int(prec), C.byref(h)))
        plan = Heff(self, h)
        self._children.add(plan)
        return plan

    def env_update(self, direction, E, A, W, out, prec=FP64):
        keep = []
        args = [t._c(keep) for t in (E, A, W, out)]
        self.check(self._lib.tnh_env_update(self.h, int(direction), *[C.byref(x) for x in args], int(prec)))
        return out

    def svd_trunc(self, T, nrow, cutoff, maxdim, mindim=1, exact_side=0):
        keep = []
        t = T._c(keep)
        h = C.c_void_p()
        self.check(self._lib.tnh_svd_trunc(self.h, C.byref(t), int(nrow), float(cutoff), int(maxdim),
                                           int(mindim), int(exact_side), C.byref(h)))
        res = Svd(self, h, T, nrow)
        self._children.add(res)
        return res

    def dmrg(self, mpo, mps, start, done, maxdim, cutoff, mindim=1, krylov_dim=32, tol=1e-10,
             prec=FP64, env_prec=FP64, ortho=(), weight=1.0, eigensolver="lanczos", resume=None,
             energy_mode=0):
        """Two-site DMRG sweeps. ``mpo`` is one MPO (list of site tensors) or,
        with ``start``/``done`` lists, a list of MPOs whose sum is H;
        ``ortho`` lists previous states (MPS) to stay orthogonal to, with the
        energy penalty ``weight``. With ``resume`` (a checkpoint file) the run
        continues from it and ``mps`` is ignored. Returns (energy, per-sweep
        stats); the final MPS is read with ``dmrg_mps``."""
        keep = []
        ns = len(maxdim)
        md = (C.c_int32 * ns)(*maxdim)
        co = (C.c_double * ns)(*cutoff)
        p = tnh_sweep_params(ns, C.cast(md, C.POINTER(C.c_int32)), C.cast(co, C.POINTER(C.c_double)),
                             int(mindim), int(krylov_dim), float(tol), int(prec), int(env_prec),
                             {"lanczos": 0, "davidson": 1}[eigensolver], int(energy_mode))
        stats = (tnh_sweep_stat * ns)()
        e = C.c_double()
        terms = isinstance(start, (list, tuple))
        N = len(mpo[0]) if terms else len(mpo)
        A = (tnh_tensor * N)(*[a._c(keep) for a in mps]) if resume is None else None
        if not terms and not ortho and resume is None:
            W = (tnh_tensor * N)(*[w._c(keep) for w in mpo])
            self.check(self._lib.tnh_dmrg(self.h, N, W, int(start), int(done), A, C.byref(p), C.byref(e), stats))
        else:
            mpos = list(mpo) if terms else [mpo]
            starts = list(start) if terms else [start]
            dones = list(done) if terms else [done]
            W = (tnh_tensor * (len(mpos) * N))(*[w._c(keep) for m in mpos for w in m])
            st = (C.c_int64 * len(mpos))(*starts)
            dn = (C.c_int64 * len(mpos))(*dones)
            no = len(ortho)
            O = (tnh_tensor * max(1, no * N))(*[a._c(keep) for m in ortho for a in m])
            prob = tnh_dmrg_problem(len(mpos), W, st, dn, no, O, float(weight))
            if resume is None:
                self.check(self._lib.tnh_dmrg_ex(self.h, N, C.byref(prob), A, C.byref(p), C.byref(e), stats))
            else:
                self.check(self._lib.tnh_dmrg_resume(self.h, N, C.byref(prob), os.fsencode(str(resume)),
                                                     C.byref(p), C.byref(e), stats))
        return e.value, [dict(sweep=s.sweep, energy=s.energy, resid=s.resid, truncerr=s.truncerr,
                              maxlink=s.maxlink, matvecs=s.matvecs, seconds=s.seconds) for s in stats]

    def tridiag_lowest(self, alpha, beta):
        """Lowest eigenpair (theta, v) of the tridiagonal (alpha, beta) by the
        eigensolver's device kernel (host float64 arrays in and out)."""
        a = np.ascontiguousarray(alpha, dtype=np.float64)
        b = np.ascontiguousarray(beta, dtype=np.float64)
        k = len(a)
        th = C.c_double()
        v = np.zeros(k)
        P = C.POINTER(C.c_double)
        self.check(self._lib.tnh_tridiag_lowest(self.h, k, a.ctypes.data_as(P),
                                                b.ctypes.data_as(P) if k > 1 else None, C.byref(th),
                                                v.ctypes.data_as(P)))
        return th.value, v

    def dmrg_checkpoint(self, path, every=0, stop_after=0):
        """Write checkpoints of later runs to ``path`` every ``every`` bonds
        (0: at sweep ends) and stop a run after ``stop_after`` bonds (0:
        never); ``path`` None turns checkpointing off."""
        self.check(self._lib.tnh_dmrg_checkpoint(self.h, None if path is None else os.fsencode(str(path)),
                                                 int(every), int(stop_after)))

    def dmrg_position(self):
        """(sweep, pass, step, finished) where the last run ended."""
        a, b, c, d = C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32()
        self.check(self._lib.tnh_dmrg_position(self.h, C.byref(a), C.byref(b), C.byref(c), C.byref(d)))
        return a.value, b.value, c.value, bool(d.value)

    def dmrg_link(self, j):
        """Sectors [(qn, dim)] of link j of the MPS left by the last DMRG run."""
        ns, nq = C.c_int32(), C.c_int32()
        self.check(self._lib.tnh_dmrg_mps_link(self.h, int(j), C.byref(ns), C.byref(nq), None, None))
        qn = (C.c_int32 * max(1, ns.value * nq.value))()
        sd = (C.c_int32 * max(1, ns.value))()
        self.check(self._lib.tnh_dmrg_mps_link(self.h, int(j), C.byref(ns), C.byref(nq), qn, sd))
        return [(tuple(qn[i * nq.value:(i + 1) * nq.value]), int(sd[i])) for i in range(ns.value)]

    def dmrg_mps(self, site):
        """The MPS left by the last DMRG run, as device tensors [link, site, link]."""
        n = C.c_int32()
        self.check(self._lib.tnh_dmrg_mps_size(self.h, C.byref(n)))
        links = [Index(self.dmrg_link(j), +1) for j in range(n.value + 1)]
        out = []
        for j in range(n.value):
            T = Tensor([links[j], site, links[j + 1].dag()])
            keep = []
            t = T._c(keep)
            self.check(self._lib.tnh_dmrg_mps_get(self.h, j, C.byref(t)))
            out.append(T)
        return out


class Heff:
    def __init__(self, ctx, h):
        self.ctx, self.h = ctx, h

    def free(self):
        if getattr(self, "h", None):
            self.ctx._lib.tnh_heff_free(self.h)
            self.h = None

    def __del__(self):
        self.free()

    def apply(self, x, y, prec=None):
        if prec is None:
            self.ctx.check(self.ctx._lib.tnh_heff_apply(self.h, _ptr(x), _ptr(y)))
        else:
            self.ctx.check(self.ctx._lib.tnh_heff_apply_prec(self.h, int(prec), _ptr(x), _ptr(y)))
        return y

    def apply_host(self, x, y):
        """y = H_eff x for CPU float64 tensors (page-locked for asynchronous
        copies): the library copies x in and y out; returns when y is ready."""
        import torch
        for t in (x, y):
            if t.device.type != "cpu" or t.dtype != torch.float64 or not t.is_contiguous():
                raise TypeError("apply_host takes contiguous CPU float64 tensors")
            if t.numel() != self.size:
                raise ValueError(f"apply_host: {t.numel()} elements, the plan has {self.size}")
        self.ctx.check(self.ctx._lib.tnh_heff_apply_host(self.h, C.c_void_p(x.data_ptr()),
                                                         C.c_void_p(y.data_ptr())))
        return y

    @property
    def flops(self):
        f = C.c_double()
        self.ctx.check(self.ctx._lib.tnh_heff_flops(self.h, C.byref(f)))
        return f.value

    @property
    def flops_detail(self):
        """{'s1', 's23', 's4'}: flops of the S1 GEMM, the W1/W2 contractions, the S4 GEMM."""
        a, b, c = C.c_double(), C.c_double(), C.c_double()
        self.ctx.check(self.ctx._lib.tnh_heff_flops_detail(self.h, C.byref(a), C.byref(b), C.byref(c)))
        return {"s1": a.value, "s23": b.value, "s4": c.value}

    @property
    def size(self):
        n = C.c_int64()
        self.ctx.check(self.ctx._lib.tnh_heff_size(self.h, C.byref(n)))
        return n.value

    @property
    def tuning(self):
        """The plan's choices: {'tiles_s1', 'split_s1', 'tiles_s4', 'split_s4',
        'measured', 'strategy', 'strategy_measured', 'fused_s4'} (see tnh_heff_tuning)."""
        c = (C.c_int32 * 8)()
        self.ctx.check(self.ctx._lib.tnh_heff_tuning(self.h, c))
        return {"tiles_s1": c[0], "split_s1": c[1], "tiles_s4": c[2], "split_s4": c[3], "measured": bool(c[4]),
                "strategy": c[5], "strategy_measured": bool(c[6]), "fused_s4": bool(c[7])}

    def diag(self, out):
        """Diagonal of the MPO part of H_eff into ``out`` (CUDA float64 [n])."""
        self.ctx.check(self.ctx._lib.tnh_heff_diag(self.h, _ptr(out)))
        return out

    def set_projectors(self, phi, weight):
        """Add weight * phi_i <phi_i, x> to every product (phi: CUDA float64
        [k, n], or None to remove)."""
        if phi is None:
            self.ctx.check(self.ctx._lib.tnh_heff_set_projectors(self.h, 0, None, 0.0))
            return
        k = phi.shape[0] if phi.dim() == 2 else 1
        self.ctx.check(self.ctx._lib.tnh_heff_set_projectors(self.h, int(k), _ptr(phi.contiguous()),
                                                             float(weight)))

    def eigsolve(self, psi, krylov_dim=64, tol=1e-10, method="lanczos"):
        e, r, k = C.c_double(), C.c_double(), C.c_int32()
        f = {"lanczos": self.ctx._lib.tnh_eigsolve, "davidson": self.ctx._lib.tnh_eigsolve_davidson}[method]
        self.ctx.check(f(self.h, _ptr(psi), int(krylov_dim), float(tol), C.byref(e), C.byref(r), C.byref(k)))
        return e.value, r.value, k.value


class Svd:
    """Result of tnh_svd_trunc: the new link and the factors on request."""

    def __init__(self, ctx, h, T, nrow):
        self.ctx, self.h, self.T, self.nrow = ctx, h, T, nrow
        ns, nq, te = C.c_int32(), C.c_int32(), C.c_double()
        L = ctx._lib
        ctx.check(L.tnh_svd_info(h, C.byref(ns), C.byref(nq), None, None, C.byref(te)))
        qn = (C.c_int32 * max(1, ns.value * nq.value))()
        sd = (C.c_int32 * max(1, ns.value))()
        ctx.check(L.tnh_svd_info(h, C.byref(ns), C.byref(nq), qn, sd, C.byref(te)))
        self.sectors = [(tuple(qn[i * nq.value:(i + 1) * nq.value]), int(sd[i])) for i in range(ns.value)]
        self.truncerr = te.value

    def free(self):
        if getattr(self, "h", None):
            self.ctx._lib.tnh_svd_free(self.h)
            self.h = None

    def __del__(self):
        self.free()

    def stats(self):
        """Rounds and rotation flops of the float32 and float64 Jacobi stages."""
        r32, r64, f32, f64 = C.c_int32(), C.c_int32(), C.c_double(), C.c_double()
        self.ctx.check(self.ctx._lib.tnh_svd_stats(self.h, C.byref(r32), C.byref(r64), C.byref(f32),
                                                   C.byref(f64)))
        return {"rounds32": r32.value, "rounds64": r64.value, "flops32": f32.value, "flops64": f64.value}

    @property
    def kept(self):
        return sum(d for _, d in self.sectors)

    def factors(self, link_label=0, absorb=0):
        """(U, S, V) as device tensors with a new link index (U's c In, V's c Out).

        absorb = 1 multiplies S into U, 2 into V (0: neither)."""
        import torch
        link = Index(self.sectors, +1, link_label)
        rows = self.T.inds[:self.nrow]
        cols = self.T.inds[self.nrow:]
        U = Tensor(list(rows) + [link.dag()], tuple(0 for _ in self.T.flux))
        V = Tensor([link] + list(cols), self.T.flux)
        S = torch.zeros(max(1, self.kept), dtype=torch.float64, device=self.T.data.device)
        keep = []
        u, v = U._c(keep), V._c(keep)
        self.ctx.check(self.ctx._lib.tnh_svd_get(self.h, C.byref(u), _ptr(S), C.byref(v), int(absorb)))
        return U, S[:self.kept], V
