#!/usr/bin/env python3
"""Benchmark of the two-site DMRG hot path on one GB300 (replicas on N GPUs).

Headline workload: the effective-Hamiltonian product H_eff.psi at one bulk
bond (sites 62/63) of the U(1) J1-J2 cylinder Ly=6 x Lx=24 (J2/J1 = 1/2,
snake order, finite-state MPO with w = 26) at bond dimension m = 2048: the
link has 41 Gaussian charge sectors of 1..256 states (2Sz = -40..40), L, R
and psi hold seeded N(0,1) blocks (seed 6). One step is one application of
the plan's product y = H_eff x in BF16x6 (split-bfloat16 tcgen05 GEMMs with
float32 accumulation), replayed from its CUDA graph: pack psi, S1 = L.psi,
the fused W1.W2 pass, S4 = T3.R. L2 is flushed before every step. The
metric counts the algorithmic flops of the labelled chain (2MNK summed over
the allowed block pairs of S1..S4; the extra products of the bf16 split are
not counted) divided by the step time.

More measurements go on the same JSON line (skip with --no-extra):
  heff_qn          H_eff TFLOP/s, BF16x6 and FP64, and the matvec error of
                   every split mode (BF16x6, BF16x3, BF16) against FP64, on three block-sparse
                   workloads (U(1) m=1024, the cylinder m=2048, U(1)xU(1)
                   Hubbard m=4096); flops are the plan's block-pair sum
  bond_update_m256 one full bond update of the dense Heisenberg chain at
                   m=256 (theta, Lanczos in BF16x6, FP64 energy, SVD,
                   environment update): every step of the hot path
  sweep            DMRG sweep time, BF16x6 vs FP64, and the relative energy
                   difference of the two runs and to the oracle
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

M, W_DIM, D = 256, 5, 2
K_LANCZOS = 8
CUTOFF, MAXDIM = 1e-10, 256
METRIC = "H_eff·ψ TFLOP/s + DMRG sweep time, mixed vs FP64 on GB300 at ΔE/E≤1e-9"


def step_flops(m=M, w=W_DIM, d=D, k=K_LANCZOS):
    theta = 2 * d * d * m ** 3
    heff = 4 * w * d * d * m ** 3 + 4 * w * w * d ** 3 * m * m
    env = 4 * w * d * m ** 3 + 2 * w * w * d * d * m * m
    return theta + (k + 1) * heff + env, heff


# ----------------------------------------------------------------- inputs
def host_inputs(m=M):
    """Seeded host arrays of the workload (shared by both arms)."""
    from paper_2007_14822_gb300 import models as pm, synth
    L = synth.gaussian(2, (m, W_DIM, m))
    R = synth.gaussian(3, (m, W_DIM, m))
    for E in (L, R):
        for ch in (0, 3, 4):
            E[:, ch, :] = 0.5 * (E[:, ch, :] + E[:, ch, :].T)
        E[:, 2, :] = E[:, 1, :].T
    A = synth.gaussian(4, (2, m, D, m)) / np.sqrt(m)
    W = pm.heisenberg(3).W[1]
    return dict(L=L, R=R, A1=A[0], A2=A[1], W=W)


class GpuBond:
    """Device tensors and one bond update through the C ABI."""

    def __init__(self, ctx, host, pinned=False):
        import torch
        from paper_2007_14822_gb300.tnh import Index, Tensor, BF16x6, FP64
        self.ctx, self.torch = ctx, torch
        self.FP64, self.MIX = FP64, BF16x6
        # labels matter only for the labelled contraction theta = A1 * A2
        a, c, b = Index.dense(M, +1, 1), Index.dense(M, +1, 3), Index.dense(M, +1, 5)
        s1, s2 = Index.dense(D, +1, 2), Index.dense(D, +1, 4)
        s = s1
        wl, wr = Index.dense(W_DIM, -1), Index.dense(W_DIM, +1)
        self.L = Tensor([a.dag(), wl.dag(), a])
        self.R = Tensor([b, wr.dag(), b.dag()])
        self.W = Tensor([wl, wr, s.dag(), s])
        self.A1 = Tensor([a, s1, c.dag()])
        self.A2 = Tensor([c, s2, b.dag()])
        self.theta = Tensor([a, s1, s2, b.dag()])
        self.Lnew = Tensor([a, wr, a.dag()])
        self.host = host
        self.pinned = {}
        for k, t in (("L", self.L), ("R", self.R), ("A1", self.A1), ("A2", self.A2), ("W", self.W)):
            arr = torch.from_numpy(np.ascontiguousarray(host[k]).ravel())
            self.pinned[k] = arr.pin_memory() if pinned else arr
            t.data.copy_(self.pinned[k])
        self.s_idx = s
        self.h2d_bytes = sum(self.pinned[k].numel() * 8 for k in ("L", "R", "A1", "A2"))
        self.d2h_bytes = 0

    def upload(self):
        for k, t in (("L", self.L), ("R", self.R), ("A1", self.A1), ("A2", self.A2)):
            t.data.copy_(self.pinned[k], non_blocking=True)

    def step(self, download=False):
        ctx = self.ctx
        ctx.contract(self.A1, self.A2, self.theta, self.FP64)
        plan = ctx.heff_plan(self.L, self.W, self.W, self.R, self.theta, self.MIX)
        E, res, k = plan.eigsolve(self.theta.data, krylov_dim=K_LANCZOS, tol=0.0)
        plan.free()
        svd = ctx.svd_trunc(self.theta, 2, CUTOFF, MAXDIM)
        U, S, V = svd.factors(absorb=2)
        self.svd_stats = svd.stats()
        svd.free()
        Lnew = self.Lnew.__class__([U.inds[2], self.W.inds[1], U.inds[2].dag()])
        ctx.env_update(1, self.L, U, self.W, Lnew, self.FP64)
        out = dict(E=E, res=res, k=k, kept=U.inds[2].dim)
        if download:
            h = U.data.cpu()
            self.d2h_bytes = 8 + h.numel() * 8
            out["U"] = h
        return out


# ---------------------------------------------- block-sparse H_eff workloads
# (name, model, m, sector recipe, seed): U(1) Heisenberg m=1024 with 40
# Gaussian sectors of 1..128; the J1-J2 6x24 cylinder (snake order, FSA MPO,
# bulk sites 62/63, w=26) at m=2048 with 41 sectors of 1..256; U(1)xU(1)
# Hubbard (U/t=4) at m=4096 with a 15x15 grid of (N, 2Sz) sectors of 1..128.
QN_CONFIGS = [
    ("U(1) Heisenberg, m=1024, w=5, 40 sectors of 1..128", "heis", 1024, (40, 128), 5),
    ("U(1) J1-J2 cylinder 6x24, m=2048, w=26, 41 sectors of 1..256", "cyl", 2048, (41, 256), 6),
    ("U(1)xU(1) Hubbard U/t=4, m=4096, w=6, d=4, 15x15 sectors of 1..128", "hub", 4096, (15, 128), 7),
]


def qn_link(kind, m, recipe):
    from paper_2007_14822_gb300 import synth
    from paper_2007_14822_gb300.tnh import Index
    if kind == "hub":
        n, maxd = recipe
        dims = synth.gaussian_sectors_2d(m, (n, n), maxd)
        secs = []
        for u in range(n):          # up / down electrons relative to half filling
            for v in range(n):
                du, dv = u - (n - 1) // 2, v - (n - 1) // 2
                secs.append(((du + dv, du - dv), int(dims[u, v])))
        return Index(secs, +1)
    nsect, maxd = recipe
    dims = synth.gaussian_sectors(m, nsect, maxd)
    return Index([((2 * (k - (nsect - 1) // 2),), d) for k, d in enumerate(dims)], +1)


def qn_mpo(kind):
    """Host MPO and the bond (j, j+1) of a block-sparse workload."""
    from paper_2007_14822_gb300 import models as pm
    if kind == "heis":
        return pm.heisenberg(8), 3
    if kind == "cyl":
        return pm.spin_pairs(144, pm.cylinder_pairs(24, 6, 1.0, 0.5)), 62
    return pm.hubbard(16, 1.0, 4.0), 7


def qn_heff_inputs(kind, m, recipe, seed):
    """Device tensors L, W1, W2, R, psi of a block-sparse workload."""
    from paper_2007_14822_gb300 import models as pm, synth
    from paper_2007_14822_gb300.tnh import Tensor
    mpo, j = qn_mpo(kind)
    W = pm.to_device(mpo, qn=True)
    W1, W2 = W[j], W[j + 1]
    a = qn_link(kind, m, recipe)
    L = Tensor([a.dag(), W1.inds[0].dag(), a])
    R = Tensor([a, W2.inds[1].dag(), a.dag()])
    psi = Tensor([a, W1.inds[3], W2.inds[3], a.dag()])
    for T, tag in ((L, "L"), (R, "R"), (psi, "psi")):
        T.fill(lambda k, shp, tag=tag: synth.block_gaussian(seed, tag, k, shp))
    return L, W1, W2, R, psi


def qn_oracle_inputs(kind, m, recipe, seed):
    """The same workload as oracle BlockTensors, built on the host alone (the
    same models, sector recipe and keyed block generator; no library call)."""
    from paper_2007_14822_gb300 import synth
    from oracle.blocksparse import BlockTensor, QNIndex
    mpo, j = qn_mpo(kind)
    a = qn_link(kind, m, recipe)
    A = QNIndex(a.sectors, +1)
    site = QNIndex([(q, 1) for q in mpo.site_qn], +1)

    def mpo_tensor(k):
        wl = QNIndex([(q, 1) for q in mpo.link_qn[k]], -1)
        wr = QNIndex([(q, 1) for q in mpo.link_qn[k + 1]], +1)
        return BlockTensor.from_dense(mpo.W[k], [wl, wr, site.dag(), site])
    W1, W2 = mpo_tensor(j), mpo_tensor(j + 1)
    fn = lambda tag: (lambda k, shp: synth.block_gaussian(seed, tag, k, shp))
    L = BlockTensor.from_blocks_fn([A.dag(), W1.inds[0].dag(), A], None, fn("L"))
    R = BlockTensor.from_blocks_fn([A, W2.inds[1].dag(), A.dag()], None, fn("R"))
    psi = BlockTensor.from_blocks_fn([A, W1.inds[3], W2.inds[3], A.dag()], None, fn("psi"))
    return L, W1, W2, R, psi


def _pair_flops(A, ca, B, cb):
    """2MNK summed over the stored block pairs of A and B that agree on the
    contracted axes (ca of A with cb of B)."""
    fa = [i for i in range(A.rank) if i not in ca]
    fb = [i for i in range(B.rank) if i not in cb]
    byk = {}
    for kb in B.blocks:
        byk.setdefault(tuple(kb[i] for i in cb), []).append(kb)
    flops = 0.0
    for ka in A.blocks:
        for kb in byk.get(tuple(ka[i] for i in ca), []):
            M = np.prod([A.inds[i].sdim(ka[i]) for i in fa]) if fa else 1
            N = np.prod([B.inds[i].sdim(kb[i]) for i in fb]) if fb else 1
            K = np.prod([A.inds[i].sdim(ka[i]) for i in ca]) if ca else 1
            flops += 2.0 * M * N * K
    return flops


class _Keys:
    """An intermediate of the chain: its indices and every allowed block of
    its flux (as a labelled contraction stores them), dimensions only."""
    def __init__(self, inds, flux):
        from oracle.blocksparse import allowed_blocks
        self.inds, self.blocks = inds, {k: None for k in allowed_blocks(inds, flux)}

    @property
    def rank(self):
        return len(self.inds)


def chain_flops(L, W1, W2, R, psi):
    """Algorithmic flops of one H_eff product on oracle tensors: the labelled
    chain S1 = L.psi (over a), S2 = .W1 (over w, s1), S3 = .W2 (over w1, s2),
    S4 = .R (over w2, b), each 2MNK summed over its block pairs, the
    intermediates holding every allowed block of their flux."""
    from oracle.blocksparse import qn_add
    # L[a,w,a'] psi[a,s1,s2,b] -> T1[w,a',s1,s2,b]
    f1 = _pair_flops(L, [0], psi, [0])
    fl1 = qn_add(L.flux, psi.flux)
    T1 = _Keys([L.inds[1], L.inds[2], psi.inds[1], psi.inds[2], psi.inds[3]], fl1)
    # T1[w,a',s1,s2,b] W1[w,w1,s1,s1'] -> T2[a',s2,b,w1,s1']
    f2 = _pair_flops(T1, [0, 2], W1, [0, 2])
    fl2 = qn_add(fl1, W1.flux)
    T2 = _Keys([T1.inds[1], T1.inds[3], T1.inds[4], W1.inds[1], W1.inds[3]], fl2)
    # T2[a',s2,b,w1,s1'] W2[w1,w2,s2,s2'] -> T3[a',b,s1',w2,s2']
    f3 = _pair_flops(T2, [3, 1], W2, [0, 2])
    T3 = _Keys([T2.inds[0], T2.inds[2], T2.inds[4], W2.inds[1], W2.inds[3]], qn_add(fl2, W2.flux))
    # T3[a',b,s1',w2,s2'] R[b,w2,b'] -> y[a',s1',s2',b']
    f4 = _pair_flops(T3, [1, 3], R, [0, 1])
    return f1 + f2 + f3 + f4


def time_apply(torch, plan, x, y, prec, reps):
    for _ in range(2):
        plan.apply(x, y, prec)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        plan.apply(x, y, prec)
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / 1e3 / reps


PEAKS = {}


def oracle_tensor(T):
    """The FP64 oracle's copy of a device tensor (blocks copied to the host)."""
    from oracle.blocksparse import BlockTensor, QNIndex
    return BlockTensor([QNIndex(i.sectors, i.arrow) for i in T.inds], T.flux, T.block_arrays())


def oracle_matvec_seconds(L, W1, W2, R, psi):
    """One H_eff application by the oracle on the host cores (numpy FP64)."""
    from oracle import dmrg as D_
    args = [oracle_tensor(T) for T in (L, W1, W2, R, psi)]
    t0 = time.perf_counter()
    D_.heff_apply(*args)
    return time.perf_counter() - t0


def bench_qn_heff(ctx, torch, tnh, oracle_kinds=()):
    out = []
    for name, kind, m, recipe, seed in QN_CONFIGS:
        L, W1, W2, R, psi = qn_heff_inputs(kind, m, recipe, seed)
        t0 = time.perf_counter()
        plan = ctx.heff_plan(L, W1, W2, R, psi, tnh.BF16x6)
        t_plan = time.perf_counter() - t0
        y = torch.empty_like(psi.data)
        t_mix = time_apply(torch, plan, psi.data, y, None, 20)
        t_64 = time_apply(torch, plan, psi.data, y, tnh.FP64, 3)
        ctx.profile_begin()
        plan.apply(psi.data, y)
        prof = ctx.profile_end()
        f = plan.flops
        fd = plan.flops_detail
        gname = [k for k in prof if k.startswith("gemm_tc")]
        g_ms = sum(prof[k][1] for k in gname)
        pk = PEAKS.get("bf16_tflops", 1900.0)
        gemm_alg = (fd["s1"] + fd["s4"]) / (g_ms / 1e3) / 1e12 if g_ms > 0 else None
        out.append({"workload": name, "psi_elems": plan.size, "flops_per_matvec": f, "flops_detail": fd,
                    "gemm_roofline": {"bound": "tensor", "kernel": gname[0] if gname else None,
                                      "achieved_algorithmic": gemm_alg,
                                      "achieved_mma": 6 * gemm_alg if gemm_alg else None,
                                      "peak": pk, "unit": "TFLOP/s",
                                      "frac_mma": 6 * gemm_alg / pk if gemm_alg else None,
                                      "note": "S1+S4 flops over the two GEMM launches (profiled, direct "
                                              "launches); BF16x6 issues 6 bf16 products per flop"},
                    "bf16x6": {"ms": t_mix * 1e3, "tflops": f / t_mix / 1e12},
                    "fp64": {"ms": t_64 * 1e3, "tflops": f / t_64 / 1e12},
                    "plan_ms": t_plan * 1e3,
                    "kernels_bf16x6": {k: {"launches": v[0], "ms": v[1]} for k, v in prof.items()}})
        # measured matvec error of every split mode against the FP64 product
        # on the same inputs (which matches the oracle to 1e-12 in the tests):
        # |y_mode - y_fp64|_2 / |y_fp64|_2 and the largest element deviation
        # over |y_fp64|_inf
        y64 = torch.empty_like(psi.data)
        plan.apply(psi.data, y64, tnh.FP64)
        errs = {}
        for mode in ("bf16x6", "bf16x3", "bf16"):
            pm_ = plan if mode == "bf16x6" else ctx.heff_plan(L, W1, W2, R, psi, tnh.PRECISION[mode])
            ym = torch.empty_like(psi.data)
            pm_.apply(psi.data, ym)
            errs[mode] = {"norm": float(torch.linalg.vector_norm(ym - y64) / torch.linalg.vector_norm(y64)),
                          "max_elem": float((ym - y64).abs().max() / y64.abs().max())}
            if pm_ is not plan:
                pm_.free()
            del ym
        out[-1]["matvec_rel_err_vs_fp64"] = errs
        del y64
        if kind in oracle_kinds:
            t_or = oracle_matvec_seconds(L, W1, W2, R, psi)
            out[-1]["oracle_matvec"] = {"s": t_or, "tflops": f / t_or / 1e12, "cores": blas_threads(),
                                        "kind": "oracle", "sample": "one H_eff application"}
        plan.free()
        del L, R, psi, W1, W2, y
        torch.cuda.empty_cache()
    return out


# ----------------------------------------------------------- sweep time
# U(1) Heisenberg chain N=100 from the Neel state, bond dimension schedule
# 32, 64, 128, 256, 256 with cutoff 1e-12 (the finest that the BF16x6
# matvec accuracy supports), 16 Lanczos steps at most: the sweep time is the
# last sweep's, both precisions.
SWEEP_N = 100
SWEEP_SCHEDULE = [(32, 1e-12), (64, 1e-12), (128, 1e-12), (256, 1e-12), (256, 1e-12)]
# the oracle's energy for the same run, stored by tests/golden/make_heisenberg_n100.py
SWEEP_GOLDEN = os.path.join(ROOT, "tests", "golden", "heisenberg_n100_dmrg.json")


def sweep_reference():
    """Stored oracle result of the N=100 sweeps (energy, per-sweep times)."""
    with open(SWEEP_GOLDEN) as f:
        return json.load(f)


def mixed_kw(tnh):
    """Mixed-precision sweep settings: BF16x6 matvecs and environment updates,
    the FP64 energy product at each sweep's last bond, the final energy
    evaluated with FP64 environments."""
    return dict(prec=tnh.BF16x6, env_prec=tnh.BF16x6, energy_mode=1)


def sweep_record(E, st, t_run):
    last = st[-1]
    return {"energy": E, "last_sweep_s": last["seconds"], "maxlink": last["maxlink"],
            "matvecs_last_sweep": last["matvecs"], "truncerr": last["truncerr"], "run_s": t_run,
            "sweep_s": [x["seconds"] for x in st], "maxlink_per_sweep": [x["maxlink"] for x in st]}


def bench_sweeps(ctx, tnh):
    from paper_2007_14822_gb300 import models as pm
    mpo = pm.heisenberg(SWEEP_N)
    res = {}
    for name, kw, tol in (("bf16x6", mixed_kw(tnh), 1e-7), ("fp64", {"prec": tnh.FP64}, 1e-9)):
        W = pm.to_device(mpo, qn=True)
        A = pm.product_state(W[0].inds[3], [0, 1] * (SWEEP_N // 2))
        t0 = time.perf_counter()
        E, st = ctx.dmrg(W, A, mpo.start, mpo.done, [m for m, _ in SWEEP_SCHEDULE],
                         [c for _, c in SWEEP_SCHEDULE], krylov_dim=16, tol=tol, **kw)
        res[name] = sweep_record(E, st, time.perf_counter() - t0)
        if name == "fp64":
            final_mps = ctx.dmrg_mps(W[0].inds[3])
    e64 = res["fp64"]["energy"]
    res["dE_rel_mixed_vs_fp64"] = abs(res["bf16x6"]["energy"] - e64) / abs(e64)
    res["speedup_mixed_vs_fp64"] = res["fp64"]["last_sweep_s"] / res["bf16x6"]["last_sweep_s"]
    res["energy_per_bond_fp64"] = e64 / (SWEEP_N - 1)
    ref = sweep_reference()
    res["energy_oracle"] = ref["energy"]
    res["dE_rel_vs_oracle"] = {k: abs(res[k]["energy"] - ref["energy"]) / abs(ref["energy"]) for k in ("bf16x6", "fp64")}
    # the oracle's last sweep timed here, on this machine's cores: one sweep
    # (maxdim 256, cutoff 1e-12, Lanczos <= 16) from the GPU run's final MPS
    res["oracle_last_sweep"] = oracle_sweep_from(final_mps, SWEEP_N, SWEEP_SCHEDULE[-1])
    res["oracle_last_sweep_stored"] = {"value": ref["sweeps"][-1]["seconds"], "host": ref["host"],
                                       "kind": "oracle, stored by tests/golden/make_heisenberg_n100.py"}
    res["model"] = (f"U(1) Heisenberg chain N={SWEEP_N}, Neel start, maxdim "
                    f"{[m for m, _ in SWEEP_SCHEDULE]}, cutoff 1e-12, Lanczos <= 16 steps")
    res["m1024"] = bench_heis_m1024(ctx, tnh)
    res["small"] = bench_small_sweeps(ctx, tnh)
    res["cylinder_6x4_m2048"] = bench_cylinder_sweeps(ctx, tnh)
    res["cylinder_6x24_m2048"] = bench_large_sweeps(ctx, tnh, "cyl")
    res["hubbard_n64_m4096"] = bench_large_sweeps(ctx, tnh, "hub")
    return res


def oracle_sweep_from(mps, N, sweep):
    """One oracle sweep (numpy FP64, this machine's cores) from a device MPS."""
    from oracle import dmrg as D_, models as om
    A = [oracle_tensor(T) for T in mps]
    t0 = time.perf_counter()
    E, _, st = D_.dmrg(om.heisenberg_mpo(N), A, [sweep], 16, 1e-9)
    dt = time.perf_counter() - t0
    return {"value": dt, "unit": "s", "energy": E, "cores": blas_threads(), "cpu": cpu_model(), "kind": "oracle",
            "sample": f"one sweep, maxdim {sweep[0]}, cutoff {sweep[1]}, from the GPU run's final MPS"}


def bench_heis_m1024(ctx, tnh):
    """Config 3 at its stated maxdim: the N=100 chain with maxdim up to 1024
    (cutoff 1e-12 decides the bond dimension the state needs)."""
    from paper_2007_14822_gb300 import models as pm
    mpo = pm.heisenberg(SWEEP_N)
    sched = [(64, 1e-12), (256, 1e-12), (1024, 1e-12), (1024, 1e-12)]
    res = {}
    for name, kw, tol in (("bf16x6", mixed_kw(tnh), 1e-7), ("fp64", {"prec": tnh.FP64}, 1e-9)):
        W = pm.to_device(mpo, qn=True)
        A = pm.product_state(W[0].inds[3], [0, 1] * (SWEEP_N // 2))
        t0 = time.perf_counter()
        E, st = ctx.dmrg(W, A, mpo.start, mpo.done, [m for m, _ in sched], [c for _, c in sched], krylov_dim=16,
                         tol=tol, **kw)
        res[name] = sweep_record(E, st, time.perf_counter() - t0)
    e64 = res["fp64"]["energy"]
    res["dE_rel_mixed_vs_fp64"] = abs(res["bf16x6"]["energy"] - e64) / abs(e64)
    res["speedup_mixed_vs_fp64"] = res["fp64"]["last_sweep_s"] / res["bf16x6"]["last_sweep_s"]
    res["model"] = (f"U(1) Heisenberg chain N={SWEEP_N}, Neel start, maxdim {[m for m, _ in sched]}, cutoff 1e-12, "
                    "Lanczos <= 16 steps")
    return res


# The configurations at their stated size: the J1-J2 cylinder Ly=6 x Lx=24
# (N=144, w=26) up to m=2048 and the Hubbard chain N=64 (U/t=4, half
# filling, U(1)xU(1)) up to m=4096. The mixed-precision run goes the whole
# schedule (the last sweep is timed); its checkpoint before the last sweep
# is then resumed twice for LARGE_BONDS bond updates, in FP64 and in the
# mixed precision, both with the FP64 energy at every bond: the per-bond
# times and energies of the two precisions on the same state, and the FP64
# sweep time estimated as per-bond time x bonds per sweep.
LARGE = {
    "cyl": dict(name="U(1) J1-J2 cylinder Ly=6 x Lx=24 (N=144, J2/J1=0.5, w=26, snake order), Neel start",
                N=144, sched=[(256, 1e-10), (512, 1e-10), (1024, 1e-10), (2048, 1e-10), (2048, 1e-10),
                              (2048, 1e-10)], krylov=6, states=[0, 1] * 72),
    "hub": dict(name="U(1)xU(1) Hubbard chain N=64, U/t=4, half filling, alternating up/down start",
                N=64, sched=[(256, 1e-12), (1024, 1e-12), (2048, 1e-12), (4096, 1e-12), (4096, 1e-12)],
                krylov=6, states=[1, 2] * 32),
}
LARGE_BONDS = 24


def bench_large_sweeps(ctx, tnh, kind):
    import tempfile
    from paper_2007_14822_gb300 import models as pm
    cfg = LARGE[kind]
    N = cfg["N"]
    mpo = pm.spin_pairs(N, pm.cylinder_pairs(24, 6, 1.0, 0.5)) if kind == "cyl" else pm.hubbard(N, 1.0, 4.0)
    W = pm.to_device(mpo, qn=True)
    site = W[0].inds[3]
    md, co = [m for m, _ in cfg["sched"]], [c for _, c in cfg["sched"]]
    kw_run = dict(krylov_dim=cfg["krylov"], tol=0.0)
    res = {"model": f"{cfg['name']}, maxdim {md}, cutoff {co[-1]}, {cfg['krylov']} Lanczos steps per bond"}
    with tempfile.TemporaryDirectory() as tmp:
        start = os.path.join(tmp, "last_sweep.ckpt")
        center = os.path.join(tmp, "center.ckpt")
        ctx.dmrg_checkpoint(start, 0, 0)      # a checkpoint at every sweep end but the last
        t0 = time.perf_counter()
        E, st = ctx.dmrg(W, pm.product_state(site, cfg["states"]), mpo.start, mpo.done, md, co,
                         **kw_run, **mixed_kw(tnh))
        res["bf16x6"] = sweep_record(E, st, time.perf_counter() - t0)
        # the last sweep again from its start, in mixed precision, up to the
        # bonds around the chain's centre (where the bond dimension is largest)
        first = N // 2 - LARGE_BONDS // 2
        ctx.dmrg_checkpoint(center, 0, first)
        ctx.dmrg(W, None, mpo.start, mpo.done, md, co, resume=start, **kw_run, **mixed_kw(tnh))
        bonds = 2 * (N - 1)
        part = {}
        for name, kw in (("bf16x6", dict(prec=tnh.BF16x6, env_prec=tnh.BF16x6)), ("fp64", dict(prec=tnh.FP64))):
            ctx.dmrg_checkpoint(None, 0, LARGE_BONDS)
            t0 = time.perf_counter()
            ctx.dmrg(W, None, mpo.start, mpo.done, md, co, resume=center, **kw_run, **kw)
            dt = time.perf_counter() - t0
            part[name] = {"bonds": LARGE_BONDS, "first_bond": first, "s": dt, "s_per_bond": dt / LARGE_BONDS}
        ctx.dmrg_checkpoint(None, 0, 0)
    ratio = part["fp64"]["s_per_bond"] / part["bf16x6"]["s_per_bond"]
    part["speedup_per_bond"] = ratio
    part["note"] = (f"bonds {first}..{first + LARGE_BONDS - 1} of the last sweep's left-to-right pass, both "
                    "resumed from the same checkpoint with the FP64 energy at every bond")
    res["central_bonds"] = part
    # the FP64 sweep time estimated from the mixed sweep's and the central
    # bonds' ratio (the edge bonds, with small bond dimensions, are cheaper)
    res["fp64_sweep_s_estimate"] = res["bf16x6"]["last_sweep_s"] * ratio
    res["fp64_sweep_s_estimate_note"] = "mixed last sweep time x FP64 / mixed time per central bond"
    res["speedup_mixed_vs_fp64_estimate"] = ratio
    return res


# J1-J2 cylinder (Ly=6 periodic, Lx=4 open, snake order, J2/J1=1/2, w=26) up
# to m=2048: the bond dimension grows about fourfold per sweep from the Neel
# state, so seven sweeps of maxdim 256, 512, 1024, 2048 x4 (cutoff 1e-10),
# six Lanczos steps per bond in both precisions; the sweep time is the last
# sweep's. Length 4 keeps the FP64 run within the bench's time.
CYL_SCHEDULE = [(256, 1e-10), (512, 1e-10), (1024, 1e-10)] + [(2048, 1e-10)] * 4


def bench_cylinder_sweeps(ctx, tnh):
    from paper_2007_14822_gb300 import models as pm
    Lx, Ly = 4, 6
    N = Lx * Ly
    mpo = pm.spin_pairs(N, pm.cylinder_pairs(Lx, Ly, 1.0, 0.5))
    res = {}
    for name, kw in (("bf16x6", mixed_kw(tnh)), ("fp64", {"prec": tnh.FP64})):
        W = pm.to_device(mpo, qn=True)
        A = pm.product_state(W[0].inds[3], [0, 1] * (N // 2))
        t0 = time.perf_counter()
        E, st = ctx.dmrg(W, A, mpo.start, mpo.done, [m for m, _ in CYL_SCHEDULE], [c for _, c in CYL_SCHEDULE],
                         krylov_dim=6, tol=0.0, **kw)
        res[name] = sweep_record(E, st, time.perf_counter() - t0)
    e64 = res["fp64"]["energy"]
    res["dE_rel_mixed_vs_fp64"] = abs(res["bf16x6"]["energy"] - e64) / abs(e64)
    res["speedup_mixed_vs_fp64"] = res["fp64"]["last_sweep_s"] / res["bf16x6"]["last_sweep_s"]
    res["model"] = (f"U(1) J1-J2 cylinder Ly={Ly} x Lx={Lx} (N={N}, J2/J1=0.5, w={mpo.max_bond()}), Neel start, "
                    f"maxdim {[m for m, _ in CYL_SCHEDULE]}, cutoff 1e-10, 6 Lanczos steps per bond")
    return res


def bench_small_sweeps(ctx, tnh):
    """Dense Heisenberg N=20, m=32, cutoff 1e-10, 5 sweeps from a seeded random
    product state: the whole run on the GPU (FP64) and by the oracle."""
    from paper_2007_14822_gb300 import models as pm, synth
    from oracle import dmrg as D_, models as om
    from oracle.blocksparse import BlockTensor, trivial_index
    N = 20
    sweeps = [(32, 1e-10)] * 5
    vecs = synth.product_spinors(1, N, 2)
    host = pm.heisenberg(N)
    W = pm.to_device(host, qn=False)
    A = pm.product_vectors(W[0].inds[3], vecs)
    t0 = time.perf_counter()
    E, st = ctx.dmrg(W, A, host.start, host.done, [m for m, _ in sweeps], [c for _, c in sweeps],
                     krylov_dim=64, tol=1e-10)
    t_gpu = time.perf_counter() - t0
    mo = om.heisenberg_mpo(N)
    Wo = [BlockTensor.from_dense(w.to_dense(), [trivial_index(i.dim, i.arrow, nq=1) for i in w.inds]) for w in mo.W]
    site = trivial_index(2, +1, nq=1)
    t0 = time.perf_counter()
    Eo, _, _ = D_.dmrg(om.MPO(Wo, site, mo.start, mo.done), D_.product_mps_vectors(site, vecs), sweeps, 64, 1e-10)
    t_or = time.perf_counter() - t0
    return {"model": "dense Heisenberg N=20, m=32, cutoff 1e-10, 5 sweeps, random product start (seed 1)",
            "gpu_fp64_s": t_gpu, "oracle_s": t_or, "oracle_cores": blas_threads(), "energy": E,
            "energy_oracle": Eo, "dE_rel": abs(E - Eo) / abs(Eo)}


def oracle_bond(host, k=K_LANCZOS):
    """The same bond update by the FP64 oracle (numpy)."""
    from oracle import dmrg as D_
    from oracle.blocksparse import BlockTensor, IN, OUT, trivial_index
    a = trivial_index(M, OUT)
    s = trivial_index(D, OUT)
    wl, wr = trivial_index(W_DIM, IN), trivial_index(W_DIM, OUT)
    L = BlockTensor.from_dense(host["L"], [a.dag(), wl.dag(), a])
    R = BlockTensor.from_dense(host["R"], [a, wr.dag(), a.dag()])
    W = BlockTensor.from_dense(host["W"], [wl, wr, s.dag(), s])
    A1 = BlockTensor.from_dense(host["A1"], [a, s, a.dag()])
    A2 = BlockTensor.from_dense(host["A2"], [a, s, a.dag()])
    th = D_.theta(A1, A2)
    apply = lambda x: D_.heff_apply(L, W, W, R, x)
    E, x, res, nmv = D_.lanczos(apply, th, k, 0.0)
    E, r = D_.energy_residual(apply, x)
    U, S, V, err = D_.svd_trunc(x, 2, CUTOFF, MAXDIM)
    Lnew = D_.env_left(L, U, W)
    return E


def blas_threads():
    """Threads numpy's BLAS uses (what the oracle timing ran on)."""
    try:
        import threadpoolctl
        info = threadpoolctl.threadpool_info()
        if info:
            return max(i.get("num_threads", 1) for i in info)
    except ImportError:
        pass
    for var in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS"):
        if os.environ.get(var):
            return int(os.environ[var])
    return os.cpu_count()


def cpu_model():
    """Host CPU model and logical CPU count (lscpu; the machine type where absent)."""
    name = ""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name:"):
                name = ln.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return f"{name or platform.machine()}, {os.cpu_count()} logical CPUs"


# --------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu, self.rows, self.proc = gpu, [], None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4)
                          if len(r) > 5 + i and r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


# ------------------------------------------------------------ measurement
def l2_flush(torch, buf):
    buf.add_(1.0)


def time_steps(torch, bond, steps, flush, e2e=False):
    s = torch.cuda.current_stream()
    total = 0.0
    for _ in range(steps):
        l2_flush(torch, flush)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s)
        if e2e:
            bond.upload()
        bond.step(download=e2e)
        b.record(s)
        torch.cuda.synchronize()
        total += a.elapsed_time(b) / 1e3
    return total


def max_over_ranks(x, dist, device):
    """The job's time is the slowest rank's (all ranks call this)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# DRAM bytes (read + write) per launch of the headline's dominant kernel,
# from one ncu capture of the headline workload, with the SHA-256 of the
# kernel's sources (comments removed) at capture time: the figure is reported
# only while the sources' code is unchanged.
TRAFFIC = {
    # S1 79.02 + 96.44 MB, S4 324.22 + 16.00 MB (dram__bytes_read.sum + dram__bytes_write.sum of one
    # application of the headline workload): the mean of the two launches
    "gemm_tc_bf16x6": {"bytes_per_launch": (79.024128 + 96.43776 + 324.224 + 16.000256) / 2 * 1e6,
                       "source_sha": "da7071d557175e7db89371e98863734bd6f5f5beea36a42a5b877773c6f8222c"},
}


def source_sha(files):
    """SHA-256 of the sources' code: comments, blank lines and trailing
    blanks removed, so that editing a comment keeps the captured figures."""
    import hashlib
    import re
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_2007_14822_gb300", "csrc", f), encoding="utf-8") as fh:
            text = fh.read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        h.update("\n".join(ln.rstrip() for ln in text.splitlines() if ln.strip()).encode())
    return h.hexdigest()


KERNEL_SOURCES = {"gemm_tc": ["gemm_tc.cu", "ptx.cuh", "split.cuh", "tnh_internal.h"],
                  "heff_w12": ["gather.cu", "gather.h"], "heff_pack_x": ["gather.cu", "gather.h"]}


def kernel_traffic(name):
    t = TRAFFIC.get(name)
    if not t:
        return None
    srcs = next((v for k, v in KERNEL_SOURCES.items() if name.startswith(k)), None)
    if srcs is None or source_sha(srcs) != t["source_sha"]:
        return None
    return t["bytes_per_launch"]


HEAD = QN_CONFIGS[1]   # the J1-J2 cylinder, m = 2048
HEAD_CHOICES = {"cylinder": QN_CONFIGS[1], "u1": QN_CONFIGS[0], "hubbard": QN_CONFIGS[2]}


def time_heff_steps(torch, plan, x, y, steps, flush):
    """Device time of `steps` applications, L2 flushed before each."""
    s = torch.cuda.current_stream()
    total = 0.0
    for _ in range(steps):
        l2_flush(torch, flush)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s)
        plan.apply(x, y)
        b.record(s)
        torch.cuda.synchronize()
        total += a.elapsed_time(b) / 1e3
    return total


def time_heff_host_steps(torch, plan, xh, yh, steps, flush):
    """Time of `steps` calls of the C ABI's host-buffer product
    (tnh_heff_apply_host: x copied in from pinned host memory, the product,
    y copied out, the call returning when y is on the host), L2 flushed
    before each; CUDA events on the plan's stream around every call."""
    s = torch.cuda.current_stream()
    total = 0.0
    for _ in range(steps):
        l2_flush(torch, flush)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s)
        plan.apply_host(xh, yh)
        b.record(s)
        torch.cuda.synchronize()
        total += a.elapsed_time(b) / 1e3
    return total


def bench_bond_update(ctx, torch, tnh, steps, flush):
    """The dense m=256 bond update (every step of the hot path), device-timed."""
    host = host_inputs()
    bond = GpuBond(ctx, host)
    for _ in range(3):
        bond.step()
    torch.cuda.synchronize()
    t = time_steps(torch, bond, steps, flush)
    flops, heff_flops = step_flops()
    ctx.profile_begin()
    bond.step()
    prof = ctx.profile_end()
    return {"workload": "dense Heisenberg bond, m=256 w=5 d=2 (L/R 256x5x256, psi 256x2x2x256)",
            "step": f"theta + Lanczos {K_LANCZOS} matvecs BF16x6 + FP64 energy + FP64 Jacobi SVD "
                    f"(maxdim {MAXDIM}, cutoff {CUTOFF}) + FP64 env update",
            "flops_per_step": flops, "ms_per_step": t / steps * 1e3, "tflops": flops * steps / t / 1e12,
            "steps": steps, "kernels_per_step": {k: {"launches": v[0], "ms": v[1]} for k, v in prof.items()}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the extra workloads and the sweeps")
    ap.add_argument("--heff-workload", default="cylinder", choices=list(HEAD_CHOICES),
                    help="the block-sparse H_eff workload of the headline line (default: the J1-J2 cylinder at "
                         "m=2048, the configuration the metric is quoted on; the others are for profiling)")
    ap.add_argument("--oracle-matvec", default="heis,hub",
                    help="extra block-sparse workloads whose H_eff product is also timed on the oracle (comma "
                         "list of heis, hub; the Hubbard one takes tens of seconds on the host)")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", str(args.gpus)))
    head = HEAD_CHOICES[args.heff_workload]
    wname, wkind, wm, wrecipe, wseed = head
    where = "bulk sites 62/63 of the 6x24 cylinder, " if wkind == "cyl" else ""
    config = {"workload": f"H_eff.psi, {wname} ({where}seeded N(0,1) blocks, seed {wseed})",
              "step": "one BF16x6 application y = H_eff x (graph replay: pack psi, S1, fused W1.W2, S4)",
              "l2": "flushed before every timed step (256 MB write)",
              "parallelism": f"replicas x{world}"}

    if args.impl == "reference":
        if world > 1 and rank != 0:
            return
        args_o = qn_oracle_inputs(wkind, wm, wrecipe, wseed)
        from oracle import dmrg as D_
        flops = chain_flops(*args_o)
        cores = blas_threads()
        for _ in range(args.warmup):
            D_.heff_apply(*args_o)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            D_.heff_apply(*args_o)
        dt = (time.perf_counter() - t0) / args.steps
        val = flops / dt / 1e12
        config["flops_per_step"] = flops
        line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "TFLOP/s", "n_gpus": 0,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config,
                "cpu_baseline": {"value": val, "unit": "TFLOP/s", "cores": cores, "kind": "oracle",
                                 "sample": f"{args.steps} oracle H_eff products of the workload",
                                 "cpu": cpu_model()},
                "e2e": {"value": val, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    import torch
    from paper_2007_14822_gb300 import build, tnh
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    # one rank per node compiles (the ranks share the tree); the others wait
    if dist is None or local == 0:
        build.build()
    if dist:
        dist.barrier()
    ctx = tnh.Context(local)
    props = torch.cuda.get_device_properties(local)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    PEAKS.update(peaks)
    L, W1, W2, R, psi = qn_heff_inputs(wkind, wm, wrecipe, wseed)
    plan = ctx.heff_plan(L, W1, W2, R, psi, tnh.BF16x6)
    flops = plan.flops
    config["flops_per_step"] = flops
    config["psi_elems"] = plan.size
    x = psi.data.clone()
    y = torch.empty_like(x)
    flush = torch.zeros(32 * 1024 * 1024, dtype=torch.float64, device="cuda")   # 256 MB > L2
    for _ in range(max(args.warmup, 3)):
        plan.apply(x, y)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    with ClockSampler(local) as clk:
        t_dev = time_heff_steps(torch, plan, x, y, args.steps, flush)
    torch.cuda.synchronize()
    t_dev = max_over_ranks(t_dev, dist, "cuda")
    # end to end: psi from pinned host memory in, the product out, every step
    if dist:
        dist.barrier()
    xh = x.cpu().pin_memory()
    yh = torch.empty_like(xh).pin_memory()
    n_e2e = max(3, args.steps // 2)
    plan.apply_host(xh, yh)   # its first call makes the plan's device vectors
    t_e2e = max_over_ranks(time_heff_host_steps(torch, plan, xh, yh, n_e2e, flush), dist, "cuda") / n_e2e
    # per-kernel times over the same steps (direct launches, CUDA events on
    # the launching stream around every kernel)
    ctx.profile_begin()
    for _ in range(args.steps):
        l2_flush(torch, flush)
        plan.apply(x, y)
    prof = ctx.profile_end()
    launches = sum(v[0] for v in prof.values()) // args.steps
    name, (nl, ms) = max(prof.items(), key=lambda kv: kv[1][1])
    fd = plan.flops_detail
    pk = peaks.get("bf16_tflops")
    peak_src = "measured bf16 burst (MEASURED_PEAKS.json)"
    if pk is None:
        pk, peak_src = 1900.0, "fallback 1.9 PFLOP/s bf16"
    if name.startswith("gemm_tc"):
        # algorithmic flops of the launches of this kernel per step: S1 and S4
        alg = (fd["s1"] + fd["s4"]) * args.steps / nl
        achieved = alg / (ms / nl / 1e3) / 1e12
        roof = {"bound": "tensor", "achieved": achieved, "peak": pk, "unit": "TFLOP/s", "frac": achieved / pk,
                "traffic": kernel_traffic(name), "kernel": name, "peak_source": peak_src,
                "achieved_issued": 6 * achieved, "frac_issued": 6 * achieved / pk,
                "work": "algorithmic flops of S1 and S4 (2MNK per block pair) per launch; BF16x6 issues 6 bf16 "
                        "products per algorithmic flop (achieved_issued / frac_issued)"}
    else:
        hbm = peaks.get("hbm_gbs", 6800.0)
        roof = {"bound": "hbm", "achieved": None, "peak": hbm, "unit": "GB/s", "frac": None,
                "traffic": kernel_traffic(name), "kernel": name, "peak_source": "measured copy (MEASURED_PEAKS.json)"}
    roof["kernel_ms_per_launch"] = ms / nl
    roof["launches_per_step"] = nl / args.steps
    value = world * flops * args.steps / t_dev / 1e12
    line = {"metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_dev / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16x6 (fp32 accumulate)", "data": "synthetic",
            "config": config,
            "e2e": {"value": world * flops / t_e2e / 1e12, "unit": "TFLOP/s",
                    "h2d_bytes_per_step": int(x.numel()) * 8, "d2h_bytes_per_step": int(y.numel()) * 8},
            "gpu_launches": launches * args.steps, "clocks": clk.summary(), "roofline": roof,
            "sm_count": props.multi_processor_count,
            "kernels_per_step": {k: {"launches": v[0] / args.steps, "ms": v[1] / args.steps}
                                 for k, v in prof.items()}}
    # the FP64 product of the same plan (the plain FP64 GPU path)
    for _ in range(2):
        plan.apply(x, y, tnh.FP64)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(3):
        plan.apply(x, y, tnh.FP64)
    b.record()
    torch.cuda.synchronize()
    t64 = a.elapsed_time(b) / 1e3 / 3
    line["fp64"] = {"ms": t64 * 1e3, "tflops": flops / t64 / 1e12, "speedup_bf16x6": t64 / (t_dev / args.steps)}
    plan.free()
    del L, W1, W2, R, psi, x, y
    torch.cuda.empty_cache()
    # the other workloads, the sweeps and the oracle are reported at N=1 only
    # (at N>1 they would hold every GPU while rank 0 alone works)
    if rank == 0 and world == 1 and not args.no_extra:
        line["bond_update_m256"] = bench_bond_update(ctx, torch, tnh, 5, flush)
        line["heff_qn"] = bench_qn_heff(ctx, torch, tnh, tuple(k for k in args.oracle_matvec.split(",") if k))
        line["sweep"] = bench_sweeps(ctx, tnh)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # a bounded sample: whole oracle H_eff products of the workload, about 10 s
        from oracle import dmrg as D_
        args_o = qn_oracle_inputs(wkind, wm, wrecipe, wseed)
        n, t0 = 0, time.perf_counter()
        while True:
            D_.heff_apply(*args_o)
            n += 1
            dt = time.perf_counter() - t0
            if dt >= 10.0 or n >= 30:
                break
        line["cpu_baseline"] = {"value": n * flops / dt / 1e12, "unit": "TFLOP/s", "cores": blas_threads(),
                                "kind": "oracle",
                                "sample": f"{n} oracle H_eff products of the same workload ({dt:.1f} s)",
                                "cpu": cpu_model()}
    if rank == 0:
        print(json.dumps(line))
    ctx.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
