"""GPU parity of the labelled contraction, H_eff, the environment update and the
eigensolver against the FP64 oracle (calls go through the C ABI)."""
import numpy as np
import pytest

import helpers as H
from oracle import dmrg as D
from oracle.blocksparse import BlockTensor, contract as ocontract

pytestmark = pytest.mark.gpu

# tolerances (relative, norm-wise over the whole output)
TOL = {"fp64": 1e-12, "bf16x6": 1e-6}


@pytest.fixture(scope="module")
def ctx():
    import torch
    from paper_2007_14822_gb300 import build, tnh
    assert torch.cuda.is_available()
    build.build()
    c = tnh.Context(0)
    yield c
    c.close()


def prec(name):
    from paper_2007_14822_gb300 import tnh
    return tnh.PRECISION[name]


# ------------------------------------------------------------ contraction
def _qn_index(rng, ns, arrow, label, maxd=4):
    from paper_2007_14822_gb300.tnh import Index
    return Index([((q,), int(rng.integers(1, maxd + 1))) for q in range(-(ns // 2), ns - ns // 2)],
                 arrow, label)


@pytest.mark.parametrize("p", ["fp64", "bf16x6"])
def test_contract_block_sparse(ctx, p):
    from paper_2007_14822_gb300.tnh import Tensor
    rng = np.random.default_rng(5)
    for trial in range(4):
        i = _qn_index(rng, 3, +1, 1)
        j = _qn_index(rng, 4, +1, 2)
        k = _qn_index(rng, 3, +1, 3)
        l = _qn_index(rng, 2, +1, 4)
        A, Ao = H.random_pair([i, j, k], (0,), 10 + trial, "A")
        B, Bo = H.random_pair([k.dag(), l, j.dag()], (1,), 10 + trial, "B")
        # output in a permuted order: (l, i)
        Cd = Tensor([l, i], (1,))
        ctx.contract(A, B, Cd, prec(p))
        want = ocontract(Ao.relabel([1, 2, 3]), Bo.relabel([3, 4, 2]), out_labels=[4, 1])
        scale = ocontract(H.abs_tensor(Ao).relabel([1, 2, 3]), H.abs_tensor(Bo).relabel([3, 4, 2]),
                          out_labels=[4, 1])
        H.assert_parity(H.to_oracle(Cd), want, scale, p, TOL[p] * 10)


def test_contract_outer_and_full(ctx):
    from paper_2007_14822_gb300.tnh import Index, Tensor
    a = Index.dense(5, +1, 1)
    b = Index.dense(7, +1, 2)
    A, Ao = H.random_pair([a], (0,), 1, "a")
    B, Bo = H.random_pair([b], (0,), 1, "b")
    C = Tensor([b, a], (0,))
    ctx.contract(A, B, C)
    np.testing.assert_allclose(C.data.cpu().numpy().reshape(7, 5),
                               np.outer(Bo.to_dense(), Ao.to_dense()), rtol=1e-14)
    B2, B2o = H.random_pair([a.dag()], (0,), 2, "c")
    S = Tensor([], (0,))
    ctx.contract(A, B2, S)
    assert abs(S.data.cpu().item() - float(Ao.to_dense() @ B2o.to_dense())) < 1e-13


def test_contract_rejects_equal_arrows(ctx):
    from paper_2007_14822_gb300.tnh import Index, Tensor, TnhError
    a = Index([((0,), 2), ((1,), 3)], +1, 1)
    A, _ = H.random_pair([a], (0,), 1, "x")
    B, _ = H.random_pair([a], (0,), 2, "y")
    with pytest.raises(TnhError) as e:
        ctx.contract(A, B, Tensor([], (0,)))
    assert e.value.code == 3


def test_contract_with_nothing_to_contract_gives_zero(ctx):
    # degenerate block-sparse products; C starts as NaN and must come out 0:
    # (1) A has no allowed block (odd flux, even charges);
    # (2) A and B hold blocks, but no pair agrees on the contracted sector
    #     (each keeps one of its two allowed blocks), as the oracle finds
    import torch
    from paper_2007_14822_gb300.tnh import Index, Tensor
    i = Index([((0,), 3), ((-2,), 2)], +1, 1)
    k = Index([((0,), 2), ((2,), 4)], +1, 2)
    l = Index([((0,), 5), ((2,), 3)], +1, 3)
    A0 = Tensor([i, k], (1,))
    assert A0.blocks == []
    B, _ = H.random_pair([k.dag(), l], (0,), 3, "B")
    A1 = Tensor([i, k], (0,), blocks=[(0, 0)], offsets=[0]).fill(lambda key, shp: synth_block(4, "A", key, shp))
    B1 = Tensor([k.dag(), l], (0,), blocks=[(1, 1)], offsets=[0]).fill(lambda key, shp: synth_block(4, "B", key, shp))
    want = ocontract(H.to_oracle(A1).relabel([1, 2]), H.to_oracle(B1).relabel([2, 3]), out_labels=[3, 1])
    assert all(not np.any(v) for v in want.blocks.values())
    for p in ("fp64", "bf16x6"):
        for A_, B_ in ((A0, B), (A1, B1)):
            Cd = Tensor([l, i], (0,))
            assert Cd.blocks == [(0, 0), (1, 1)]
            Cd.data.fill_(float("nan"))
            ctx.contract(A_, B_, Cd, prec(p))
            assert torch.all(Cd.data == 0), p


def synth_block(seed, tag, key, shp):
    from paper_2007_14822_gb300 import synth
    return synth.block_gaussian(seed, tag, key, shp)


# ------------------------------------------------------------------ H_eff
def heff_scale(Lo, W1o, W2o, Ro, xo):
    """The oracle's H_eff on the absolute values of every input: the sum of
    |terms| of each output element, the scale of its rounding error."""
    A = H.abs_tensor
    return D.heff_apply(A(Lo), A(W1o), A(W2o), A(Ro), A(xo))


def _heff_case(ctx, m, nsect, p, seed=7, maxd=None):
    """One product against the oracle; asserts the norm-wise, per-block and
    per-element bounds and returns the norm-wise error and the plan."""
    d = H.heff_inputs(m, None, seed, nsect=nsect, maxd=maxd)
    plan = ctx.heff_plan(d["L"], d["W"], d["W"], d["R"], d["psi"], prec(p))
    import torch
    y = torch.zeros_like(d["psi"].data)
    plan.apply(d["psi"].data, y)
    ytens = d["psi"].with_inds(d["psi"].inds)
    ytens.data = y
    got = H.to_oracle(ytens)
    want = D.heff_apply(d["Lo"], d["Wo"], d["Wo"], d["Ro"], d["psio"])
    scale = heff_scale(d["Lo"], d["Wo"], d["Wo"], d["Ro"], d["psio"])
    err, _ = H.assert_parity(got, want, scale, p, TOL[p])
    return err, plan


@pytest.mark.parametrize("m", [1, 3, 24, 130])
@pytest.mark.parametrize("p", ["fp64", "bf16x6"])
def test_heff_dense(ctx, m, p):
    err, plan = _heff_case(ctx, m, 1, p)
    assert err < TOL[p], err
    # algorithmic flops: S1+S4 = 4 w d^2 m^3, S2+S3 = 4 w^2 d^3 m^2 (MPO counted dense)
    w, dd = 5, 2
    assert plan.flops == pytest.approx(4 * w * dd * dd * m ** 3 + 4 * w * w * dd ** 3 * m * m)


@pytest.mark.parametrize("m,nsect,maxd", [(12, 5, 4), (64, 9, 16), (300, 15, 60)])
@pytest.mark.parametrize("p", ["fp64", "bf16x6"])
def test_heff_qn(ctx, m, nsect, maxd, p):
    err, _ = _heff_case(ctx, m, nsect, p, maxd=maxd)
    assert err < TOL[p], err


@pytest.mark.parametrize("p", ["fp64", "bf16x6"])
def test_heff_apply_host_buffers(ctx, p):
    # the host-buffer entry point: x copied in, product, y copied out; the
    # result is the device product's, bit for bit, within the oracle bound,
    # in pinned and pageable memory, and with y the same array as x
    import torch
    d = H.heff_inputs(64, None, 11, nsect=9, maxd=16)
    plan = ctx.heff_plan(d["L"], d["W"], d["W"], d["R"], d["psi"], prec(p))
    ydev = torch.zeros_like(d["psi"].data)
    plan.apply(d["psi"].data, ydev)
    want = ydev.cpu()
    for pinned in (True, False):
        xh = d["psi"].data.cpu()
        yh = torch.full_like(xh, float("nan"))
        if pinned:
            xh, yh = xh.pin_memory(), yh.pin_memory()
        for _ in range(2):
            plan.apply_host(xh, yh)
            assert torch.equal(yh, want)
        inplace = xh.clone()
        plan.apply_host(inplace, inplace)
        assert torch.equal(inplace, want)
    ytens = d["psi"].with_inds(d["psi"].inds)
    ytens.data = yh.cuda()
    scale = heff_scale(d["Lo"], d["Wo"], d["Wo"], d["Ro"], d["psio"])
    H.assert_parity(H.to_oracle(ytens), D.heff_apply(d["Lo"], d["Wo"], d["Wo"], d["Ro"], d["psio"]), scale, p,
                    TOL[p])
    with pytest.raises(TypeError):
        plan.apply_host(d["psi"].data, yh)


@pytest.mark.parametrize("p", ["fp64", "bf16x6"])
@pytest.mark.parametrize("m,nsect,maxd,split", [(40, 7, 12, None), (300, 3, 200, "2,4")])
def test_heff_graph_replay_with_new_buffers(ctx, p, m, nsect, maxd, split, monkeypatch):
    # the first application launches directly, the second captures a CUDA
    # graph, later ones replay it with the x / y arguments patched: every
    # call must give the oracle's result for its own input (also when the
    # last launch is a K-split reduction: forced here for the split modes;
    # the FP64 GEMM splits the long K of the few-tile m=300 case itself)
    import torch
    if split:
        monkeypatch.setenv("TNH_HEFF_SPLIT", split)
    d = H.heff_inputs(m, None, 5, nsect=nsect, maxd=maxd)
    plan = ctx.heff_plan(d["L"], d["W"], d["W"], d["R"], d["psi"], prec(p))
    from oracle.blocksparse import BlockTensor
    xs = [d["psi"].data.clone() * (1.0 + 0.5 * i) for i in range(3)]
    xs[2] = torch.flip(xs[2], [0])
    ys = [torch.full_like(d["psi"].data, float("nan")) for _ in range(2)]
    for call, (xi, yi) in enumerate([(0, 0), (0, 1), (1, 1), (2, 0), (1, 0), (2, 1)]):
        x, y = xs[xi], ys[yi]
        plan.apply(x, y)
        xt = d["psi"].with_inds(d["psi"].inds)
        xt.data = x
        yt = d["psi"].with_inds(d["psi"].inds)
        yt.data = y
        xo = H.to_oracle(xt)
        want = D.heff_apply(d["Lo"], d["Wo"], d["Wo"], d["Ro"], xo)
        scale = heff_scale(d["Lo"], d["Wo"], d["Wo"], d["Ro"], xo)
        H.assert_parity(H.to_oracle(yt), want, scale, p, TOL[p])


@pytest.mark.parametrize("split", ["2,8", "4,3", "1,2"])
@pytest.mark.parametrize("m,nsect,maxd", [(130, 1, 130), (300, 15, 60)])
def test_heff_k_split_matches_oracle(ctx, split, m, nsect, maxd, monkeypatch):
    # the plan autotuner may cut the S1 / S4 GEMMs into K ranges with float32
    # partials and a reduction; force each shape of it and check the result
    monkeypatch.setenv("TNH_HEFF_SPLIT", split)
    err, plan = _heff_case(ctx, m, nsect, "bf16x6", maxd=maxd)
    assert err < TOL["bf16x6"], err


@pytest.mark.parametrize("tiles,split", [("1,1", "1,1"), ("2,2", "1,1"), ("2,1", "2,4"), ("0,2", "1,2")])
@pytest.mark.parametrize("m,nsect,maxd", [(300, 15, 60), (160, 9, 90), (70, 1, 70)])
def test_heff_tile_widths_match_oracle(ctx, tiles, split, m, nsect, maxd, monkeypatch):
    # N tiles of 64 and 32 columns (slices of the 128-row packed B tiles),
    # alone and with K splits, on blocks of every width
    monkeypatch.setenv("TNH_HEFF_TILES", tiles)
    monkeypatch.setenv("TNH_HEFF_SPLIT", split)
    err, plan = _heff_case(ctx, m, nsect, "bf16x6", maxd=maxd)
    t = plan.tuning
    assert (t["tiles_s1"], t["tiles_s4"]) == tuple(int(x) for x in tiles.split(",")) and not t["measured"]


def test_heff_tuning_cache_file(ctx, tmp_path, monkeypatch):
    # the autotuner's choices go to the TNH_TUNE_CACHE file; a new context
    # reads them back for a plan of the same shapes instead of timing again
    from paper_2007_14822_gb300 import tnh
    path = tmp_path / "tune.txt"
    monkeypatch.setenv("TNH_TUNE_CACHE", str(path))
    monkeypatch.setenv("TNH_HEFF_STRATEGY", "0")
    monkeypatch.delenv("TNH_HEFF_SPLIT", raising=False)
    monkeypatch.delenv("TNH_HEFF_TILES", raising=False)
    d = H.heff_inputs(96, None, 11, nsect=9, maxd=24)
    c1 = tnh.Context(0)
    p1 = c1.heff_plan(d["L"], d["W"], d["W"], d["R"], d["psi"], prec("bf16x6"))
    t1 = p1.tuning
    assert t1["measured"]
    lines = path.read_text().splitlines()
    assert len(lines) == 1 and lines[0].startswith("heff ")
    c1.close()
    c2 = tnh.Context(0)
    p2 = c2.heff_plan(d["L"], d["W"], d["W"], d["R"], d["psi"], prec("bf16x6"))
    t2 = p2.tuning
    assert not t2["measured"] and {k: v for k, v in t2.items() if k != "measured"} == \
        {k: v for k, v in t1.items() if k != "measured"}
    y = __import__("torch").zeros_like(d["psi"].data)
    p2.apply(d["psi"].data, y)
    yt = d["psi"].with_inds(d["psi"].inds)
    yt.data = y
    want = D.heff_apply(d["Lo"], d["Wo"], d["Wo"], d["Ro"], d["psio"])
    assert H.rel_err(H.to_oracle(yt), want) < TOL["bf16x6"]
    c2.close()


def test_heff_config2_full_size(ctx):
    # dense m=256, w=5, d=2: L/R (256,5,256), psi (256,2,2,256), Gaussian, seeded
    for p in ("fp64", "bf16x6"):
        err, _ = _heff_case(ctx, 256, 1, p, seed=2)
        assert err < TOL[p], (p, err)


def _hub_link(rng, arrow):
    from paper_2007_14822_gb300.tnh import Index
    # (N, 2Sz) charges with N - 2Sz even, as on a Hubbard link
    secs = [((n, sz), int(rng.integers(1, 6))) for n in range(-2, 3) for sz in range(-2, 3) if (n - sz) % 2 == 0]
    return Index(secs, arrow)


@pytest.mark.parametrize("model,j", [("j1j2", 0), ("j1j2", 3), ("j1j2", 6), ("hubbard", 2)])
@pytest.mark.parametrize("p", ["fp64", "bf16x6"])
def test_heff_distinct_mpo_tensors(ctx, model, j, p):
    # W1 != W2 (long-range J1-J2 MPO incl. the boundary sites; Hubbard with
    # U(1) x U(1) charges and d = 4), random environments on a QN link
    import torch
    from paper_2007_14822_gb300 import models as pm
    rng = np.random.default_rng(17 + j)
    if model == "j1j2":
        mpo = pm.to_device(pm.j1j2_chain(8, 1.0, 0.5), qn=True)
        a = H.link_index(36, 7, 9, +1)
    else:
        mpo = pm.to_device(pm.hubbard(6, 1.0, 4.0), qn=True)
        a = _hub_link(rng, +1)
    W1, W2 = mpo[j], mpo[j + 1]
    L, Lo = H.random_pair([a.dag(), W1.inds[0].dag(), a], None, 21 + j, "L")
    R, Ro = H.random_pair([a, W2.inds[1].dag(), a.dag()], None, 22 + j, "R")
    psi, psio = H.random_pair([a, W1.inds[3], W2.inds[3], a.dag()], None, 23 + j, "psi")
    plan = ctx.heff_plan(L, W1, W2, R, psi, prec(p))
    y = torch.zeros_like(psi.data)
    plan.apply(psi.data, y)
    yt = psi.with_inds(psi.inds)
    yt.data = y
    want = D.heff_apply(Lo, H.to_oracle(W1), H.to_oracle(W2), Ro, psio)
    scale = heff_scale(Lo, H.to_oracle(W1), H.to_oracle(W2), Ro, psio)
    H.assert_parity(H.to_oracle(yt), want, scale, p, TOL[p])


@pytest.mark.parametrize("p,tol", [("bf16x3", 1e-3), ("bf16", 2e-2)])
def test_heff_low_precision_modes_error_bounded(ctx, p, tol):
    # norm-wise only: these modes are not meant to meet the split-mode bounds
    import torch
    d = H.heff_inputs(64, None, 7, nsect=1)
    plan = ctx.heff_plan(d["L"], d["W"], d["W"], d["R"], d["psi"], prec(p))
    y = torch.zeros_like(d["psi"].data)
    plan.apply(d["psi"].data, y)
    yt = d["psi"].with_inds(d["psi"].inds)
    yt.data = y
    want = D.heff_apply(d["Lo"], d["Wo"], d["Wo"], d["Ro"], d["psio"])
    err = H.rel_err(H.to_oracle(yt), want)
    assert err < tol, err


# ------------------------------------------------------------ environments
@pytest.mark.parametrize("direction", [1, -1])
@pytest.mark.parametrize("p", ["fp64", "bf16x6"])
@pytest.mark.parametrize("nsect", [1, 7])
def test_env_update(ctx, direction, p, nsect):
    from paper_2007_14822_gb300.tnh import Tensor
    m = 40
    d = H.heff_inputs(m, None, 9, nsect=nsect, maxd=12)
    a = d["psi"].inds[0]
    s = d["psi"].inds[1]
    # MPS tensor A[a, s, b] with b = a-link shifted by one site
    A, Ao = H.random_pair([a, s, a.dag()], None, 11, "A")
    if direction == 1:
        E, Eo = d["L"], d["Lo"]
        out = Tensor(list(d["L"].inds), (0,))
        ctx.env_update(1, E, A, d["W"], out, prec(p))
        f = D.env_left
    else:
        E, Eo = d["R"], d["Ro"]
        out = Tensor(list(d["R"].inds), (0,))
        ctx.env_update(-1, E, A, d["W"], out, prec(p))
        f = D.env_right
    want = f(Eo, Ao, d["Wo"])
    scale = f(H.abs_tensor(Eo), H.abs_tensor(Ao), H.abs_tensor(d["Wo"]))
    H.assert_parity(H.to_oracle(out), want, scale, p, TOL[p])


# -------------------------------------------------------------- eigsolve
@pytest.mark.parametrize("p", ["fp64", "bf16x6"])
def test_eigsolve_dense(ctx, p):
    m = 20
    d = H.heff_inputs(m, None, 13, nsect=1, symmetric=True)
    plan = ctx.heff_plan(d["L"], d["W"], d["W"], d["R"], d["psi"], prec(p))
    Hm = D.heff_dense_matrix(d["Lo"], d["Wo"], d["Wo"], d["Ro"], d["psio"])
    assert np.abs(Hm - Hm.T).max() < 1e-10 * np.abs(Hm).max()
    w, v = np.linalg.eigh(Hm)
    psi = d["psi"].data.clone()
    E, r, k = plan.eigsolve(psi, krylov_dim=200, tol=1e-10 if p == "fp64" else 1e-6)
    scale = abs(w[0])
    assert abs(E - w[0]) < 1e-9 * scale, (E, w[0])
    x = psi.cpu().numpy()
    ov = abs(float(x @ v[:, 0]))
    assert ov > 1 - (1e-10 if p == "fp64" else 1e-7)


@pytest.mark.parametrize("m,k", [(20, 6), (1, 8)])
def test_eigsolve_fixed_length_matches_oracle_lanczos(ctx, m, k):
    # tol = 0: exactly k steps (the tridiagonal problem is solved only at the
    # end) unless the Krylov space is exhausted first (m = 1: dim 4 < k)
    d = H.heff_inputs(m, None, 13, nsect=1, symmetric=True)
    plan = ctx.heff_plan(d["L"], d["W"], d["W"], d["R"], d["psi"], prec("fp64"))
    psi = d["psi"].data.clone()
    E, r, nmv = plan.eigsolve(psi, krylov_dim=k, tol=0.0)
    apply = lambda x: D.heff_apply(d["Lo"], d["Wo"], d["Wo"], d["Ro"], x)
    Eo, xo, res, nmo = D.lanczos(apply, d["psio"], k, 0.0)
    assert nmv == nmo
    assert abs(E - Eo) < 1e-10 * abs(Eo)


# ------------------------------------------- sums of MPOs, projectors
@pytest.mark.parametrize("p", ["fp64", "bf16x6"])
@pytest.mark.parametrize("nsect", [1, 7])
def test_heff_plan_sum_matches_sum_of_terms(ctx, p, nsect):
    # H = H_J1J2 + H_Heisenberg (different MPO link dimensions): one plan of
    # the terms' direct sum against the oracle's sum of the two products
    import torch
    from paper_2007_14822_gb300 import models as pm
    j = 3
    terms = [pm.to_device(pm.j1j2_chain(8, 1.0, 0.5), qn=True), pm.to_device(pm.heisenberg(8), qn=True)]
    a = H.link_index(40, nsect, 12 if nsect > 1 else 40, +1)
    Ls, Rs, Los, Ros, W1s, W2s = [], [], [], [], [], []
    for t, mpo in enumerate(terms):
        W1, W2 = mpo[j], mpo[j + 1]
        L, Lo = H.random_pair([a.dag(), W1.inds[0].dag(), a], None, 31 + t, "L")
        R, Ro = H.random_pair([a, W2.inds[1].dag(), a.dag()], None, 41 + t, "R")
        Ls.append(L), Rs.append(R), Los.append(Lo), Ros.append(Ro), W1s.append(W1), W2s.append(W2)
    psi, psio = H.random_pair([a, W1s[0].inds[3], W2s[0].inds[3], a.dag()], None, 51, "psi")
    plan = ctx.heff_plan_sum(Ls, W1s, W2s, Rs, psi, prec(p))
    y = torch.zeros_like(psi.data)
    plan.apply(psi.data, y)
    plan.apply(psi.data, y)      # second call: graph capture
    yt = psi.with_inds(psi.inds)
    yt.data = y
    want = scale = None
    for t in range(2):
        wt = D.heff_apply(Los[t], H.to_oracle(W1s[t]), H.to_oracle(W2s[t]), Ros[t], psio)
        st = heff_scale(Los[t], H.to_oracle(W1s[t]), H.to_oracle(W2s[t]), Ros[t], psio)
        want = wt if want is None else want.axpy(1.0, wt)
        scale = st if scale is None else scale.axpy(1.0, st)
    H.assert_parity(H.to_oracle(yt), want, scale, p, TOL[p])
    # the flops are the two terms' flops
    f = [ctx.heff_plan(Ls[t], W1s[t], W2s[t], Rs[t], psi, prec(p)).flops for t in range(2)]
    assert plan.flops == pytest.approx(sum(f))


@pytest.mark.parametrize("p", ["fp64", "bf16x6"])
def test_heff_projectors_added(ctx, p):
    # y = H_eff x + w sum_i phi_i <phi_i, x> with two random phi
    import torch
    d = H.heff_inputs(24, None, 9, nsect=5, maxd=8)
    plan = ctx.heff_plan(d["L"], d["W"], d["W"], d["R"], d["psi"], prec(p))
    n = plan.size
    phis = [H.random_pair(d["psi"].inds, d["psi"].flux, 60 + i, "phi") for i in range(2)]
    phi = torch.stack([t.data[:n] for t, _ in phis])
    w = 3.5
    plan.set_projectors(phi, w)
    y = torch.zeros_like(d["psi"].data)
    for _ in range(3):           # direct, captured, replayed
        plan.apply(d["psi"].data, y)
    yt = d["psi"].with_inds(d["psi"].inds)
    yt.data = y
    want = D.heff_apply(d["Lo"], d["Wo"], d["Wo"], d["Ro"], d["psio"])
    scale0 = heff_scale(d["Lo"], d["Wo"], d["Wo"], d["Ro"], d["psio"])
    scale = scale0.copy()
    for _, po in phis:
        want = want.axpy(w * po.vdot(d["psio"]), po)
        scale = scale.axpy(w * H.abs_tensor(po).vdot(H.abs_tensor(d["psio"])), H.abs_tensor(po))
    H.assert_parity(H.to_oracle(yt), want, scale, p, TOL[p])
    # removing them gives H_eff alone
    plan.set_projectors(None, 0.0)
    plan.apply(d["psi"].data, y)
    yt.data = y
    want0 = D.heff_apply(d["Lo"], d["Wo"], d["Wo"], d["Ro"], d["psio"])
    H.assert_parity(H.to_oracle(yt), want0, scale0, p, TOL[p])


# ------------------------------------------------- diagonal and Davidson
@pytest.mark.parametrize("m,nsect,maxd", [(6, 1, 6), (12, 5, 4)])
def test_heff_diag_matches_dense_matrix(ctx, m, nsect, maxd):
    import torch
    d = H.heff_inputs(m, None, 19, nsect=nsect, maxd=maxd)
    plan = ctx.heff_plan(d["L"], d["W"], d["W"], d["R"], d["psi"], prec("fp64"))
    out = torch.zeros(plan.size, dtype=torch.float64, device="cuda")
    plan.diag(out)
    Hm = D.heff_dense_matrix(d["Lo"], d["Wo"], d["Wo"], d["Ro"], d["psio"])
    np.testing.assert_allclose(out.cpu().numpy(), np.diag(Hm), rtol=0, atol=1e-12 * np.abs(Hm).max())


def test_heff_diag_distinct_mpo_qn(ctx):
    # W1 != W2 on a QN link (J1-J2 long-range MPO, sites 3 and 4)
    import torch
    from paper_2007_14822_gb300 import models as pm
    mpo = pm.to_device(pm.j1j2_chain(8, 1.0, 0.5), qn=True)
    W1, W2 = mpo[3], mpo[4]
    a = H.link_index(10, 3, 4, +1)
    L, Lo = H.random_pair([a.dag(), W1.inds[0].dag(), a], None, 71, "L")
    R, Ro = H.random_pair([a, W2.inds[1].dag(), a.dag()], None, 72, "R")
    psi, psio = H.random_pair([a, W1.inds[3], W2.inds[3], a.dag()], None, 73, "psi")
    plan = ctx.heff_plan(L, W1, W2, R, psi, prec("fp64"))
    out = torch.zeros(plan.size, dtype=torch.float64, device="cuda")
    plan.diag(out)
    Hm = D.heff_dense_matrix(Lo, H.to_oracle(W1), H.to_oracle(W2), Ro, psio)
    np.testing.assert_allclose(out.cpu().numpy(), np.diag(Hm), rtol=0, atol=1e-12 * np.abs(Hm).max())


@pytest.mark.parametrize("p", ["fp64", "bf16x6"])
@pytest.mark.parametrize("nsect", [1, 5])
def test_davidson_matches_eigh(ctx, p, nsect):
    m = 20 if nsect == 1 else 24
    d = H.heff_inputs(m, None, 13, nsect=nsect, maxd=8 if nsect > 1 else None, symmetric=True)
    plan = ctx.heff_plan(d["L"], d["W"], d["W"], d["R"], d["psi"], prec(p))
    Hm = D.heff_dense_matrix(d["Lo"], d["Wo"], d["Wo"], d["Ro"], d["psio"])
    w, v = np.linalg.eigh(0.5 * (Hm + Hm.T))
    psi = d["psi"].data.clone()
    E, r, k = plan.eigsolve(psi, krylov_dim=48, tol=1e-9 if p == "fp64" else 1e-6, method="davidson")
    scale = abs(w[0])
    assert abs(E - w[0]) < 1e-9 * scale, (E, w[0], k)
    x = psi[:plan.size].cpu().numpy()
    assert abs(float(x @ v[:, 0])) > 1 - (1e-10 if p == "fp64" else 1e-7)
    assert r < (1e-8 if p == "fp64" else 1e-5) * scale


# ------------------------------------------- block-sparse workloads, full size
@pytest.mark.parametrize("which", [0, 1, 2])
def test_heff_qn_workloads_full_size(ctx, which):
    # the bench's block-sparse H_eff workloads at full size (U(1) m=1024;
    # J1-J2 cylinder m=2048, w=26; U(1)xU(1) Hubbard m=4096, d=4), the plan
    # the bench times (BF16x6 after graph capture, and its FP64 product), each
    # against the oracle on the full input: norm-wise, per block and per
    # element (the oracle takes up to tens of seconds for the Hubbard one)
    import torch
    import bench
    name, kind, m, recipe, seed = bench.QN_CONFIGS[which]
    L, W1, W2, R, psi = bench.qn_heff_inputs(kind, m, recipe, seed)
    plan = ctx.heff_plan(L, W1, W2, R, psi, prec("bf16x6"))
    x = psi.data.clone()
    y64 = torch.zeros_like(x)
    ymx = torch.zeros_like(x)
    for _ in range(3):
        plan.apply(x, ymx)
    plan.apply(x, y64, prec("fp64"))
    args = [H.to_oracle(T) for T in (L, W1, W2, R)]
    if which != 2:   # the host count of the Hubbard chain enumerates for tens of seconds
        assert plan.flops == pytest.approx(bench.chain_flops(*args, H.to_oracle(psi)), rel=1e-12)
    want = D.heff_apply(*args, H.to_oracle(psi))
    scale = heff_scale(*args, H.to_oracle(psi))
    results = [("fp64", y64), ("bf16x6", ymx)]
    # the other S4 form of the split precision (the tuned plan used one)
    import os
    os.environ["TNH_HEFF_FUSED"] = "0" if plan.tuning["fused_s4"] else "1"
    try:
        plan2 = ctx.heff_plan(L, W1, W2, R, psi, prec("bf16x6"))
    finally:
        del os.environ["TNH_HEFF_FUSED"]
    assert plan2.tuning["fused_s4"] != plan.tuning["fused_s4"]
    y2 = torch.zeros_like(x)
    for _ in range(3):
        plan2.apply(x, y2)
    results.append(("bf16x6", y2))
    for p, y in results:
        yt = psi.with_inds(psi.inds)
        yt.data = y
        err, rep = H.assert_parity(H.to_oracle(yt), want, scale, p, TOL[p])
        print(name, p, "norm-wise", err, "worst block", rep["block"], "worst element", rep["elem"])


@pytest.mark.parametrize("strategy", ["0", "1"])
@pytest.mark.parametrize("p", ["fp64", "bf16x6"])
@pytest.mark.parametrize("m,nsect,maxd", [(64, 9, 16), (300, 15, 60), (40, 1, 40)])
def test_heff_block_strategies_match_oracle(ctx, strategy, p, m, nsect, maxd, monkeypatch):
    # combine-then-contract and block pairs (Sec. 9.4), each forced, against
    # the oracle: norm-wise, per block and per element
    monkeypatch.setenv("TNH_HEFF_STRATEGY", strategy)
    err, plan = _heff_case(ctx, m, nsect, p, maxd=maxd)
    t = plan.tuning
    assert t["strategy"] == int(strategy) and not t["strategy_measured"]


@pytest.mark.parametrize("strategy", ["0", "1"])
@pytest.mark.parametrize("split", ["1,1", "1,3", "2,8"])
@pytest.mark.parametrize("m,nsect,maxd", [(64, 9, 16), (300, 15, 60), (70, 1, 70), (200, 5, 90)])
def test_heff_s4_forming_its_operand_matches_oracle(ctx, strategy, split, m, nsect, maxd, monkeypatch):
    # S4 forms its operand A from T1 inside the GEMM (the W1.W2 step fused),
    # alone, with K splits and with both block strategies, against the oracle
    monkeypatch.setenv("TNH_HEFF_FUSED", "1")
    monkeypatch.setenv("TNH_HEFF_SPLIT", split)
    monkeypatch.setenv("TNH_HEFF_STRATEGY", strategy)
    err, plan = _heff_case(ctx, m, nsect, "bf16x6", maxd=maxd)
    assert plan.tuning["fused_s4"]


@pytest.mark.parametrize("model,j", [("j1j2", 0), ("j1j2", 3), ("hubbard", 2)])
def test_heff_s4_forming_its_operand_distinct_mpo_tensors(ctx, model, j, monkeypatch):
    monkeypatch.setenv("TNH_HEFF_FUSED", "1")
    test_heff_distinct_mpo_tensors(ctx, model, j, "bf16x6")


def test_heff_s4_forming_its_operand_graph_replay(ctx, monkeypatch):
    monkeypatch.setenv("TNH_HEFF_FUSED", "1")
    test_heff_graph_replay_with_new_buffers(ctx, "bf16x6", 40, 7, 12, None, monkeypatch)
    test_heff_graph_replay_with_new_buffers(ctx, "bf16x6", 300, 3, 200, "2,4", monkeypatch)


@pytest.mark.parametrize("model,j", [("j1j2", 3), ("hubbard", 2)])
def test_heff_block_pairs_distinct_mpo_tensors(ctx, model, j, monkeypatch):
    monkeypatch.setenv("TNH_HEFF_STRATEGY", "1")
    test_heff_distinct_mpo_tensors(ctx, model, j, "bf16x6")
    test_heff_distinct_mpo_tensors(ctx, model, j, "fp64")


def test_heff_strategy_timed_once_per_shape(ctx, monkeypatch):
    # without TNH_HEFF_STRATEGY both strategies are timed for a new shape and
    # the choice is reused for the next plan of that shape
    from paper_2007_14822_gb300 import tnh
    monkeypatch.delenv("TNH_HEFF_STRATEGY", raising=False)
    c = tnh.Context(0)
    d = H.heff_inputs(80, None, 4, nsect=9, maxd=20)
    p1 = c.heff_plan(d["L"], d["W"], d["W"], d["R"], d["psi"], prec("bf16x6"))
    p2 = c.heff_plan(d["L"], d["W"], d["W"], d["R"], d["psi"], prec("bf16x6"))
    t1, t2 = p1.tuning, p2.tuning
    assert t1["strategy_measured"] and not t2["strategy_measured"] and t1["strategy"] == t2["strategy"]
    c.close()


# ------------------------------------------------- tridiagonal eigensolve
def _tridiag_cases():
    rng = np.random.default_rng(8)
    cases = []
    for k in (1, 2, 3, 17, 64, 255):
        cases.append(("random", rng.standard_normal(k) * 10, rng.standard_normal(k - 1) * 3))
    # Wilkinson W+ (pairs of eigenvalues close to rounding at the top; the
    # bottom is simple), and its negative (close pairs at the bottom)
    for m in (10, 30):
        a = np.abs(np.arange(-m, m + 1, dtype=float))
        cases.append(("wilkinson", a, np.ones(2 * m)))
        cases.append(("-wilkinson", -a, np.ones(2 * m)))
    # an exactly degenerate lowest pair: two copies of a block, split by b = 0
    a1, b1 = rng.standard_normal(12), rng.standard_normal(11)
    cases.append(("degenerate", np.concatenate([a1, a1]), np.concatenate([b1, [0.0], b1])))
    # graded entries over sixteen decades and a Lanczos-like matrix of a
    # converged run (tiny trailing beta)
    g = 10.0 ** np.linspace(-8, 8, 40)
    cases.append(("graded", g, np.sqrt(g[:-1] * g[1:]) * 0.3))
    a = -40 + rng.standard_normal(48)
    b = np.abs(rng.standard_normal(47)) * 5
    b[-8:] = 1e-9
    cases.append(("converged", a, b))
    return cases


@pytest.mark.parametrize("name,alpha,beta", _tridiag_cases(), ids=[c[0] + str(len(c[1])) for c in _tridiag_cases()])
def test_tridiag_lowest_matches_lapack(ctx, name, alpha, beta):
    # the Lanczos inner step on its own, against LAPACK's tridiagonal solver
    from scipy.linalg import eigh_tridiagonal
    th, v = ctx.tridiag_lowest(alpha, beta)
    w, V = eigh_tridiagonal(alpha, beta) if len(alpha) > 1 else (alpha.copy(), np.ones((1, 1)))
    scale = max(1.0, float(np.max(np.abs(alpha))) + (2 * float(np.max(np.abs(beta))) if len(beta) else 0.0))
    assert abs(th - w[0]) < 1e-13 * scale, (th, w[0])
    T = np.diag(alpha) + np.diag(beta, 1) + np.diag(beta, -1)
    assert abs(np.linalg.norm(v) - 1.0) < 1e-12
    assert np.linalg.norm(T @ v - th * v) < 1e-10 * scale
