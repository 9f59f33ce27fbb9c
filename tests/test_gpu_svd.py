"""GPU truncated SVD (batched one-sided Jacobi, FP64) against the oracle's
LAPACK SVD and the Eckart-Young identity."""
import numpy as np
import pytest

import helpers as H
from oracle import dmrg as D

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2007_14822_gb300 import build, tnh
    build.build()
    c = tnh.Context(0)
    yield c
    c.close()


def theta_inputs(m, nsect, maxd, seed):
    from paper_2007_14822_gb300 import models as pm
    a = H.link_index(m, nsect, maxd, +1)
    s = pm.site_index(pm.SPIN_QN, qn=nsect > 1)
    return H.random_pair([a, s, s, a.dag()], None, seed, "theta")


def factor(ctx, T, cutoff, maxdim, mindim=1, side=0, absorb=0):
    svd = ctx.svd_trunc(T, 2, cutoff, maxdim, mindim, exact_side=side)
    U, S, V = svd.factors(absorb=absorb)
    Uo, Vo = H.to_oracle(U), H.to_oracle(V)
    s = S.cpu().numpy()
    Sd, pos = {}, 0
    for q, dim in svd.sectors:
        Sd[q] = s[pos:pos + dim]
        pos += dim
    return svd, Uo, Sd, Vo, s


@pytest.mark.parametrize("m,nsect,maxd", [(1, 1, 1), (5, 1, 5), (24, 7, 6), (40, 1, 40), (96, 11, 20)])
def test_svd_full_rank_matches_oracle(ctx, m, nsect, maxd):
    T, To = theta_inputs(m, nsect, maxd, 3)
    svd, Uo, Sd, Vo, s = factor(ctx, T, 0.0, 10 ** 6)
    _, So, _, _ = D.svd_trunc(To, 2, 0.0, 10 ** 6)
    want = np.sort(np.concatenate(list(So.values())))[::-1]
    got = np.sort(s)[::-1]
    assert got.shape == want.shape
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-13 * want[0])
    # every sector is descending and the factors reproduce theta
    for v in Sd.values():
        assert np.all(np.diff(v) <= 0)
    rec = D.theta(D.scale_link(Uo, Sd, 2), Vo)
    assert H.rel_err(rec, To) < 1e-12
    Ud = Uo.to_dense().reshape(-1, Uo.inds[2].dim)
    np.testing.assert_allclose(Ud.T @ Ud, np.eye(Ud.shape[1]), atol=1e-12)
    Vd = Vo.to_dense().reshape(Vo.inds[0].dim, -1)
    np.testing.assert_allclose(Vd @ Vd.T, np.eye(Vd.shape[0]), atol=1e-12)


@pytest.mark.parametrize("keep", [1, 7, 30])
def test_svd_truncation_matches_oracle(ctx, keep):
    T, To = theta_inputs(48, 9, 10, 4)
    svd, Uo, Sd, Vo, s = factor(ctx, T, 0.0, keep)
    Uw, Sw, Vw, errw = D.svd_trunc(To, 2, 0.0, keep)
    assert svd.kept == keep
    assert [d for _, d in svd.sectors] == [len(v) for _, v in sorted(Sw.items())]
    assert abs(svd.truncerr - errw) < 1e-12
    rec = D.theta(D.scale_link(Uo, Sd, 2), Vo)
    disc = float(np.sum((rec.to_dense() - To.to_dense()) ** 2)) / To.norm() ** 2
    assert abs(disc - errw) < 1e-11


def test_svd_cutoff_rule(ctx):
    T, To = theta_inputs(48, 9, 10, 5)
    _, So, _, _ = D.svd_trunc(To, 2, 0.0, 10 ** 6)
    sv = np.sort(np.concatenate(list(So.values())))[::-1]
    tot = float(np.sum(sv ** 2))
    tail = np.cumsum((sv ** 2)[::-1])[::-1] / tot
    for k in (5, 20, 40):
        cutoff = 0.5 * (tail[k] + tail[k - 1])      # strictly between two tails
        svd = ctx.svd_trunc(T, 2, cutoff, 10 ** 6)
        assert svd.kept == k
        svd = ctx.svd_trunc(T, 2, cutoff, k - 2)    # maxdim binds
        assert svd.kept == k - 2


def test_svd_config2_size(ctx):
    # theta of the dense m=256, d=2 workload: a 512 x 512 matrix
    T, To = theta_inputs(256, 1, 256, 6)
    svd, Uo, Sd, Vo, s = factor(ctx, T, 1e-10, 256)
    Uw, Sw, Vw, errw = D.svd_trunc(To, 2, 1e-10, 256)
    want = np.concatenate(list(Sw.values()))
    np.testing.assert_allclose(np.sort(s)[::-1], np.sort(want)[::-1], rtol=1e-11, atol=1e-12 * want.max())
    assert abs(svd.truncerr - errw) < 1e-12


@pytest.mark.parametrize("side", [0, 1])
@pytest.mark.parametrize("absorb", [0, 1, 2])
def test_svd_exact_side_and_absorb(ctx, side, absorb):
    T, To = theta_inputs(40, 7, 12, 8)
    svd, Uo, Sd, Vo, s = factor(ctx, T, 0.0, 30, side=side, absorb=absorb)
    Sn = {q: np.ones_like(v) for q, v in Sd.items()}
    Su = Sd if absorb == 0 else Sn
    rec = D.theta(D.scale_link(Uo, Su, 2), Vo)
    _, _, _, err = D.svd_trunc(To, 2, 0.0, 30)
    disc = float(np.sum((rec.to_dense() - To.to_dense()) ** 2)) / To.norm() ** 2
    assert abs(disc - err) < 1e-11
    # the exact side is orthonormal to float64 accuracy
    if side == 0 and absorb != 1:
        Ud = Uo.to_dense().reshape(-1, Uo.inds[2].dim)
        np.testing.assert_allclose(Ud.T @ Ud, np.eye(Ud.shape[1]), atol=1e-13)
    if side == 1 and absorb != 2:
        Vd = Vo.to_dense().reshape(Vo.inds[0].dim, -1)
        np.testing.assert_allclose(Vd @ Vd.T, np.eye(Vd.shape[0]), atol=1e-13)


@pytest.mark.parametrize("side", [0, 1])
def test_svd_rank_deficient(ctx, side):
    # theta = A B with a rank smaller than the matrix: exact zero singular values
    from paper_2007_14822_gb300.tnh import Index, Tensor, FP64
    from paper_2007_14822_gb300 import models as pm
    a = H.link_index(24, 5, 8, +1)
    c = H.link_index(6, 3, 2, +1)
    s1, s2 = pm.site_index(pm.SPIN_QN, qn=True), pm.site_index(pm.SPIN_QN, qn=True)
    A, Ao = H.random_pair([a, s1, c.dag()], None, 3, "A")
    B, Bo = H.random_pair([c, s2, a.dag()], None, 4, "B")
    for t, lab in ((A, (1, 2, 3)), (B, (3, 4, 5))):
        for ix, l in zip(t.inds, lab):
            ix.label = l
    th = Tensor([A.inds[0], A.inds[1], B.inds[1], B.inds[2]])
    ctx.contract(A, B, th, FP64)
    tho = H.to_oracle(th)
    svd, Uo, Sd, Vo, s = factor(ctx, th, 1e-14, 64, side=side, absorb=2 - side)
    _, So, _, err = D.svd_trunc(tho, 2, 1e-14, 64)
    assert svd.kept == sum(len(v) for v in So.values())
    rec = D.theta(Uo, Vo)
    assert H.rel_err(rec, tho) < 1e-12


def test_svd_float64_zeros_dropped_only_below_cutoff_resolution(ctx):
    # The library drops singular values with s^2 < 1e-16 of the total even at
    # cutoff 0 (float64 cannot resolve their vectors); Sec. 5's rule, which
    # the oracle follows, keeps them. The two agree for every cutoff of at
    # least n * 1e-16 (n values): the values the library drops weigh less
    # than that together, so the cutoff drops them too. theta is a dense
    # 16 x 16 matrix U diag(s) V^T with four values below 1e-8 of the norm.
    from paper_2007_14822_gb300.tnh import Index, Tensor
    from oracle.blocksparse import BlockTensor
    rng = np.random.default_rng(3)
    s = np.array([10.0 ** (-k / 2) for k in range(12)] + [1e-9, 3e-10, 1e-11, 2e-12])
    U, _ = np.linalg.qr(rng.standard_normal((16, 16)))
    V, _ = np.linalg.qr(rng.standard_normal((16, 16)))
    M = (U * s) @ V.T
    a, sd = Index.dense(8, +1), Index.dense(2, +1)
    T = Tensor([a, sd, sd, a.dag()])
    T.fill(lambda key, shp: M.reshape(shp))
    To = H.to_oracle(T)
    n = 16
    resolved = int(np.sum(s ** 2 >= 1e-16 * np.sum(s ** 2)))
    assert resolved == 12
    # cutoff 0: the oracle keeps all 16, the library the 12 resolved ones
    _, So, _, _ = D.svd_trunc(To, 2, 0.0, 10 ** 6)
    assert sum(len(v) for v in So.values()) == n
    svd = ctx.svd_trunc(T, 2, 0.0, 10 ** 6)
    assert svd.kept == resolved
    # cutoff >= n * 1e-16: both keep the same values with the same error
    for cutoff in (n * 1e-16, 1e-14, 1e-12, 1e-10):
        _, So, _, erro = D.svd_trunc(To, 2, cutoff, 10 ** 6)
        svd = ctx.svd_trunc(T, 2, cutoff, 10 ** 6)
        assert svd.kept == sum(len(v) for v in So.values()), cutoff
        assert abs(svd.truncerr - erro) < 1e-15, cutoff
