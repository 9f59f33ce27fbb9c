"""Pins of the oracle's H_eff, environments, Lanczos, truncated SVD and DMRG."""
import math

import numpy as np
import pytest

from oracle import dmrg as D
from oracle import ed, models
from oracle.blocksparse import OUT, BlockTensor, QNIndex, trivial_index
from paper_2007_14822_gb300 import synth

from test_oracle_models import mpo_full


def random_mps(mpo, dims, seed, nsect=None, qn_link_fn=None):
    """Random real MPS with given link dims (dense: one trivial sector)."""
    site = mpo.site_index
    N = mpo.N
    A = []
    left = QNIndex([((0,) * site.nq, 1)], OUT)
    for j in range(N):
        if j == N - 1:
            right = QNIndex([(left.qn(0) if left.nsect == 1 else (0,) * site.nq, 1)], OUT)
        else:
            right = QNIndex([((0,) * site.nq, dims[j])], OUT)
        inds = [left, site, right.dag()]
        A.append(BlockTensor.from_blocks_fn(inds, None,
                 lambda key, shp, j=j: synth.block_gaussian(seed, f"A{j}", key, shp)))
        left = right
    return A


def dense_site_mpo(mpo):
    """The same MPO with every index flattened to one trivial sector."""
    W = []
    for w in mpo.W:
        inds = [trivial_index(i.dim, i.arrow, nq=w.inds[0].nq) for i in w.inds]
        W.append(BlockTensor.from_dense(w.to_dense(), inds))
    site = trivial_index(mpo.site_index.dim, OUT, nq=mpo.site_index.nq)
    return models.MPO(W, site, mpo.start, mpo.done)


def projector(A, j):
    """P maps theta[a_j, s_j, s_j+1, b] to the full state (site 0 slowest)."""
    N = len(A)
    left = np.ones((1, 1))                       # [full_left, a]
    for i in range(j):
        t = np.einsum("pa,asb->psb", left, A[i].to_dense())
        left = t.reshape(-1, t.shape[2])
    right = np.ones((1, 1))                      # [b, full_right]
    for i in range(N - 1, j + 1, -1):
        t = np.einsum("asb,bq->asq", A[i].to_dense(), right)
        right = t.reshape(t.shape[0], -1)
    # P[(l, s1, s2, r), (a, s1, s2, b)] = left[l,a] right[b,r]
    da, db = left.shape[1], right.shape[0]
    d = A[0].inds[1].dim
    P = np.einsum("la,sx,uy,br->lsuraxyb", left, np.eye(d), np.eye(d), right)
    return P.reshape(left.shape[0] * d * d * right.shape[1], da * d * d * db)


def envs_at(mpo, A, j):
    W = mpo.W
    N = mpo.N
    L = D.left_boundary(A[0], W[0], mpo.start)
    for i in range(j):
        L = D.env_left(L, A[i], W[i])
    R = D.right_boundary(A[N - 1], W[N - 1], mpo.done)
    for i in range(N - 1, j + 1, -1):
        R = D.env_right(R, A[i], W[i])
    return L, R


@pytest.mark.parametrize("model", ["heis", "hub"])
def test_heff_equals_projected_hamiltonian(model):
    if model == "heis":
        N, d = 6, 2
        mpo = dense_site_mpo(models.heisenberg_mpo(N))
        terms = models.spin_pair_terms(models.heisenberg_pairs(N))
        dims = [2, 3, 4, 3, 2]
    else:
        N, d = 4, 4
        mpo = dense_site_mpo(models.hubbard_mpo(N, 1.0, 4.0))
        terms = models.hubbard_terms(N, 1.0, 4.0)
        dims = [3, 4, 2]
    A = random_mps(mpo, dims, seed=21)
    H = ed.hamiltonian_dense(N, d, terms)
    for j in range(N - 1):
        P = projector(A, j)
        L, R = envs_at(mpo, A, j)
        th = D.theta(A[j], A[j + 1])
        Hm = D.heff_dense_matrix(L, mpo.W[j], mpo.W[j + 1], R, th)
        np.testing.assert_allclose(Hm, P.T @ H @ P, atol=1e-12 * max(1, np.abs(Hm).max()))


def qn_random_mps(mpo, maxd, seed, states):
    """Random QN MPS: start from a product state's link charges, widen links."""
    site = mpo.site_index
    N = mpo.N
    nq = site.nq
    # link sectors: every charge reachable from the left and completable to
    # the right target, dims capped by maxd
    qs = [site.qn(s) for s in range(site.nsect)]
    total = tuple(sum(site.qn(site.sector_of(st)[0])[k] for st in states) for k in range(nq))
    reach = [{(0,) * nq}]
    for j in range(N):
        reach.append({tuple(a + b for a, b in zip(q, s)) for q in reach[-1] for s in qs})
    back = [None] * (N + 1)
    back[N] = {total}
    for j in range(N - 1, -1, -1):
        back[j] = {tuple(a - b for a, b in zip(q, s)) for q in back[j + 1] for s in qs}
    links = []
    rng = np.random.default_rng(seed)
    for j in range(N + 1):
        ok = sorted(reach[j] & back[j])
        links.append(QNIndex([(q, 1 if j in (0, N) else int(rng.integers(1, maxd + 1)))
                              for q in ok], OUT))
    A = []
    for j in range(N):
        inds = [links[j], site, links[j + 1].dag()]
        A.append(BlockTensor.from_blocks_fn(inds, None,
                 lambda key, shp, j=j: synth.block_gaussian(seed, f"Q{j}", key, shp)))
    return A


def dense_tensor(T):
    inds = [trivial_index(i.dim, i.arrow, nq=i.nq) for i in T.inds]
    return BlockTensor.from_dense(T.to_dense(), inds, tuple(0 for _ in T.flux))


def test_qn_heff_embeds_dense_heff():
    N = 6
    mpo = models.heisenberg_mpo(N)
    A = qn_random_mps(mpo, 3, seed=22, states=[0, 1] * 3)
    dmpo = dense_site_mpo(mpo)
    for j in range(N - 1):
        L, R = envs_at(mpo, A, j)
        th = D.theta(A[j], A[j + 1])
        x = BlockTensor.from_blocks_fn(th.inds, th.flux,
                                       lambda k, s: synth.block_gaussian(5, "x", k, s))
        y = D.heff_apply(L, mpo.W[j], mpo.W[j + 1], R, x)
        # flux preserved: y has only allowed blocks
        BlockTensor.from_dense(y.to_dense(), y.inds, y.flux, atol=0.0)
        yd = D.heff_apply(dense_tensor(L), dmpo.W[j], dmpo.W[j + 1], dense_tensor(R),
                          dense_tensor(x))
        np.testing.assert_allclose(y.to_dense(), yd.to_dense(), atol=1e-12)


def test_heff_hermitian_and_matches_chain_energy():
    N = 8
    mpo = models.heisenberg_mpo(N)
    A = qn_random_mps(mpo, 4, seed=23, states=[0, 1] * 4)
    j = 3
    L, R = envs_at(mpo, A, j)
    th = D.theta(A[j], A[j + 1])
    x = BlockTensor.from_blocks_fn(th.inds, th.flux, lambda k, s: synth.block_gaussian(6, "x", k, s))
    z = BlockTensor.from_blocks_fn(th.inds, th.flux, lambda k, s: synth.block_gaussian(7, "z", k, s))
    Hx = D.heff_apply(L, mpo.W[j], mpo.W[j + 1], R, x)
    Hz = D.heff_apply(L, mpo.W[j], mpo.W[j + 1], R, z)
    assert abs(z.vdot(Hx) - Hz.vdot(x)) < 1e-12 * abs(z.vdot(Hx))
    # <theta|H_eff|theta> / <P theta|P theta> equals the full-chain expectation
    Hth = D.heff_apply(L, mpo.W[j], mpo.W[j + 1], R, th)
    num = th.vdot(Hth)
    want_num = D.mps_expectation(mpo, A)
    # normalisation through the same projector
    P = projector([dense_tensor(a) for a in A], j)
    nrm = float(np.sum((P @ th.to_dense().ravel()) ** 2))
    assert abs(num / nrm - want_num) < 1e-11 * abs(want_num)


def test_lanczos_matches_eigh():
    rng = np.random.default_rng(31)
    n = 60
    M = rng.standard_normal((n, n))
    M = M + M.T
    w = np.linalg.eigvalsh(M)
    ops = dict(vdot=lambda u, v: float(u @ v), norm=lambda u: float(np.linalg.norm(u)),
               scale=lambda u, a: u * a, axpy=lambda u, a, v: u + a * v)
    E, x, res, k = D.lanczos(lambda v: M @ v, rng.standard_normal(n), 60, 1e-12, **ops)
    assert abs(E - w[0]) < 1e-10
    assert np.linalg.norm(M @ x - E * x) < 1e-8


def test_energy_residual_rayleigh_quotient():
    # E = <x|Hx>/<x|x> and r = |Hx - Ex|: zero residual on an eigenvector,
    # and r^2 = |Hx|^2/|x|^2 - E^2 for a unit vector (Pythagoras, Hx - Ex is
    # orthogonal to x); vectors are plain numpy arrays with the BlockTensor
    # operations the function uses
    class V:
        def __init__(self, a):
            self.a = np.asarray(a, dtype=np.float64)

        def vdot(self, o):
            return float(self.a @ o.a)

        def axpy(self, c, o):
            return V(self.a + c * o.a)

        def norm(self):
            return float(np.linalg.norm(self.a))
    rng = np.random.default_rng(41)
    M = rng.standard_normal((30, 30))
    M = M + M.T
    w, U = np.linalg.eigh(M)
    apply = lambda v: V(M @ v.a)
    E, r = D.energy_residual(apply, V(3.0 * U[:, 4]))
    assert abs(E - w[4]) < 1e-12 * np.abs(w).max() and r < 1e-11 * np.abs(w).max() * 3.0
    x = rng.standard_normal(30)
    E, r = D.energy_residual(apply, V(x))
    u = x / np.linalg.norm(x)
    assert abs(E - u @ M @ u) < 1e-12 * np.abs(w).max()
    assert abs(r / np.linalg.norm(x) - np.sqrt(np.sum((M @ u) ** 2) - E ** 2)) < 1e-10 * np.abs(w).max()


def test_truncation_count_rule():
    s = np.array([1.0, 0.5, 0.1, 0.01])
    tot = float(np.sum(s ** 2))
    # cutoff just above the smallest weight -> drop one
    k, err = D.truncation_count(s, 1.0001e-4 / tot, 10)
    assert k == 3 and abs(err - 1e-4 / tot) < 1e-15
    # cutoff just below -> keep all
    k, err = D.truncation_count(s, 0.9999e-4 / tot, 10)
    assert k == 4 and err == 0.0
    # cutoff covering the two smallest
    k, _ = D.truncation_count(s, (0.01 ** 2 + 0.1 ** 2) / tot, 10)
    assert k == 2
    # maxdim binds
    k, err = D.truncation_count(s, 0.0, 2)
    assert k == 2 and abs(err - (0.01 ** 2 + 0.1 ** 2) / tot) < 1e-15
    # mindim binds
    k, _ = D.truncation_count(s, 1.0, 10, mindim=2)
    assert k == 2
    # at least one is kept
    k, _ = D.truncation_count(s, 1.0, 10)
    assert k == 1
    # Sec. 5 discards only what the cutoff covers: at cutoff 0 even values far
    # below float64 resolution of the norm are kept; an exact zero is
    # discarded (its weight 0 is within the cutoff); a cutoff just above the
    # tail of the two tiny values drops them
    s2 = np.array([1.0, 1e-3, 2e-9, 1e-12])
    k, err = D.truncation_count(s2, 0.0, 10)
    assert k == 4 and err == 0.0
    k, err = D.truncation_count(np.array([1.0, 1e-3, 0.0]), 0.0, 10)
    assert k == 2 and err == 0.0
    tot2 = float(np.sum(s2 ** 2))
    k, err = D.truncation_count(s2, 1.01 * (4e-18 + 1e-24) / tot2, 10)
    assert k == 2 and abs(err - (4e-18 + 1e-24) / tot2) < 1e-30


def test_svd_trunc_eckart_young_and_predicted_count():
    # theta built as U diag(sigma) V^T per charge sector with chosen sigma
    site = QNIndex([((1,), 1), ((-1,), 1)], OUT)
    a = QNIndex([((0,), 3), ((2,), 2), ((-2,), 2)], OUT)
    b = QNIndex([((0,), 3), ((2,), 2), ((-2,), 2)], OUT)
    inds = [a, site, site, b.dag()]
    rng = np.random.default_rng(41)
    th = BlockTensor.from_blocks_fn(inds, None, lambda k, s: rng.standard_normal(s))
    U, S, V, err0 = D.svd_trunc(th, 2, 0.0, 10 ** 6)
    rec = D.theta(D.scale_link(U, S, 2), V)
    np.testing.assert_allclose(rec.to_dense(), th.to_dense(), atol=1e-12)
    allsv = np.sort(np.concatenate(list(S.values())))[::-1]
    n = len(allsv)
    for keep in [1, 3, n // 2, n - 1]:
        U, S, V, err = D.svd_trunc(th, 2, 0.0, keep)
        assert sum(len(v) for v in S.values()) == keep
        rec = D.theta(D.scale_link(U, S, 2), V)
        disc = float(np.sum(allsv[keep:] ** 2))
        diff = th.to_dense() - rec.to_dense()
        assert abs(float(np.sum(diff ** 2)) - disc) < 1e-10 * float(np.sum(allsv ** 2))
        assert abs(err - disc / float(np.sum(allsv ** 2))) < 1e-12
    # U is an isometry
    Ud = U.to_dense().reshape(-1, U.inds[2].dim)
    np.testing.assert_allclose(Ud.T @ Ud, np.eye(Ud.shape[1]), atol=1e-12)


def _dmrg(mpo, mps, sweeps, **kw):
    return D.dmrg(mpo, mps, sweeps, **kw)


def test_dmrg_heisenberg_dense_vs_ed():
    N = 10
    mpo = dense_site_mpo(models.heisenberg_mpo(N))
    vecs = synth.product_spinors(1, N, 2)
    A = D.product_mps_vectors(mpo.site_index, vecs)
    E, A, st = _dmrg(mpo, A, [(8, 1e-12), (16, 1e-12), (32, 1e-13), (32, 1e-13)])
    e_ed = ed.ground_energy(N, 2, models.spin_pair_terms(models.heisenberg_pairs(N)))
    assert abs(E - e_ed) < 1e-10 * abs(e_ed)
    assert abs(D.mps_expectation(mpo, A) - E) < 1e-9


def test_dmrg_heisenberg_qn_vs_ed():
    N = 12
    mpo = models.heisenberg_mpo(N)
    A = D.product_mps_basis(mpo.site_index, [0, 1] * (N // 2), 1)
    E, A, st = _dmrg(mpo, A, [(8, 1e-12), (32, 1e-12), (64, 1e-13), (64, 1e-13)])
    e_ed = ed.ground_energy(N, 2, models.spin_pair_terms(models.heisenberg_pairs(N)),
                            models.SPIN_QN, (0,))
    assert abs(E - e_ed) < 1e-10 * abs(e_ed)


def test_dmrg_tfim_free_fermion():
    from test_oracle_models import tfim_closed_form
    N = 12
    mpo = models.tfim_mpo(N, 1.0, 1.3)
    A = D.product_mps_vectors(mpo.site_index, synth.product_spinors(2, N, 2))
    E, A, st = _dmrg(mpo, A, [(8, 1e-12), (24, 1e-13), (32, 1e-13)])
    assert abs(E - tfim_closed_form(N, 1.0, 1.3)) < 1e-10 * abs(E)


def test_dmrg_majumdar_ghosh():
    N = 12
    mpo = models.heisenberg_like_mpo(N, models.j1j2_chain_pairs(N, 1.0, 0.5))
    A = D.product_mps_basis(mpo.site_index, [0, 1] * (N // 2), 1)
    E, A, st = _dmrg(mpo, A, [(8, 1e-12), (32, 1e-12), (64, 1e-13), (64, 1e-13)])
    assert abs(E + 3 * N / 8) < 1e-10 * 3 * N / 8


def test_dmrg_hubbard_vs_ed():
    N = 4
    mpo = models.hubbard_mpo(N, 1.0, 4.0)
    A = D.product_mps_basis(mpo.site_index, [1, 2] * (N // 2), 2)
    E, A, st = _dmrg(mpo, A, [(16, 1e-12), (64, 1e-13), (64, 1e-13)])
    e_ed = ed.ground_energy(N, 4, models.hubbard_terms(N, 1.0, 4.0), models.HUB_QN, (N, 0))
    assert abs(E - e_ed) < 1e-10 * abs(e_ed)


def test_dmrg_is_variational_and_truncation_bounded():
    # N=20 Heisenberg, m=32, cutoff 1e-10, 5 sweeps, random product state
    N = 20
    mpo = dense_site_mpo(models.heisenberg_mpo(N))
    A = D.product_mps_vectors(mpo.site_index, synth.product_spinors(1, N, 2))
    E, A, st = _dmrg(mpo, A, [(32, 1e-10)] * 5, krylov_dim=64, tol=1e-10)
    e_ed = ed.ground_energy(N, 2, models.spin_pair_terms(models.heisenberg_pairs(N)),
                            models.SPIN_QN, (0,))
    # variational, and the energy error is set by the weight the last sweep
    # discarded: 0 <= E - E_ED <= 10 * sum(truncerr) * |E| (the error of a
    # truncated two-site step is first order in its discarded weight)
    assert E >= e_ed - 1e-12 * abs(e_ed)
    assert st[-1]["truncerr_sum"] > 0.0
    assert E - e_ed <= 10.0 * st[-1]["truncerr_sum"] * abs(E)


def test_dmrg_heisenberg_n20_converged_vs_ed():
    # the same chain at maxdim 256 and cutoff 1e-12 (U(1) storage, Neel
    # start) reaches the exact ground energy of the Sz=0 sector (sparse
    # Lanczos over its 184 756 states) to 1e-9 relative
    N = 20
    mpo = models.heisenberg_mpo(N)
    A = D.product_mps_basis(mpo.site_index, [0, 1] * (N // 2), 1)
    E, A, st = _dmrg(mpo, A, [(16, 1e-12), (64, 1e-12), (256, 1e-12)])
    e_ed = ed.ground_energy(N, 2, models.spin_pair_terms(models.heisenberg_pairs(N)),
                            models.SPIN_QN, (0,))
    assert E >= e_ed - 1e-12 * abs(e_ed)
    assert abs(E - e_ed) < 1e-9 * abs(e_ed)
    assert st[-1]["truncerr"] <= 1e-12


# ------------------------------------------- sums of MPOs, excited states
def full_state(A, j=None, th=None):
    """The d^N vector of an MPS by dense contraction; with ``j`` and ``th``
    the pair (A[j], A[j+1]) is replaced by the two-site tensor th."""
    mats = [T.to_dense() for T in A]
    if j is not None:
        t = th.to_dense()
        mats = mats[:j] + [t.reshape(t.shape[0], -1, t.shape[3])] + mats[j + 2:]
    v = mats[0][0]                              # (s, b)
    for t in mats[1:]:
        v = np.einsum("xa,asb->xsb", v, t).reshape(-1, t.shape[2])
    return v[:, 0]


def test_mps_overlap_and_projected_state_match_full_vectors():
    # random dense MPS P and A; bond (2, 3) of A holds a random theta
    N, j = 6, 2
    mpo = dense_site_mpo(models.heisenberg_mpo(N))
    P = random_mps(mpo, [2, 4, 5, 4, 2], 21)
    A = random_mps(mpo, [2, 3, 4, 3, 2], 22)
    ref = float(full_state(P) @ full_state(A))
    assert abs(D.mps_overlap(P, A) - ref) < 1e-12 * max(1.0, abs(ref))
    LO, RO = D.overlap_boundaries(P, A)
    for k in range(j):
        LO = D.overlap_left(LO, P[k], A[k])
    for k in range(N - 1, j + 1, -1):
        RO = D.overlap_right(RO, P[k], A[k])
    phi = D.projected_state(LO, P[j], P[j + 1], RO)
    th = D.theta(A[j], A[j + 1])
    assert abs(phi.vdot(th) - ref) < 1e-12 * max(1.0, abs(ref))
    # <phi, theta2> = <P|psi(theta2)> for any theta2 in the same space
    th2 = D.from_vector(synth.gaussian(23, (D.to_vector(th).size,)), th)
    ref2 = float(full_state(P) @ full_state(A, j, th2))
    assert abs(phi.vdot(th2) - ref2) < 1e-12 * max(1.0, abs(ref2))


def test_dmrg_sum_of_mpos_majumdar_ghosh():
    # H = H_J1 + H_J2 as two MPOs; J2/J1 = 1/2 has E0 = -3N/8 exactly
    N = 10
    h1 = models.heisenberg_like_mpo(N, [(i, i + 1, 1.0) for i in range(N - 1)])
    h2 = models.heisenberg_like_mpo(N, [(i, i + 2, 0.5) for i in range(N - 2)])
    A = D.product_mps_basis(h1.site_index, [0, 1] * (N // 2), 1)
    E, A, st = _dmrg([h1, h2], A, [(8, 1e-12), (32, 1e-12), (64, 1e-13), (64, 1e-13)])
    assert abs(E + 3 * N / 8) < 1e-10 * 3 * N / 8
    assert abs(D.mps_expectation([h1, h2], A) - E) < 1e-9
    # the ground state is the dimer product of singlets, on which every
    # next-nearest-neighbour S_i . S_(i+2) has zero expectation (the two
    # spins sit in different singlets)
    assert abs(D.mps_expectation(h2, A)) < 1e-9


def test_dmrg_sum_of_mpos_tfim_free_fermion():
    from test_oracle_models import tfim_closed_form
    N, J, h = 10, 1.0, 1.3
    terms = [models.tfim_mpo(N, J, 0.0), models.tfim_mpo(N, 0.0, h)]
    A = D.product_mps_vectors(terms[0].site_index, synth.product_spinors(3, N, 2))
    E, A, st = _dmrg(terms, A, [(8, 1e-12), (24, 1e-13), (32, 1e-13)])
    assert abs(E - tfim_closed_form(N, J, h)) < 1e-10 * abs(E)


def tfim_levels(N, J, h):
    """Lowest levels of the open TFIM: E0 = -sum eps_k, E0 + 2 eps_k for one
    excited Jordan-Wigner mode (eps_k = singular values of the bidiagonal)."""
    M = np.diag([h] * N) + np.diag([J] * (N - 1), 1)
    eps = np.sort(np.linalg.svd(M, compute_uv=False))
    E0 = -float(np.sum(eps))
    return E0, E0 + 2 * eps[0], E0 + 2 * eps[1]


def test_tfim_levels_match_ed():
    N, J, h = 6, 1.0, 1.5
    e = ed.ground_energy(N, 2, models.tfim_terms(N, J, h), k=3)
    np.testing.assert_allclose(e, tfim_levels(N, J, h), rtol=0, atol=1e-12)


def test_dmrg_excited_states_tfim():
    N, J, h = 8, 1.0, 1.5
    E0x, E1x, E2x = tfim_levels(N, J, h)
    mpo = models.tfim_mpo(N, J, h)
    sweeps = [(8, 1e-13), (32, 1e-14), (32, 1e-14), (32, 1e-14)]
    start = lambda seed: D.product_mps_vectors(mpo.site_index, synth.product_spinors(seed, N, 2))
    E0, A0, _ = _dmrg(mpo, start(4), sweeps)
    E1, A1, _ = _dmrg(mpo, start(5), sweeps + [(32, 1e-14)] * 2, ortho=[A0], weight=20.0)
    E2, A2, _ = _dmrg(mpo, start(6), sweeps + [(32, 1e-14)] * 2, ortho=[A0, A1], weight=20.0)
    assert abs(E0 - E0x) < 1e-10 * abs(E0x)
    assert abs(E1 - E1x) < 1e-9 * abs(E1x)
    assert abs(E2 - E2x) < 1e-9 * abs(E2x)
    assert abs(D.mps_overlap(A0, A1)) < 1e-6
    assert abs(D.mps_overlap(A0, A2)) < 1e-6 and abs(D.mps_overlap(A1, A2)) < 1e-6
    # without the projector the same start falls back to the ground state
    Eg, _, _ = _dmrg(mpo, start(5), sweeps)
    assert abs(Eg - E0x) < 1e-9 * abs(E0x)


def test_dmrg_excited_state_heisenberg_qn_vs_ed():
    N = 8
    mpo = models.heisenberg_mpo(N)
    e_ed = ed.ground_energy(N, 2, models.spin_pair_terms(models.heisenberg_pairs(N)),
                            models.SPIN_QN, (0,), k=2)
    sweeps = [(8, 1e-13), (16, 1e-14), (16, 1e-14), (16, 1e-14), (16, 1e-14), (16, 1e-14)]
    E0, A0, _ = _dmrg(mpo, D.product_mps_basis(mpo.site_index, [0, 1] * (N // 2), 1), sweeps)
    E1, A1, _ = _dmrg(mpo, D.product_mps_basis(mpo.site_index, [1, 0] * (N // 2), 1), sweeps,
                      ortho=[A0], weight=5.0)
    assert abs(E0 - e_ed[0]) < 1e-10 * abs(e_ed[0])
    assert abs(E1 - e_ed[1]) < 1e-9 * abs(e_ed[1])
    assert abs(D.mps_overlap(A0, A1)) < 1e-6


def test_heisenberg_bethe_ansatz_energy_density():
    # bulk energy per bond of the spin-1/2 Heisenberg chain: 1/4 - ln 2 (Bethe
    # ansatz). On open chains E0(N) = N e + surface + O(1/N), so the slope
    # between two lengths approaches e: exact diagonalisation at N = 14, 16 and
    # the oracle's DMRG at N = 24 (beyond exact diagonalisation here)
    e_bulk = 0.25 - math.log(2)
    e = {N: ed.ground_energy(N, 2, models.spin_pair_terms(models.heisenberg_pairs(N)), models.SPIN_QN, (0,))
         for N in (14, 16)}
    assert abs((e[16] - e[14]) / 2 - e_bulk) < 1e-3
    N = 24
    mpo = models.heisenberg_mpo(N)
    A = D.product_mps_basis(mpo.site_index, [0, 1] * (N // 2), 1)
    E24, _, _ = _dmrg(mpo, A, [(16, 1e-10), (64, 1e-10), (64, 1e-10)], krylov_dim=16, tol=1e-8)
    slope = (E24 - e[16]) / 8
    assert abs(slope - e_bulk) < 6e-4, slope
    # and a longer chain lies lower per site than a shorter one, toward e
    assert E24 / N < e[16] / 16
