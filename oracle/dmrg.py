"""Two-site DMRG hot path, stated plainly (oracle side).

Test infrastructure (see the package header). All arithmetic is numpy
float64 on ``BlockTensor`` objects; a dense tensor is the one-sector case.

Tensor conventions (arrows per Sec. 8.2; Out adds, In subtracts):

* MPS site tensor  ``A[a, s, b]``           a Out, s Out, b In, flux 0 --
  the link QN is the total charge of the sites to its left (the paper's MPS
  of Sec. 7.3 with real entries).
* MPO site tensor  ``W[wl, wr, s, s']``      wl In, wr Out, s In, s' Out.
* left environment ``L[a, w, a']``           a In, w Out, a' Out.
* right environment``R[b, w, b']``           b Out, w In, b' In.
* two-site state   ``psi[a, s1, s2, b]``     as the product of two A's.

H_eff . psi is (Sec. 7.2: DMRG is the dominant eigenvector problem of the
MPO Hamiltonian; Sec. 9.4: contraction dominates)

    y[a', s1', s2', b'] = sum L[a,w,a'] W1[w,w1,s1,s1'] W2[w1,w2,s2,s2']
                              R[b,w2,b'] psi[a,s1,s2,b]

evaluated as four pairwise contractions S1..S4 in that order.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from .blocksparse import BlockTensor, IN, OUT, QNIndex, contract, qn_add


# ------------------------------------------------------------ primitives
def dag(T):
    """Reverse every arrow and negate the flux (real data is unchanged);
    the conjugate of Sec. 8.2 and Sec. 8.3 for real tensors."""
    return BlockTensor([i.dag() for i in T.inds], tuple(-x for x in T.flux),
                       T.blocks)


def heff_apply(L, W1, W2, R, psi):
    """H_eff . psi via S1 (sum a), S2 (sum w, s1), S3 (sum w1, s2), S4 (sum w2, b).

    The local effective Hamiltonian of two-site DMRG (Sec. 7.2), applied as
    four pairwise labelled contractions (Sec. 4, Sec. 9.4).
    """
    L = L.relabel(["a", "w", "ap"])
    W1 = W1.relabel(["w", "w1", "s1", "s1p"])
    W2 = W2.relabel(["w1", "w2", "s2", "s2p"])
    R = R.relabel(["b", "w2", "bp"])
    psi = psi.relabel(["a", "s1", "s2", "b"])
    T1 = contract(L, psi)                 # S1: [w, ap, s1, s2, b]
    T2 = contract(T1, W1)                 # S2: [ap, s2, b, w1, s1p]
    T3 = contract(T2, W2)                 # S3: [ap, b, s1p, w2, s2p]
    y = contract(T3, R, out_labels=["ap", "s1p", "s2p", "bp"])   # S4
    return y.relabel(["a", "s1", "s2", "b"])


def heff_dense_matrix(L, W1, W2, R, psi_like):
    """H_eff (Sec. 7.2) as an explicit matrix on the stored entries of ``psi_like``.

    Column j is H_eff applied to the j-th unit vector of the block-sparse
    vector space (blocks in sorted order, row-major inside a block).
    """
    keys = sorted(psi_like.blocks)
    sizes = [psi_like.blocks[k].size for k in keys]
    n = sum(sizes)
    Hm = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        Hm[:, j] = to_vector(heff_apply(L, W1, W2, R, from_vector(e, psi_like)))
    return Hm


def to_vector(T):
    return np.concatenate([T.blocks[k].ravel() for k in sorted(T.blocks)]) \
        if T.blocks else np.zeros(0)


def from_vector(v, like):
    out = BlockTensor(like.inds, like.flux)
    pos = 0
    for k in sorted(like.blocks):
        shp = like.blocks[k].shape
        n = int(np.prod(shp))
        out.blocks[k] = np.asarray(v[pos:pos + n], dtype=np.float64).reshape(shp)
        pos += n
    return out


def env_left(L, A, W):
    """L_new[b, w', b'] = sum L[a,w,a'] A[a,s,b] W[w,w',s,s'] A[a',s',b'].

    Forming the left environment tensor one site further (Sec. 7.2).

    Three pairwise contractions in the order: sum a; sum (w, s); sum (a', s').
    The bra tensor is ``dag(A)`` (real entries, reversed arrows).
    """
    L = L.relabel(["a", "w", "ap"])
    Ak = A.relabel(["a", "s", "b"])
    Wt = W.relabel(["w", "w1", "s", "sp"])
    Ab = dag(A).relabel(["ap", "sp", "bp"])
    X = contract(L, Ak)                   # [w, ap, s, b]
    Y = contract(X, Wt)                   # [ap, b, w1, sp]
    return contract(Y, Ab, out_labels=["b", "w1", "bp"])


def env_right(R, A, W):
    """R_new[a, w, a'] = sum A[a,s,b] W[w,w',s,s'] A[a',s',b'] R[b,w',b'].

    Forming the right environment tensor one site further (Sec. 7.2), in the
    same three pairwise contractions as ``env_left``.
    """
    R = R.relabel(["b", "w1", "bp"])
    Ak = A.relabel(["a", "s", "b"])
    Wt = W.relabel(["w", "w1", "s", "sp"])
    Ab = dag(A).relabel(["ap", "sp", "bp"])
    X = contract(Ak, R)                   # [a, s, w1, bp]
    Y = contract(X, Wt)                   # [a, bp, w, sp]
    return contract(Y, Ab, out_labels=["a", "w", "ap"])


def theta(A1, A2):
    """Two-site state theta[a,s1,s2,b] = sum_c A1[a,s1,c] A2[c,s2,b]: two MPS
    tensors (Sec. 7.3) contracted over their shared link (Sec. 4)."""
    A1 = A1.relabel(["a", "s1", "c"])
    A2 = A2.relabel(["c", "s2", "b"])
    return contract(A1, A2)


def left_boundary(A0, W0, start):
    """L_0[a, w, a'] = 1 at the MPO link state ``start`` (a, a' have dim 1):
    the left end of the environment recursion of Sec. 7.2."""
    a = A0.inds[0]
    inds = [a.dag(), W0.inds[0].dag(), a]
    T = BlockTensor.zeros(inds)
    sec, pos = inds[1].sector_of(start)
    for key in T.blocks:
        if key[1] == sec:
            T.blocks[key][0, pos, 0] = 1.0
    return T


def right_boundary(AN, WN, done):
    """R_N[b, w, b'] = 1 at the MPO link state ``done`` (b, b' have dim 1):
    the right end of the environment recursion of Sec. 7.2."""
    b = AN.inds[2]
    inds = [b.dag(), WN.inds[1].dag(), b]
    T = BlockTensor.zeros(inds)
    sec, pos = inds[1].sector_of(done)
    for key in T.blocks:
        if key[1] == sec:
            T.blocks[key][0, pos, 0] = 1.0
    return T


# -------------------------------------------------------------- Lanczos
def lanczos(apply, x0, krylov_dim=64, tol=1e-10, vdot=None, axpy=None,
            norm=None, scale=None):
    """Lowest eigenpair by Lanczos with full reorthogonalisation.

    The paper only says that a few Krylov (Lanczos) steps are taken per DMRG
    step (Sec. 12.2); the algorithm is the textbook one: q1 = x0/|x0|, k
    steps of w = H q_j - alpha_j q_j - beta_{j-1} q_{j-1}, then classical
    Gram-Schmidt against every previous q applied twice, beta_j = |w|. The
    tridiagonal eigenproblem is solved by LAPACK (scipy.linalg
    eigh_tridiagonal). Stops when the Ritz residual beta_j |s_j| <= tol
    (relative to |theta|) or on breakdown. Returns (energy, Ritz vector,
    residual estimate, number of matvecs).
    """
    vdot = vdot or (lambda u, v: u.vdot(v))
    norm = norm or (lambda u: u.norm())
    scale = scale or (lambda u, a: u.scaled(a))
    axpy = axpy or (lambda u, a, v: u.axpy(a, v))
    q = [scale(x0, 1.0 / norm(x0))]
    alpha, beta = [], []
    lam, s, res = None, None, np.inf
    for j in range(krylov_dim):
        w = apply(q[j])
        a = vdot(q[j], w)
        alpha.append(a)
        w = axpy(w, -a, q[j])
        if j > 0:
            w = axpy(w, -beta[j - 1], q[j - 1])
        for _ in range(2):
            h = [vdot(qi, w) for qi in q]
            for qi, hi in zip(q, h):
                w = axpy(w, -hi, qi)
        b = norm(w)
        if len(alpha) == 1:
            lam, s = alpha[0], np.array([1.0])
        else:
            ev, evec = sla.eigh_tridiagonal(np.array(alpha), np.array(beta),
                                            select="i", select_range=(0, 0))
            lam, s = float(ev[0]), evec[:, 0]
        res = b * abs(s[-1])
        if res <= tol * max(1.0, abs(lam)) or b <= 1e-14 * max(1.0, abs(lam)):
            break
        beta.append(b)
        q.append(scale(w, 1.0 / b))
    x = scale(q[0], s[0])
    for qi, si in zip(q[1:len(s)], s[1:]):
        x = axpy(x, si, qi)
    x = scale(x, 1.0 / norm(x))
    return float(lam), x, float(res), len(alpha)


def energy_residual(apply, x):
    """E = <x|H x>/<x|x> and r = |H x - E x| (all float64), for the local
    eigenproblem of Sec. 7.2."""
    y = apply(x)
    nx2 = x.vdot(x)
    E = y.vdot(x) / nx2
    r = y.axpy(-E, x).norm()
    return float(E), float(r)


# ------------------------------------------------------ truncated SVD
def truncation_count(svals_desc, cutoff, maxdim, mindim=1):
    """Number of singular values kept, and the truncation error.

    Sec. 5: squares of the singular values are summed from the smallest
    upward while the truncation error stays within ``cutoff``; at most
    ``maxdim`` values are kept. Reading used: the error is relative,
    sum(discarded s^2) / sum(all s^2); the boundary is non-strict; at least
    ``mindim`` (and at least one) values are kept. Nothing else is dropped:
    at cutoff 0 every value whose weight is above zero is kept.
    """
    s2 = np.asarray(svals_desc, dtype=np.float64) ** 2
    n = len(s2)
    total = float(s2.sum())
    if n == 0:
        return 0, 0.0
    if total == 0.0:
        keep = min(n, max(1, mindim))
        return keep, 0.0
    # discarded weight when keeping the first k values
    tail = np.concatenate([np.cumsum(s2[::-1])[::-1], [0.0]]) / total
    keep = n
    for k in range(n, 0, -1):
        if tail[k - 1] <= cutoff:
            keep = k - 1
        else:
            break
    keep = max(keep, 1, mindim)
    keep = min(keep, maxdim, n)
    keep = max(keep, min(mindim, n), 1)
    return keep, float(tail[keep])


def svd_trunc(T, nrow, cutoff, maxdim, mindim=1):
    """Truncated SVD of a block-sparse tensor (Sec. 5, Sec. 8.3).

    The first ``nrow`` indices are the row indices. Blocks are grouped by
    their row charge (combined index, as a combiner would group equal-QN
    sectors, Sec. 4); each group is one dense matrix factorised by
    ``numpy.linalg.svd``. Singular values of all groups are pooled, sorted
    descending (ties: group order, then position), and truncated with
    ``truncation_count``. Returns (U, S, V, truncerr) with U[rows..., c],
    V[c, cols...], S a dict charge -> kept values, and ``c`` a new link whose
    sectors are the kept charges in ascending order (U's c is In, V's c is
    Out).
    """
    rinds, cinds = T.inds[:nrow], T.inds[nrow:]
    nq = T.inds[0].nq

    def rcharge(key):
        q = (0,) * nq
        for ind, s in zip(rinds, key[:nrow]):
            q = qn_add(q, tuple(ind.arrow * x for x in ind.qn(s)))
        return q

    groups = {}
    for key in T.allowed():
        groups.setdefault(rcharge(key), []).append(key)
    mats = {}
    for Q, keys in sorted(groups.items()):
        rkeys = sorted({k[:nrow] for k in keys})
        ckeys = sorted({k[nrow:] for k in keys})
        roff, coff, r, c = {}, {}, 0, 0
        for rk in rkeys:
            roff[rk] = r
            r += int(np.prod([ind.sdim(s) for ind, s in zip(rinds, rk)]))
        for ck in ckeys:
            coff[ck] = c
            c += int(np.prod([ind.sdim(s) for ind, s in zip(cinds, ck)]))
        M = np.zeros((r, c))
        for k in keys:
            blk = T.blocks.get(k)
            if blk is None:
                continue
            rr = int(np.prod(blk.shape[:nrow]))
            cc = int(np.prod(blk.shape[nrow:]))
            M[roff[k[:nrow]]:roff[k[:nrow]] + rr,
              coff[k[nrow:]]:coff[k[nrow:]] + cc] = blk.reshape(rr, cc)
        U, s, Vt = np.linalg.svd(M, full_matrices=False)
        mats[Q] = (rkeys, ckeys, roff, coff, U, s, Vt)
    pool = []
    for gi, Q in enumerate(sorted(mats)):
        for p, v in enumerate(mats[Q][5]):
            pool.append((-v, gi, p, Q))
    pool.sort()
    svals = [-t[0] for t in pool]
    keep, err = truncation_count(svals, cutoff, maxdim, mindim)
    kept = {}
    for t in pool[:keep]:
        kept.setdefault(t[3], []).append(t[2])
    Qs = sorted(kept)
    link = QNIndex([(Q, len(kept[Q])) for Q in Qs], OUT)
    Uinds = list(rinds) + [link.dag()]
    Vinds = [link] + list(cinds)
    Ut = BlockTensor(Uinds, (0,) * nq)
    Vt_ = BlockTensor(Vinds, T.flux)
    S = {}
    for ci, Q in enumerate(Qs):
        rkeys, ckeys, roff, coff, U, s, Vt = mats[Q]
        idx = sorted(kept[Q])
        S[Q] = s[idx]
        for rk in rkeys:
            shp = tuple(ind.sdim(x) for ind, x in zip(rinds, rk))
            rr = int(np.prod(shp))
            Ut.blocks[rk + (ci,)] = U[roff[rk]:roff[rk] + rr, idx].reshape(shp + (len(idx),))
        for ck in ckeys:
            shp = tuple(ind.sdim(x) for ind, x in zip(cinds, ck))
            cc = int(np.prod(shp))
            Vt_.blocks[(ci,) + ck] = Vt[idx, coff[ck]:coff[ck] + cc].reshape((len(idx),) + shp)
    return Ut, S, Vt_, err


def scale_link(T, S, axis):
    """Multiply T by diag(S) along its link ``axis`` (sector order = sorted Q):
    the singular values of Sec. 5 moved into one factor."""
    out = T.copy()
    Qs = sorted(S)
    for key, v in out.blocks.items():
        sv = S[Qs[key[axis]]]
        shp = [1] * v.ndim
        shp[axis] = len(sv)
        out.blocks[key] = v * sv.reshape(shp)
    return out


# ----------------------------------------------------------------- MPS
def product_mps_basis(site_index, states, nq):
    """Product state with site j in basis state ``states[j]`` (QN MPS), the
    initial state of the DMRG example of Sec. 7.2."""
    N = len(states)
    A = []
    q = (0,) * nq
    left = QNIndex([(q, 1)], OUT)
    for j in range(N):
        sec = site_index.sector_of(states[j])
        qs = site_index.qn(sec[0])
        q = qn_add(q, qs)
        right = QNIndex([(q, 1)], OUT)
        inds = [left, site_index, right.dag()]
        T = BlockTensor.zeros(inds)
        key = (0, sec[0], 0)
        T.blocks[key][0, sec[1], 0] = 1.0
        A.append(T)
        left = right
    return A


def product_mps_vectors(site_index, vecs):
    """Dense product state with site j in the normalised vector ``vecs[j]``
    (an initial MPS for Sec. 7.2 without conserved charges)."""
    A = []
    left = QNIndex([((0,) * site_index.nq, 1)], OUT)
    for v in vecs:
        v = np.asarray(v, dtype=np.float64)
        v = v / np.linalg.norm(v)
        inds = [left, site_index, left.dag()]
        A.append(BlockTensor.from_dense(v.reshape(1, -1, 1), inds))
    return A


# ------------------------------------- sums of MPOs and excited states
def overlap_left(LO, P, A):
    """LO'[pb, b] = sum LO[pa, a] P[pa, s, pb] A[a, s, b].

    The overlap of a previous state P with the current MPS A over the sites
    left of a bond (Sec. 7.2, excited states). Real data: the bra is P with
    its arrows reversed.
    """
    LO = LO.relabel(["pa", "a"])
    Pb = dag(P).relabel(["pa", "s", "pb"])
    Ak = A.relabel(["a", "s", "b"])
    return contract(contract(LO, Pb), Ak, out_labels=["pb", "b"])


def overlap_right(RO, P, A):
    """RO'[pa, a] = sum P[pa, s, pb] A[a, s, b] RO[pb, b]: one site of the
    overlap with a previous state (Sec. 7.2, excited states)."""
    RO = RO.relabel(["pb", "b"])
    Pb = dag(P).relabel(["pa", "s", "pb"])
    Ak = A.relabel(["a", "s", "b"])
    return contract(contract(Pb, RO), Ak, out_labels=["pa", "a"])


def overlap_boundaries(P, A):
    """LO_0 and RO_N: 1 on the boundary links (both of dimension 1), or no
    block at all when the two states carry different total charge."""
    N = len(A)
    LO = BlockTensor.zeros([P[0].inds[0], A[0].inds[0].dag()])
    RO = BlockTensor.zeros([P[N - 1].inds[2], A[N - 1].inds[2].dag()])
    for T in (LO, RO):
        for v in T.blocks.values():
            v[0, 0] = 1.0
    return LO, RO


def projected_state(LO, P1, P2, RO):
    """phi[a, s1, s2, b] = sum LO[pa, a] P1[pa, s1, pc] P2[pc, s2, pb] RO[pb, b].

    The previous state P written in the two-site basis of the current MPS
    (left-orthogonal left of the bond, right-orthogonal right of it): the
    vector whose projector, times the weight, is added to H_eff. The
    contraction gives the bra; with real data its arrow-reversed copy is the
    ket in theta's layout.
    """
    t = contract(LO.relabel(["pa", "a"]), dag(P1).relabel(["pa", "s1", "pc"]))
    t = contract(t, dag(P2).relabel(["pc", "s2", "pb"]))
    t = contract(t, RO.relabel(["pb", "b"]), out_labels=["a", "s1", "s2", "b"])
    return dag(t)


def dmrg(mpo, mps, sweeps, krylov_dim=64, tol=1e-10, mindim=1, observer=None,
         ortho=(), weight=1.0):
    """Two-site DMRG (Sec. 7.2) with the schedule ``sweeps``.

    ``sweeps`` is a list of (maxdim, cutoff), one entry per sweep. The MPS
    must be right-orthogonal from site 1 on (a normalised product state
    is). Reading used where the paper is silent: a sweep is a left-to-right
    pass over bonds (0,1)..(N-2,N-1) followed by a right-to-left pass over
    the same bonds in reverse; each bond runs Lanczos from the current
    two-site state, splits it with the truncated SVD (U -> A_j and S V ->
    A_{j+1} going right, U S -> A_j and V -> A_{j+1} going left) and updates
    one environment. No noise or subspace expansion. The returned energy is
    the eigenvalue at the last bond of the last sweep. Each sweep's stats hold
    its last energy, the largest link dimension, the largest and the summed
    truncation error of its bonds (svd_trunc's relative discarded weight) and
    its Lanczos products.

    ``mpo`` may be a list of MPOs: H is their sum (Sec. 7.2), kept as
    separate terms, each with its own environments, and H_eff . x is the
    sum of the terms' products. ``ortho`` lists previous states (MPS): the
    projector onto each, times ``weight``, is added to H (Sec. 7.2, excited
    states), so H_eff . x gains weight * phi <phi, x> per previous state,
    phi being that state in the current two-site basis.
    """
    mpos = list(mpo) if isinstance(mpo, (list, tuple)) else [mpo]
    N = len(mpos[0].W)
    A = [a.copy() for a in mps]
    T = len(mpos)
    Ls = [[None] * (N + 1) for _ in range(T)]
    Rs = [[None] * (N + 1) for _ in range(T)]
    for t, m in enumerate(mpos):
        Ls[t][0] = left_boundary(A[0], m.W[0], m.start)
        Rs[t][N] = right_boundary(A[N - 1], m.W[N - 1], m.done)
        for j in range(N - 1, 1, -1):
            Rs[t][j] = env_right(Rs[t][j + 1], A[j], m.W[j])
    P = [list(p) for p in ortho]
    LO = [[None] * (N + 1) for _ in P]
    RO = [[None] * (N + 1) for _ in P]
    for i, p in enumerate(P):
        LO[i][0], RO[i][N] = overlap_boundaries(p, A)
        for j in range(N - 1, 1, -1):
            RO[i][j] = overlap_right(RO[i][j + 1], p[j], A[j])
    energy = None
    stats = []
    for sw, (maxdim, cutoff) in enumerate(sweeps):
        maxerr, sumerr, nmv = 0.0, 0.0, 0
        for j, direction in [(j, +1) for j in range(N - 1)] + \
                            [(j, -1) for j in range(N - 2, -1, -1)]:
            th = theta(A[j], A[j + 1])
            phis = [projected_state(LO[i][j], p[j], p[j + 1], RO[i][j + 2])
                    for i, p in enumerate(P)]

            def apply(x, j=j, phis=phis):
                y = None
                for t, m in enumerate(mpos):
                    yt = heff_apply(Ls[t][j], m.W[j], m.W[j + 1], Rs[t][j + 2], x)
                    y = yt if y is None else y.axpy(1.0, yt)
                for phi in phis:
                    y = y.axpy(weight * phi.vdot(x), phi)
                return y

            energy, th, res, k = lanczos(apply, th, krylov_dim, tol)
            nmv += k
            U, S, V, err = svd_trunc(th, 2, cutoff, maxdim, mindim)
            maxerr = max(maxerr, err)
            sumerr += err
            if direction > 0:
                A[j] = U
                A[j + 1] = scale_link(V, S, 0)
                for t, m in enumerate(mpos):
                    Ls[t][j + 1] = env_left(Ls[t][j], A[j], m.W[j])
                for i, p in enumerate(P):
                    LO[i][j + 1] = overlap_left(LO[i][j], p[j], A[j])
            else:
                A[j] = scale_link(U, S, 2)
                A[j + 1] = V
                for t, m in enumerate(mpos):
                    Rs[t][j + 1] = env_right(Rs[t][j + 2], A[j + 1], m.W[j + 1])
                for i, p in enumerate(P):
                    RO[i][j + 1] = overlap_right(RO[i][j + 2], p[j + 1], A[j + 1])
        st = dict(sweep=sw, energy=energy, maxdim=max(a.inds[2].dim for a in A),
                  truncerr=maxerr, truncerr_sum=sumerr, matvecs=nmv)
        stats.append(st)
        if observer:
            observer(st)
    return energy, A, stats


def mps_overlap(P, A):
    """<P|A> of two MPS (real data), by a left-to-right overlap sweep
    (the MPS inner product of Sec. 7.3)."""
    LO, _ = overlap_boundaries(P, A)
    for j in range(len(A)):
        LO = overlap_left(LO, P[j], A[j])
    return sum(float(np.sum(v)) for v in LO.blocks.values())


def mps_expectation(mpo, A):
    """<psi|H|psi>/<psi|psi> by full left-to-right environment sweeps
    (``mpo`` may be a list of MPOs: the sum of their expectations)."""
    num = 0.0
    for m in (list(mpo) if isinstance(mpo, (list, tuple)) else [mpo]):
        W = m.W
        N = len(W)
        L = left_boundary(A[0], W[0], m.start)
        for j in range(N):
            L = env_left(L, A[j], W[j])
        Rb = right_boundary(A[N - 1], W[N - 1], m.done)
        num += L.vdot(Rb)
    a0 = A[0].inds[0]
    E = BlockTensor.zeros([a0.dag(), a0])
    for v in E.blocks.values():
        v[0, 0] = 1.0
    for j in range(N):
        t = contract(E.relabel(["a", "ap"]), A[j].relabel(["a", "s", "b"]))
        E = contract(t, dag(A[j]).relabel(["ap", "s", "bp"]), out_labels=["b", "bp"])
    n2 = sum(float(np.sum(v)) for v in E.blocks.values())
    return num / n2
