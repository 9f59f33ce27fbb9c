"""Model Hamiltonians as MPO tensors for the library (host arrays + QN indices).

An MPO site tensor is W[wl, wr, s, s'] = <s'| op(wl, wr) |s> with arrows
(wl In, wr Out, s In, s' Out); a block is allowed when
q(wr) = q(wl) + q(s) - q(s'). The MPO is lower triangular: the left
boundary selects link state ``start`` and the right boundary ``done``.

* ``heisenberg``     S=1/2 chain, H = sum S_i . S_{i+1} (Eq. (1) of Sec. 7.1);
                     bulk bond dimension 5 as the paper states; rows/columns
                     (I, S+, S-, Sz, I).
* ``spin_pairs``     sum over arbitrary pairs J_ij S_i . S_j (J1-J2 chains and
                     snake-ordered cylinders); one open link state per
                     (first site, operator type).
* ``hubbard``        Fermi-Hubbard chain with Jordan-Wigner strings, (N, 2Sz)
                     charges, bulk bond dimension 6.
* ``tfim``           transverse-field Ising chain (no U(1) charge).

``to_device`` turns the host description into ``tnh.Tensor`` objects.
"""
from __future__ import annotations

import numpy as np

# S=1/2 basis: 0 = up (2Sz=+1), 1 = down (2Sz=-1); op[s_out, s_in]
_SZ = np.diag([0.5, -0.5])
_SP = np.array([[0.0, 1.0], [0.0, 0.0]])
_SM = _SP.T.copy()
_X = np.array([[0.0, 1.0], [1.0, 0.0]])
_Z = np.diag([1.0, -1.0])
SPIN_QN = [(1,), (-1,)]

# Hubbard basis: |0>, |up>, |dn>, |up dn> = c+_up c+_dn |0>; charges (N, 2Sz)
HUB_QN = [(0, 0), (1, 1), (1, -1), (2, 0)]


def _hub_ops():
    cu = np.zeros((4, 4))
    cd = np.zeros((4, 4))
    # c_up: |up> -> |0>, |updn> -> |dn> (up is first in the site's JW order)
    cu[0, 1] = 1.0
    cu[2, 3] = 1.0
    # c_dn: |dn> -> |0>, |updn> = c+_up c+_dn|0> -> c_dn c+_up c+_dn |0> = -|up>
    cd[0, 2] = 1.0
    cd[1, 3] = -1.0
    parity = np.diag([1.0, -1.0, -1.0, 1.0])
    return cu, cd, parity


class HostMPO:
    """List of site tensors W[j] (numpy) with link charges and boundaries."""

    def __init__(self, W, link_qn, site_qn, start, done):
        self.W = W                # list of arrays [wl, wr, d, d]
        self.link_qn = link_qn    # list of N+1 lists of charges (one per link state)
        self.site_qn = site_qn
        self.start = start
        self.done = done

    @property
    def N(self):
        return len(self.W)

    def max_bond(self):
        return max(w.shape[1] for w in self.W)


def _charge(op, site_qn):
    nz = np.argwhere(op != 0)
    if len(nz) == 0:
        return tuple(0 for _ in site_qn[0])
    ch = {tuple(np.subtract(site_qn[o], site_qn[i])) for o, i in nz}
    if len(ch) != 1:
        raise ValueError("operator without a definite charge")
    return tuple(int(v) for v in ch.pop())


def heisenberg(N):
    """Bulk 5x5 Heisenberg tensor at every site; start = 4, done = 0."""
    W = np.zeros((5, 5, 2, 2))
    ops = {(0, 0): np.eye(2), (1, 0): _SP, (2, 0): _SM, (3, 0): _SZ,
           (4, 1): 0.5 * _SM, (4, 2): 0.5 * _SP, (4, 3): _SZ, (4, 4): np.eye(2)}
    for (r, c), op in ops.items():
        W[r, c] = op.T
    qn = [(0,), (2,), (-2,), (0,), (0,)]
    return HostMPO([W.copy() for _ in range(N)], [list(qn) for _ in range(N + 1)], SPIN_QN, 4, 0)


def _pair_mpo(N, site_qn, onsite, terms):
    """terms: list of (i, j, type, coef, op_i, op_j), i < j. States per bond:
    done, open (i, type) for every first site still waiting for a partner, start."""
    d = len(site_qn)
    nq = len(site_qn[0])
    opener, last = {}, {}
    for i, j, ty, c, oi, oj in terms:
        key = (i, ty)
        if key in opener and not np.array_equal(opener[key], oi):
            raise ValueError("one opening operator per (site, type)")
        opener[key] = oi
        last[key] = max(last.get(key, j), j)
    states = []
    for b in range(N + 1):
        # link b sits between sites b-1 and b; (i, type) is open from the
        # link right of site i up to the link left of its last partner
        mid = [k for k in sorted(opener) if k[0] < b <= last[k]]
        states.append(["done"] + mid + ["start"])
    link_qn = []
    for b in range(N + 1):
        q = []
        for st in states[b]:
            if st in ("done", "start"):
                q.append((0,) * nq)
            else:
                q.append(tuple(-v for v in _charge(opener[st], site_qn)))
        link_qn.append(q)
    W = []
    for j in range(N):
        L, R = states[j], states[j + 1]
        li = {s: n for n, s in enumerate(L)}
        ri = {s: n for n, s in enumerate(R)}
        T = np.zeros((len(L), len(R), d, d))
        T[li["done"], ri["done"]] += np.eye(d)
        T[li["start"], ri["start"]] += np.eye(d)
        if onsite is not None and onsite[j] is not None:
            T[li["start"], ri["done"]] += onsite[j].T
        for key, oi in opener.items():
            if key[0] == j:
                T[li["start"], ri[key]] += oi.T
            elif key[0] < j < last[key]:
                T[li[key], ri[key]] += np.eye(d)
        for i, jj, ty, c, oi, oj in terms:
            if jj == j:
                T[li[(i, ty)], ri["done"]] += c * oj.T
        W.append(T)
    return HostMPO(W, link_qn, site_qn, len(states[0]) - 1, 0)


def spin_pairs(N, pairs):
    """sum_(i,j,J) J S_i . S_j for S=1/2 sites with (2Sz,) charges."""
    terms = []
    for i, j, J in pairs:
        i, j = min(i, j), max(i, j)
        terms += [(i, j, 0, 0.5 * J, _SP, _SM), (i, j, 1, 0.5 * J, _SM, _SP), (i, j, 2, J, _SZ, _SZ)]
    return _pair_mpo(N, SPIN_QN, None, terms)


def j1j2_chain(N, J1=1.0, J2=0.5):
    return spin_pairs(N, [(i, i + 1, J1) for i in range(N - 1)] + [(i, i + 2, J2) for i in range(N - 2)])


def cylinder_pairs(Lx, Ly, J1=1.0, J2=0.5):
    """J1-J2 square lattice, periodic in y, snake-ordered (up even columns)."""
    def site(x, y):
        return x * Ly + (y if x % 2 == 0 else Ly - 1 - y)
    acc = {}
    for x in range(Lx):
        for y in range(Ly):
            bonds = [(site(x, (y + 1) % Ly), J1)]
            if x + 1 < Lx:
                bonds += [(site(x + 1, y), J1), (site(x + 1, (y + 1) % Ly), J2),
                          (site(x + 1, (y - 1) % Ly), J2)]
            for t, J in bonds:
                a, b = sorted((site(x, y), t))
                acc[(a, b)] = acc.get((a, b), 0.0) + J
    return [(a, b, J) for (a, b), J in sorted(acc.items())]


def hubbard(N, t=1.0, U=4.0):
    cu, cd, F = _hub_ops()
    terms = []
    for i in range(N - 1):
        for ty, c in enumerate((cu, cd)):
            # -t (c+_i c_{i+1} + c+_{i+1} c_i) with the parity string on site i
            terms.append((i, i + 1, 2 * ty, -t, c.T @ F, c))
            terms.append((i, i + 1, 2 * ty + 1, t, c @ F, c.T))
    n_up = cu.T @ cu
    n_dn = cd.T @ cd
    return _pair_mpo(N, HUB_QN, [U * n_up @ n_dn] * N, terms)


def tfim(N, J=1.0, h=1.0):
    """H = -J sum X X - h sum Z; charges are all zero (one trivial sector)."""
    terms = [(i, i + 1, 0, -J, _X, _X) for i in range(N - 1)]
    m = _pair_mpo(N, [(0,), (0,)], [-h * _Z] * N, terms)
    return m


def site_index(site_qn, qn=True):
    from .tnh import Index
    if qn:
        return Index([(q, 1) for q in site_qn], +1)
    return Index.dense(len(site_qn), +1, nq=len(site_qn[0]))


def to_device(mpo, qn=True):
    """MPO as a list of tnh.Tensor [wl (In), wr (Out), s (In), s' (Out)].

    With ``qn`` every link state and site state is its own sector; without,
    every index is one trivial sector (dense storage).
    """
    import torch
    from .tnh import Index, Tensor
    out = []
    nq = len(mpo.site_qn[0])
    s = site_index(mpo.site_qn, qn)
    for j, W in enumerate(mpo.W):
        if qn:
            wl = Index([(q, 1) for q in mpo.link_qn[j]], -1)
            wr = Index([(q, 1) for q in mpo.link_qn[j + 1]], +1)
        else:
            wl = Index.dense(W.shape[0], -1, nq=nq)
            wr = Index.dense(W.shape[1], +1, nq=nq)
        T = Tensor([wl, wr, s.dag(), s])

        def block(key, shp, W=W, T=T):
            sl = []
            for ax, sec in enumerate(key):
                o = sum(dd for _, dd in T.inds[ax].sectors[:sec])
                sl.append(slice(o, o + T.inds[ax].sectors[sec][1]))
            return W[tuple(sl)]
        # check nothing lies outside the allowed blocks
        tot = np.abs(W).sum()
        got = sum(np.abs(block(k, None)).sum() for k in T.blocks)
        if abs(tot - got) > 1e-12 * max(1.0, tot):
            raise ValueError(f"MPO site {j} has weight outside its allowed blocks")
        T.fill(block)
        out.append(T)
    return out


def splitblocks(mpo, qn=True):
    """MPO as device tensors in the sparse form of ``splitblocks`` (Sec. 12.2):
    every link state is a sector of its own (dimension 1, its charge, or the
    trivial charge without ``qn``) and only the blocks holding a nonzero
    entry are stored. The site index keeps the layout of ``to_device``.
    H_eff applies only nonzero MPO entries either way; the environment
    update's contraction with W then skips the zero blocks too."""
    from .tnh import Index, Tensor
    nq = len(mpo.site_qn[0])
    s = site_index(mpo.site_qn, qn)
    zero = (0,) * nq
    out = []
    for j, W in enumerate(mpo.W):
        wl = Index([(q if qn else zero, 1) for q in mpo.link_qn[j]], -1)
        wr = Index([(q if qn else zero, 1) for q in mpo.link_qn[j + 1]], +1)
        inds = [wl, wr, s.dag(), s]
        soff = np.cumsum([0] + [d for _, d in s.sectors])
        blocks, offs, data = [], [], []
        pos = 0
        for a in range(W.shape[0]):
            for b in range(W.shape[1]):
                for u in range(s.nsect):
                    for v in range(s.nsect):
                        blk = W[a, b, soff[u]:soff[u + 1], soff[v]:soff[v + 1]]
                        if not np.any(blk != 0.0):
                            continue
                        if qn:
                            # the block must carry the tensor's (zero) flux
                            f = tuple(-x + y - p + q for x, y, p, q in
                                      zip(wl.sectors[a][0], wr.sectors[b][0], s.sectors[u][0], s.sectors[v][0]))
                            if any(f):
                                raise ValueError(f"MPO site {j} has weight outside its allowed blocks")
                        blocks.append((a, b, u, v))
                        offs.append(pos)
                        data.append(blk.ravel())
                        pos += blk.size
        T = Tensor(inds, None, blocks=blocks, offsets=offs)
        host = np.concatenate(data) if data else np.zeros(1)
        import torch
        T.data = torch.from_numpy(np.ascontiguousarray(host)).to(T.data.device)
        out.append(T)
    return out


def product_state(site, states):
    """MPS (list of tnh.Tensor [left, s, right]) of a product of basis states.

    ``states[j]`` is the sector number of site j's state; every link has one
    sector (dim 1) carrying the total charge to its left.
    """
    from .tnh import Index, Tensor
    nq = site.nq
    q = (0,) * nq
    left = Index([(q, 1)], +1)
    out = []
    for st in states:
        q = tuple(a + b for a, b in zip(q, site.sectors[st][0]))
        right = Index([(q, 1)], +1)
        T = Tensor([left, site, right.dag()], None)
        T.fill(lambda k, shp: np.ones(shp))
        out.append(T)
        left = right
    return out


def product_vectors(site, vecs):
    """MPS of a product state with one (normalised) vector per site; one
    trivial link sector (site must be a dense index)."""
    from .tnh import Index, Tensor
    link = Index([((0,) * site.nq, 1)], +1)
    out = []
    for v in vecs:
        v = np.asarray(v, dtype=np.float64)
        v = v / np.linalg.norm(v)
        T = Tensor([link, site, link.dag()], None)
        T.fill(lambda k, shp, v=v: v.reshape(shp))
        out.append(T)
    return out
