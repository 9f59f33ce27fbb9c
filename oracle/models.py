"""Site operators, operator-term lists and finite-state MPOs (oracle side).

Test infrastructure (see the package header).

Conventions (real arithmetic throughout):

* an operator matrix ``op[s_out, s_in]`` acts on a site ket;
* an MPO tensor is ``W[wl, wr, s, s']`` with ``s`` the ket index it consumes
  and ``s'`` the ket index it produces, so ``W[wl, wr, s, s'] =
  op(wl, wr)[s', s]``;
* the MPO is lower triangular: the left boundary selects the ``start`` state
  and the right boundary the ``done`` state; the product of the W's along the
  chain between those two states is the Hamiltonian;
* QNs are integer tuples; S=1/2 sites carry (2 Sz,), Hubbard sites carry
  (N, 2 Sz). Index arrows follow Sec. 8.2: the MPO has ``wl`` In, ``wr`` Out,
  ``s`` In, ``s'`` Out, so a block is allowed when
  ``q(wr) = q(wl) + q(s) - q(s')`` (a link state carries minus the charge that
  the operators placed to its left have added).

The Heisenberg Hamiltonian is Eq. (1) of Sec. 7.1, whose exact MPO has bond
dimension 5. The paper does not print the matrix; the reading used is the
standard lower-triangular form with rows/columns (I, S+, S-, Sz, I):
``W[0,0]=I, W[1,0]=S+, W[2,0]=S-, W[3,0]=Sz, W[4,1]=S-/2, W[4,2]=S+/2,
W[4,3]=Sz, W[4,4]=I``, left boundary row 4, right boundary column 0.
The other models (TFIM, J1-J2, Hubbard) are not in the paper; they are the
workloads named for the benchmarks and serve as pins.
"""
from __future__ import annotations

import numpy as np

from .blocksparse import BlockTensor, IN, OUT, QNIndex, trivial_index

# ---------------------------------------------------------------- S = 1/2
# basis: 0 = up (2Sz = +1), 1 = down (2Sz = -1)
SZ = np.array([[0.5, 0.0], [0.0, -0.5]])
SP = np.array([[0.0, 1.0], [0.0, 0.0]])   # |up><dn|
SM = np.array([[0.0, 0.0], [1.0, 0.0]])   # |dn><up|
ID2 = np.eye(2)
PX = np.array([[0.0, 1.0], [1.0, 0.0]])   # Pauli X
PZ = np.array([[1.0, 0.0], [0.0, -1.0]])  # Pauli Z
SPIN_QN = [(1,), (-1,)]

# ------------------------------------------------------------- Hubbard site
# basis: 0 = |0>, 1 = |up>, 2 = |dn>, 3 = |up dn> = c+_up c+_dn |0>.
# Inside a site the up mode precedes the down mode in the Jordan-Wigner order.
def _hubbard_site_ops():
    # two modes (up, dn); state index = n_up + 2 n_dn
    a = np.array([[0.0, 1.0], [0.0, 0.0]])      # annihilator on one mode
    z = np.diag([1.0, -1.0])                    # (-1)^n on one mode
    i2 = np.eye(2)
    # kron ordering: index = n_up + 2 n_dn -> dn is the slow factor
    c_up = np.kron(i2, a)                       # first mode, no string
    c_dn = np.kron(a, z)                        # second mode, string over up
    # map state order (n_up + 2 n_dn) = (|0>,|up>,|dn>,|updn>) matches basis
    return c_up, c_dn


C_UP, C_DN = _hubbard_site_ops()
CD_UP, CD_DN = C_UP.T.copy(), C_DN.T.copy()
N_UP = CD_UP @ C_UP
N_DN = CD_DN @ C_DN
F_SITE = np.diag([1.0, -1.0, -1.0, 1.0])          # (-1)^(n_up + n_dn)
ID4 = np.eye(4)
HUB_QN = [(0, 0), (1, 1), (1, -1), (2, 0)]


def op_charge(op, site_qn):
    """Charge q(s_out) - q(s_in) that a definite-charge operator adds: its
    flux (Sec. 8.3)."""
    nz = np.argwhere(np.abs(op) > 0)
    if len(nz) == 0:
        return tuple(0 for _ in site_qn[0])
    charges = {tuple(np.subtract(site_qn[o], site_qn[i])) for o, i in nz}
    if len(charges) != 1:
        raise ValueError("operator has no definite charge")
    return tuple(int(x) for x in charges.pop())


# ----------------------------------------------------------- term lists
# A term is (coef, [(site, op_matrix), ...]) with distinct sites; the full
# operator is coef * tensor product of the listed matrices (identity
# elsewhere). The ED module builds H from these lists, independently of the
# MPO construction below.

def heisenberg_pairs(N, J=1.0):
    """Open chain, Eq. (1) of Sec. 7.1 (J = 1)."""
    return [(i, i + 1, J) for i in range(N - 1)]


def j1j2_chain_pairs(N, J1=1.0, J2=0.5):
    return [(i, i + 1, J1) for i in range(N - 1)] + \
           [(i, i + 2, J2) for i in range(N - 2)]


def snake_site(x, y, Ly):
    """Snake ordering on a cylinder: up the even columns, down the odd ones."""
    return x * Ly + (y if x % 2 == 0 else Ly - 1 - y)


def j1j2_cylinder_pairs(Lx, Ly, J1=1.0, J2=0.5):
    """Square lattice, periodic in y (Ly sites), open in x, snake ordered.

    J1 on nearest neighbours (vertical bonds wrap around), J2 on both
    diagonals of every plaquette. For Ly = 2 the wrapped bond doubles the
    vertical one; that case is not used.
    """
    pairs = {}

    def add(a, b, J):
        i, j = min(a, b), max(a, b)
        pairs[(i, j)] = pairs.get((i, j), 0.0) + J

    for x in range(Lx):
        for y in range(Ly):
            s = snake_site(x, y, Ly)
            add(s, snake_site(x, (y + 1) % Ly, Ly), J1)
            if x + 1 < Lx:
                add(s, snake_site(x + 1, y, Ly), J1)
                add(s, snake_site(x + 1, (y + 1) % Ly, Ly), J2)
                add(s, snake_site(x + 1, (y - 1) % Ly, Ly), J2)
    return [(i, j, J) for (i, j), J in sorted(pairs.items())]


def spin_pair_terms(pairs):
    """S_i . S_j = Sz Sz + (S+ S- + S- S+)/2 for each (i, j, J), the bond
    term of Eq. (1) in Sec. 7.1."""
    terms = []
    for i, j, J in pairs:
        terms.append((J, [(i, SZ), (j, SZ)]))
        terms.append((0.5 * J, [(i, SP), (j, SM)]))
        terms.append((0.5 * J, [(i, SM), (j, SP)]))
    return terms


def tfim_terms(N, J=1.0, h=1.0):
    """H = -J sum X_i X_{i+1} - h sum Z_i (open chain)."""
    terms = [(-J, [(i, PX), (i + 1, PX)]) for i in range(N - 1)]
    terms += [(-h, [(i, PZ)]) for i in range(N)]
    return terms


def hubbard_terms(N, t=1.0, U=4.0):
    """H = -t sum_{i,s} (c+_{i s} c_{i+1 s} + h.c.) + U sum n_up n_dn.

    Jordan-Wigner over the mode order (1 up, 1 dn, 2 up, 2 dn, ...). For
    neighbouring sites the strings reduce to one parity factor on site i:
    c+_{i s} c_{i+1 s} = (c+_s F)_i (c_s)_{i+1} and
    c+_{i+1 s} c_{i s} = -(c_s F)_i (c+_s)_{i+1}.
    """
    terms = []
    for i in range(N - 1):
        for cd, c in ((CD_UP, C_UP), (CD_DN, C_DN)):
            terms.append((-t, [(i, cd @ F_SITE), (i + 1, c)]))
            terms.append((t, [(i, c @ F_SITE), (i + 1, cd)]))
    terms += [(U, [(i, N_UP @ N_DN)]) for i in range(N)]
    return terms


# ------------------------------------------------------------ MPO builder
class MPO:
    """Site-dependent MPO: ``W[j]`` is a BlockTensor [wl, wr, s, s'].

    ``start``/``done`` are the link-state numbers that the left/right
    boundary environments select (on the first site's wl and last site's wr).
    """

    def __init__(self, W, site_index, start, done):
        self.W = W
        self.site_index = site_index
        self.start = start
        self.done = done

    @property
    def N(self):
        return len(self.W)

    def max_bond(self):
        return max(w.inds[1].dim for w in self.W)


def _link_index(states, qns, arrow):
    return QNIndex([(q, 1) for q in qns], arrow)


def fsa_mpo(N, site_ops_qn, onsite, pairs_ops):
    """Finite-state-automaton MPO for on-site terms plus two-site products.

    An exact MPO of a sum of operator products, as OpSum/AutoMPO builds
    one (Sec. 7.1).

    ``onsite[i]``: matrix (or None) added at site i.
    ``pairs_ops``: list of (i, j, [(coef, op_i, op_j), ...]) with i < j; the
    operator between i and j is the identity (strings, if any, are already
    folded into op_i). Position k in the list is the term's type: every pair
    starting at site i must use the same op_i for type k, so one open state
    (i, k) serves all partners j of site i.
    Link states on bond b (between sites b and b+1): ``done``, one state per
    open (i, k) with i <= b < (last partner of i), and ``start``. Every state
    is a sector of dimension 1 whose QN is minus the charge of the operator
    that opened it.
    """
    site_qn = site_ops_qn
    d = len(site_qn)
    nq = len(site_qn[0])
    zero = (0,) * nq
    first_op, last_j, closers = {}, {}, {}
    for i, j, lst in pairs_ops:
        for k, (c, op_i, op_j) in enumerate(lst):
            st = (i, k)
            if st in first_op and not np.array_equal(first_op[st], op_i):
                raise ValueError("pairs from one site must share op_i per type")
            first_op[st] = op_i
            last_j[st] = max(last_j.get(st, j), j)
            closers.setdefault(j, []).append((st, c, op_j))
    opens = [[] for _ in range(N - 1)]
    for st in sorted(first_op):
        for b in range(st[0], last_j[st]):
            opens[b].append(st)

    def states(b):
        # bond b in [-1, N-1]; -1 and N-1 are the boundary links
        if b < 0 or b >= N - 1:
            return ["done", "start"]
        return ["done"] + opens[b] + ["start"]

    def state_qn(st):
        if st in ("done", "start"):
            return zero
        return tuple(-x for x in op_charge(first_op[st], site_qn))

    site = QNIndex([(q, 1) for q in site_qn], OUT)
    W = []
    for j in range(N):
        left, right = states(j - 1), states(j)
        li = {s: n for n, s in enumerate(left)}
        ri = {s: n for n, s in enumerate(right)}
        arr = np.zeros((len(left), len(right), d, d))

        def put(sl, sr, op):
            arr[li[sl], ri[sr]] += op.T   # W[wl,wr,s,s'] = op[s',s]

        put("done", "done", np.eye(d))
        put("start", "start", np.eye(d))
        if onsite[j] is not None:
            put("start", "done", onsite[j])
        for st in first_op:
            if st[0] == j:
                put("start", st, first_op[st])
            elif st[0] < j < last_j[st]:
                put(st, st, np.eye(d))
        for st, c, op_j in closers.get(j, []):
            put(st, "done", c * op_j)
        wl = _link_index(left, [state_qn(s) for s in left], IN)
        wr = _link_index(right, [state_qn(s) for s in right], OUT)
        inds = [wl, wr, site.dag(), site]
        W.append(BlockTensor.from_dense(arr, inds, None))
    return MPO(W, site, start=1, done=0)


def heisenberg_like_mpo(N, pairs):
    """MPO of sum_(i,j,J) J S_i . S_j with S=1/2 sites and (2Sz,) QNs (the
    bond terms of Eq. (1), Sec. 7.1, on any set of pairs)."""
    plist = [(i, j, [(0.5 * J, SP, SM), (0.5 * J, SM, SP), (J, SZ, SZ)])
             for i, j, J in pairs]
    return fsa_mpo(N, SPIN_QN, [None] * N, plist)


def tfim_mpo(N, J=1.0, h=1.0):
    """TFIM MPO; no U(1) symmetry, so every index is one trivial sector."""
    d = 2
    W = []
    for j in range(N):
        wl = 2 if j == 0 else 3
        wr = 2 if j == N - 1 else 3
        bulk = np.zeros((3, 3, d, d))
        bulk[0, 0] = ID2.T
        bulk[1, 0] = PX.T
        bulk[2, 0] = (-h * PZ).T
        bulk[2, 1] = (-J * PX).T
        bulk[2, 2] = ID2.T
        # boundary links keep only done(0) and start(2)
        rows = [0, 2] if j == 0 else [0, 1, 2]
        cols = [0, 2] if j == N - 1 else [0, 1, 2]
        arr = bulk[np.ix_(rows, cols)]
        inds = [trivial_index(len(rows), IN), trivial_index(len(cols), OUT),
                trivial_index(d, IN), trivial_index(d, OUT)]
        W.append(BlockTensor.from_dense(arr, inds))
    site = trivial_index(d, OUT)
    return MPO(W, site, start=1, done=0)


def hubbard_mpo(N, t=1.0, U=4.0):
    """Hubbard chain MPO with (N, 2Sz) QNs; bulk bond dimension 6. The
    Hubbard model is one of the benchmark systems of Sec. 12.1 (there on a
    cylinder); the charges are those of Sec. 8.1."""
    plist = []
    for i in range(N - 1):
        lst = []
        for cd, c in ((CD_UP, C_UP), (CD_DN, C_DN)):
            lst.append((-t, cd @ F_SITE, c))
            lst.append((t, c @ F_SITE, cd))
        plist.append((i, i + 1, lst))
    onsite = [U * (N_UP @ N_DN) for _ in range(N)]
    return fsa_mpo(N, HUB_QN, onsite, plist)


def heisenberg_bulk_W():
    """The 5x5 bulk Heisenberg tensor as a dense array W[wl, wr, s, s'].

    Rows/columns (I, S+, S-, Sz, I) in the reading stated in the header.
    """
    W = np.zeros((5, 5, 2, 2))
    W[0, 0] = ID2.T
    W[1, 0] = SP.T
    W[2, 0] = SM.T
    W[3, 0] = SZ.T
    W[4, 1] = (0.5 * SM).T
    W[4, 2] = (0.5 * SP).T
    W[4, 3] = SZ.T
    W[4, 4] = ID2.T
    return W


HEIS_LINK_QN = [(0,), (2,), (-2,), (0,), (0,)]


def heisenberg_mpo(N):
    """Heisenberg chain MPO built from the bulk 5x5 tensor of Eq. (1).

    Every site uses the bulk tensor; the boundary environments select row 4
    (start) on the left and column 0 (done) on the right.
    """
    Wb = heisenberg_bulk_W()
    site = QNIndex([(q, 1) for q in SPIN_QN], OUT)
    W = []
    for j in range(N):
        wl = QNIndex([(q, 1) for q in HEIS_LINK_QN], IN)
        wr = QNIndex([(q, 1) for q in HEIS_LINK_QN], OUT)
        W.append(BlockTensor.from_dense(Wb, [wl, wr, site.dag(), site]))
    return MPO(W, site, start=4, done=0)
