"""QN block-sparse tensors and the labelled contraction, in plain numpy float64.

Test infrastructure (see the package header). Follows the ITensor paper:

* QN objects (Sec. 8.1): a QN is a tuple of integers, added and subtracted
  element-wise. Z_N moduli are out of scope (every model here is U(1) or
  U(1)xU(1)).
* QN Index (Sec. 8.2): an ordered list of sectors ``(qn, dim)`` plus an arrow.
  ``OUT`` (+1) is the default; the QNs of an ``OUT`` index are added and those
  of an ``IN`` index subtracted when the flux of a block is computed.
* QN ITensor (Sec. 8.3): only the blocks whose flux equals the tensor's flux
  are stored; contracted index pairs must have opposite arrows.
* Block-sparse storage (Sec. 6, Sec. 9.2): a dictionary from the block's
  sector tuple to a dense array. A dense tensor is the special case of one
  sector per index with an all-zero QN.
* Contraction (Sec. 4, Sec. 9.1, Sec. 9.4): equal labels are summed; a
  block-sparse contraction is the sum of dense contractions over every pair
  of blocks whose contracted sectors agree, several pairs possibly adding
  into the same output block.
"""
from __future__ import annotations

import itertools

import numpy as np

OUT = +1
IN = -1


def qn_add(a, b):
    """Element-wise sum of two QN tuples (Sec. 8.1)."""
    return tuple(int(x) + int(y) for x, y in zip(a, b))


def qn_sub(a, b):
    """Element-wise difference of two QN tuples (Sec. 8.1)."""
    return tuple(int(x) - int(y) for x, y in zip(a, b))


def qn_scale(s, a):
    return tuple(int(s) * int(x) for x in a)


class QNIndex:
    """An index with QN sectors and an arrow (Sec. 8.2).

    ``sectors`` is a list of ``(qn_tuple, dim)``; the element index runs over
    the sectors in the given order. ``label`` is the integer that the labelled
    contraction matches (Sec. 9.1); it stands for the id + prime level pair of
    Sec. 3.
    """

    def __init__(self, sectors, arrow=OUT, label=None):
        self.sectors = [(tuple(int(x) for x in q), int(d)) for q, d in sectors]
        if arrow not in (OUT, IN):
            raise ValueError("arrow must be OUT (+1) or IN (-1)")
        self.arrow = arrow
        self.label = label

    @property
    def nsect(self):
        return len(self.sectors)

    @property
    def nq(self):
        return len(self.sectors[0][0]) if self.sectors else 0

    @property
    def dim(self):
        return sum(d for _, d in self.sectors)

    def qn(self, i):
        return self.sectors[i][0]

    def sdim(self, i):
        return self.sectors[i][1]

    def offset(self, i):
        return sum(d for _, d in self.sectors[:i])

    def sector_of(self, elem):
        """(sector number, position inside the sector) of element ``elem``."""
        for i, (_, d) in enumerate(self.sectors):
            if elem < d:
                return i, elem
            elem -= d
        raise IndexError("element beyond the index dimension")

    def dag(self):
        """Same sectors, reversed arrow (Sec. 8.3: dag reverses arrows)."""
        return QNIndex(self.sectors, -self.arrow, self.label)

    def with_label(self, label):
        return QNIndex(self.sectors, self.arrow, label)

    def same_space(self, other):
        return self.sectors == other.sectors

    def __repr__(self):
        return f"QNIndex({self.sectors}, arrow={self.arrow}, label={self.label})"


def trivial_index(dim, arrow=OUT, label=None, nq=1):
    """A dense index: one sector of dimension ``dim`` with an all-zero QN."""
    return QNIndex([((0,) * nq, dim)], arrow, label)


def block_flux(inds, key, nq=None):
    """Flux of the block ``key``: Out QNs added, In QNs subtracted (Sec. 8.2)."""
    nq = inds[0].nq if inds else (nq or 0)
    f = (0,) * nq
    for ind, s in zip(inds, key):
        f = qn_add(f, qn_scale(ind.arrow, ind.qn(s)))
    return f


def allowed_blocks(inds, flux):
    """All sector tuples whose block flux equals ``flux`` (Sec. 8.3).

    Enumeration of the product of the sectors of all indices but the last,
    in lexicographic order; for each such prefix the flux rule fixes the QN
    the last index must carry, and its sectors with that QN complete the
    tuple in increasing order. The result is the lexicographic list of the
    full product filtered by the flux rule.
    """
    flux = tuple(flux)
    if not inds:
        return [()] if not any(flux) else []
    nq = len(flux)
    last = inds[-1]
    by_qn = {}
    for s in range(last.nsect):
        by_qn.setdefault(tuple(last.qn(s)), []).append(s)
    out = []
    for prefix in itertools.product(*[range(ind.nsect) for ind in inds[:-1]]):
        f = block_flux(inds[:-1], prefix, nq)
        # arrow * q_last = flux - f  ->  q_last = arrow * (flux - f)
        need = qn_scale(last.arrow, qn_sub(flux, f))
        for s in by_qn.get(tuple(need), ()):
            out.append(prefix + (s,))
    return out


class BlockTensor:
    """Block-sparse tensor: indices, flux and a dict sector-tuple -> array
    (block-sparse storage, Sec. 6 and Sec. 9.2; the stored blocks obey the
    flux rule of Sec. 8.3)."""

    def __init__(self, inds, flux=None, blocks=None):
        self.inds = list(inds)
        nq = self.inds[0].nq if self.inds else 0
        self.flux = tuple(flux) if flux is not None else (0,) * nq
        self.blocks = {} if blocks is None else dict(blocks)
        for key, arr in self.blocks.items():
            if arr.shape != self.block_shape(key):
                raise ValueError(f"block {key} has shape {arr.shape}")
            if block_flux(self.inds, key, len(self.flux)) != self.flux:
                raise ValueError(f"block {key} violates the flux {self.flux}")

    # ---- structure -----------------------------------------------------
    @property
    def rank(self):
        return len(self.inds)

    @property
    def shape(self):
        return tuple(ind.dim for ind in self.inds)

    def block_shape(self, key):
        return tuple(ind.sdim(s) for ind, s in zip(self.inds, key))

    def allowed(self):
        return allowed_blocks(self.inds, self.flux)

    @property
    def labels(self):
        return [ind.label for ind in self.inds]

    def nnz(self):
        return sum(int(np.prod(self.block_shape(k))) for k in self.allowed())

    # ---- constructors --------------------------------------------------
    @staticmethod
    def zeros(inds, flux=None):
        t = BlockTensor(inds, flux)
        for key in t.allowed():
            t.blocks[key] = np.zeros(t.block_shape(key))
        return t

    @staticmethod
    def from_blocks_fn(inds, flux, fn):
        """Allocate every allowed block and fill it with ``fn(key, shape)``."""
        t = BlockTensor(inds, flux)
        for key in t.allowed():
            shp = t.block_shape(key)
            t.blocks[key] = np.asarray(fn(key, shp), dtype=np.float64).reshape(shp)
        return t

    @staticmethod
    def from_dense(arr, inds, flux=None, atol=0.0):
        """Cut a full array into the allowed blocks.

        Entries outside the allowed blocks must be zero (within ``atol``),
        otherwise the array does not have the stated flux.
        """
        t = BlockTensor(inds, flux)
        arr = np.asarray(arr, dtype=np.float64)
        if arr.shape != t.shape:
            raise ValueError("shape mismatch")
        mask = np.zeros(arr.shape, dtype=bool)
        for key in t.allowed():
            sl = tuple(slice(ind.offset(s), ind.offset(s) + ind.sdim(s))
                       for ind, s in zip(t.inds, key))
            t.blocks[key] = arr[sl].copy()
            mask[sl] = True
        rest = np.abs(arr[~mask]).max() if (~mask).any() else 0.0
        if rest > atol:
            raise ValueError(f"array has weight {rest} outside the flux {t.flux}")
        return t

    def to_dense(self):
        out = np.zeros(self.shape)
        for key, arr in self.blocks.items():
            sl = tuple(slice(ind.offset(s), ind.offset(s) + ind.sdim(s))
                       for ind, s in zip(self.inds, key))
            out[sl] = arr
        return out

    # ---- elementwise -----------------------------------------------------
    def copy(self):
        return BlockTensor(self.inds, self.flux,
                           {k: v.copy() for k, v in self.blocks.items()})

    def scaled(self, s):
        return BlockTensor(self.inds, self.flux,
                           {k: s * v for k, v in self.blocks.items()})

    def norm(self):
        return float(np.sqrt(sum(float(np.sum(v * v)) for v in self.blocks.values())))

    def vdot(self, other):
        """Real inner product over the stored blocks (same index structure)."""
        s = 0.0
        for k, v in self.blocks.items():
            if k in other.blocks:
                s += float(np.sum(v * other.blocks[k]))
        return s

    def axpy(self, a, other):
        """self + a * other, same structure."""
        out = self.copy()
        for k, v in other.blocks.items():
            if k in out.blocks:
                out.blocks[k] = out.blocks[k] + a * v
            else:
                out.blocks[k] = a * v
        return out

    def relabel(self, labels):
        return BlockTensor([ind.with_label(l) for ind, l in zip(self.inds, labels)],
                           self.flux, self.blocks)

    def permute(self, perm):
        """Reorder the indices: new index ``j`` is old index ``perm[j]``."""
        inds = [self.inds[p] for p in perm]
        blocks = {tuple(k[p] for p in perm): np.transpose(v, perm)
                  for k, v in self.blocks.items()}
        return BlockTensor(inds, self.flux, blocks)

    def permute_to(self, labels):
        pos = [self.labels.index(l) for l in labels]
        return self.permute(pos)


def contract(A, B, out_labels=None):
    """Labelled contraction ``A * B`` (Sec. 4, Sec. 9.1, Sec. 9.4).

    Indices of ``A`` and ``B`` with equal labels are summed. Contracted pairs
    must have the same sectors and opposite arrows (Sec. 8.3). The free
    indices of ``A`` come first, then those of ``B``, unless ``out_labels``
    gives the order. The flux of the result is the sum of the two fluxes.
    Every pair of stored blocks whose contracted sectors agree contributes
    one dense ``tensordot`` to the output block its free sectors select.
    """
    la, lb = A.labels, B.labels
    if len(set(la)) != len(la) or len(set(lb)) != len(lb):
        raise ValueError("repeated label inside one tensor")
    common = [l for l in la if l in lb]
    ia = [la.index(l) for l in common]
    ib = [lb.index(l) for l in common]
    for p, q in zip(ia, ib):
        if not A.inds[p].same_space(B.inds[q]):
            raise ValueError(f"contracted label {la[p]} has different sectors")
        if A.inds[p].arrow == B.inds[q].arrow:
            raise ValueError(f"contracted label {la[p]} has equal arrows")
    fa = [p for p in range(A.rank) if p not in ia]
    fb = [q for q in range(B.rank) if q not in ib]
    inds = [A.inds[p] for p in fa] + [B.inds[q] for q in fb]
    flux = qn_add(A.flux, B.flux)
    C = BlockTensor(inds, flux)
    for key in C.allowed():
        C.blocks[key] = np.zeros(C.block_shape(key))
    # the blocks of B by their contracted sectors, in B's own order
    by_contracted = {}
    for kb, vb in B.blocks.items():
        by_contracted.setdefault(tuple(kb[q] for q in ib), []).append((kb, vb))
    for ka, va in A.blocks.items():
        for kb, vb in by_contracted.get(tuple(ka[p] for p in ia), ()):
            kc = tuple(ka[p] for p in fa) + tuple(kb[q] for q in fb)
            prod = np.tensordot(va, vb, axes=(ia, ib))
            if kc not in C.blocks:
                # A pair of flux-respecting blocks can only land on an
                # allowed output block; reaching here means a flux error.
                raise AssertionError(f"pair lands on forbidden block {kc}")
            C.blocks[kc] = C.blocks[kc] + prod
    if out_labels is not None:
        C = C.permute_to(list(out_labels))
    return C
