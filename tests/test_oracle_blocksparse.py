"""Pins of the oracle's QN / block-sparse layer against the paper and brute force."""
import json
import os

import numpy as np
import pytest

from oracle.blocksparse import (IN, OUT, BlockTensor, QNIndex, allowed_blocks,
                                block_flux, contract, qn_add, trivial_index)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def test_paper_qn_arithmetic():
    g = load("paper_qn_examples.json")
    for a, b, c in g["qn_sums"]["cases"]:
        assert qn_add(tuple(a), tuple(b)) == tuple(c)


def test_paper_index_dims():
    g = load("paper_qn_examples.json")["index_dims"]
    for case in g["cases"]:
        ind = QNIndex([(tuple(q), d) for q, d in case["sectors"]])
        assert ind.dim == case["dim"]
        assert ind.nsect == len(case["sectors"])


def test_paper_flux_of_set_element():
    g = load("paper_qn_examples.json")["flux_example"]
    i = QNIndex([(tuple(q), d) for q, d in g["i"]])
    j = QNIndex([(tuple(q), d) for q, d in g["j"]])
    # 1-based element numbers as printed in the paper
    si, _ = i.sector_of(g["element"][0] - 1)
    sj, _ = j.sector_of(g["element"][1] - 1)
    assert block_flux([i, j], (si, sj)) == tuple(g["flux"])


def test_paper_boson_operators():
    g = load("paper_qn_examples.json")["boson_ops"]
    s = QNIndex([(tuple(q), d) for q, d in g["s"]])
    inds = [s, s.dag()]              # (s', dag(s))
    # a[s'=>1, s=>2] = 1  -> block (0, 1)
    assert block_flux(inds, (0, 1)) == tuple(g["flux_a"])
    assert len(allowed_blocks(inds, (0,))) == g["n_blocks_flux0"]


def test_paper_block_sparse_example():
    g = load("paper_qn_examples.json")["block_sparse"]
    # charges chosen so that exactly the printed nonzero blocks are allowed
    i1 = QNIndex([((0,), d) for d in g["blockdims"][0][:1]] +
                 [((1,), d) for d in g["blockdims"][0][1:]])
    i2 = QNIndex([((0,), d) for d in g["blockdims"][1][:1]] +
                 [((1,), d) for d in g["blockdims"][1][1:]])
    blocks = allowed_blocks([i1, i2], (1,))
    assert sorted(tuple(k + 1 for k in b) for b in blocks) == \
        sorted(tuple(b) for b in g["nzblocks"])
    T = BlockTensor.zeros([i1, i2], (1,))
    assert T.shape == tuple(g["dims"])
    assert T.nnz() == g["nnz"]


def _brute_contract(A, la, B, lb, lc):
    """Explicit nested loops over every label value (no library contraction)."""
    dims = {}
    for arr, ls in ((A, la), (B, lb)):
        for d, l in zip(arr.shape, ls):
            dims[l] = d
    allb = sorted(dims)
    C = np.zeros([dims[l] for l in lc])
    import itertools
    for vals in itertools.product(*[range(dims[l]) for l in allb]):
        v = dict(zip(allb, vals))
        C[tuple(v[l] for l in lc)] += A[tuple(v[l] for l in la)] * B[tuple(v[l] for l in lb)]
    return C


def test_paper_ndtensors_labelled_contract():
    # contract(A,(-1,1,-2),B,(2,-2,-1)) with A 3x7x2 and B 4x2x3 (Sec. 9.1)
    rng = np.random.default_rng(11)
    A = rng.standard_normal((3, 7, 2))
    B = rng.standard_normal((4, 2, 3))
    la, lb = [-1, 1, -2], [2, -2, -1]
    ia = [trivial_index(d, OUT, l) for d, l in zip(A.shape, la)]
    ib = [trivial_index(d, IN, l) for d, l in zip(B.shape, lb)]
    # labelled indices 1 and 2 are free: give them any arrows
    ib[0] = trivial_index(4, OUT, 2)
    C = contract(BlockTensor.from_dense(A, ia), BlockTensor.from_dense(B, ib))
    assert C.labels == [1, 2]
    np.testing.assert_allclose(C.to_dense(), _brute_contract(A, la, B, lb, [1, 2]),
                               rtol=1e-14, atol=1e-14)


def test_paper_contraction_example():
    # A(a,b,d,c) * B(i,d,j) with a3 b2 c4 d5 i2 j6 (Appendix contraction example)
    rng = np.random.default_rng(12)
    A = rng.standard_normal((3, 2, 5, 4))
    B = rng.standard_normal((2, 5, 6))
    ia = [trivial_index(3, OUT, "a"), trivial_index(2, OUT, "b"),
          trivial_index(5, OUT, "d"), trivial_index(4, OUT, "c")]
    ib = [trivial_index(2, OUT, "i"), trivial_index(5, IN, "d"), trivial_index(6, OUT, "j")]
    C = contract(BlockTensor.from_dense(A, ia), BlockTensor.from_dense(B, ib))
    assert set(C.labels) == {"a", "b", "c", "i", "j"}
    want = _brute_contract(A, ["a", "b", "d", "c"], B, ["i", "d", "j"], C.labels)
    np.testing.assert_allclose(C.to_dense(), want, rtol=1e-13, atol=1e-13)


def test_index_order_independence():
    # A(i,j,k) * B(k,i,j) is the same scalar for any storage order (Sec. 2, 4)
    rng = np.random.default_rng(13)
    A = rng.standard_normal((2, 3, 4))
    B = np.transpose(rng.standard_normal((2, 3, 4)), (2, 0, 1)).copy()  # (k,i,j)
    want = float(np.sum(A * np.transpose(B, (1, 2, 0))))
    ta = BlockTensor.from_dense(A, [trivial_index(2, OUT, "i"), trivial_index(3, OUT, "j"),
                                    trivial_index(4, OUT, "k")])
    tb = BlockTensor.from_dense(B, [trivial_index(4, IN, "k"), trivial_index(2, IN, "i"),
                                    trivial_index(3, IN, "j")])
    for perm in [(0, 1, 2), (2, 0, 1), (1, 2, 0)]:
        c = contract(ta.permute(perm), tb)
        assert c.rank == 0
        got = sum(float(v) for v in c.blocks.values())
        assert abs(got - want) < 1e-12


def _random_qn_index(rng, nsect, arrow, label, maxd=3):
    return QNIndex([((int(q),), int(rng.integers(1, maxd + 1)))
                    for q in range(-nsect // 2, nsect - nsect // 2)], arrow, label)


def test_blocksparse_contract_equals_dense():
    rng = np.random.default_rng(14)
    for trial in range(6):
        i = _random_qn_index(rng, 3, OUT, "i")
        j = _random_qn_index(rng, 4, OUT, "j")
        k = _random_qn_index(rng, 3, OUT, "k")
        l = _random_qn_index(rng, 2, OUT, "l")
        fa, fb = (int(rng.integers(-1, 2)),), (int(rng.integers(-1, 2)),)
        A = BlockTensor.from_blocks_fn([i, j, k], fa, lambda key, s: rng.standard_normal(s))
        B = BlockTensor.from_blocks_fn([k.dag(), l, j.dag()], fb,
                                       lambda key, s: rng.standard_normal(s))
        C = contract(A, B)
        want = np.tensordot(A.to_dense(), B.to_dense(), axes=([1, 2], [2, 0]))
        np.testing.assert_allclose(C.to_dense(), want, rtol=1e-13, atol=1e-13)
        assert C.flux == qn_add(fa, fb)
        # the product stays inside its flux (no weight outside allowed blocks)
        BlockTensor.from_dense(want, C.inds, C.flux, atol=1e-12)


def test_contract_rejects_equal_arrows():
    i = QNIndex([((0,), 1), ((1,), 2)], OUT, "i")
    A = BlockTensor.zeros([i])
    B = BlockTensor.zeros([i])
    with pytest.raises(ValueError):
        contract(A, B)


def test_allowed_blocks_equals_filtered_full_product():
    # the enumeration completes the last sector from the flux rule; it must be
    # the lexicographic full product filtered by the flux rule
    import itertools
    from oracle.blocksparse import QNIndex, allowed_blocks, block_flux
    rng = np.random.default_rng(3)
    for trial in range(30):
        nq = int(rng.integers(1, 3))
        rank = int(rng.integers(1, 5))
        inds = []
        for _ in range(rank):
            ns = int(rng.integers(1, 5))
            secs = [(tuple(int(x) for x in rng.integers(-2, 3, size=nq)), int(rng.integers(1, 3))) for _ in range(ns)]
            inds.append(QNIndex(secs, int(rng.choice([-1, 1]))))
        flux = tuple(int(x) for x in rng.integers(-2, 3, size=nq))
        brute = [k for k in itertools.product(*[range(i.nsect) for i in inds])
                 if block_flux(inds, k, nq) == flux]
        assert allowed_blocks(inds, flux) == brute
