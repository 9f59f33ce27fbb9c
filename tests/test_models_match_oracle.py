"""The library's MPO builders against the oracle's (host arrays, no GPU)."""
import numpy as np
import pytest

from oracle import models as om
from paper_2007_14822_gb300 import models as pm


def _cmp(pmpo, ompo):
    assert pmpo.N == ompo.N
    assert pmpo.start == ompo.start and pmpo.done == ompo.done
    for j in range(pmpo.N):
        np.testing.assert_array_equal(pmpo.W[j], ompo.W[j].to_dense())
        ql = [q for q, _ in ompo.W[j].inds[0].sectors]
        qr = [q for q, _ in ompo.W[j].inds[1].sectors]
        if len(ompo.W[j].inds[0].sectors) == pmpo.W[j].shape[0]:
            assert ql == list(pmpo.link_qn[j]) and qr == list(pmpo.link_qn[j + 1])


def test_heisenberg_bulk():
    _cmp(pm.heisenberg(6), om.heisenberg_mpo(6))


def test_j1j2_chain():
    pairs = om.j1j2_chain_pairs(9, 1.0, 0.5)
    _cmp(pm.j1j2_chain(9, 1.0, 0.5), om.heisenberg_like_mpo(9, pairs))


def test_cylinder():
    assert pm.cylinder_pairs(4, 6) == om.j1j2_cylinder_pairs(4, 6)
    pairs = om.j1j2_cylinder_pairs(3, 4)
    _cmp(pm.spin_pairs(12, pm.cylinder_pairs(3, 4)), om.heisenberg_like_mpo(12, pairs))


def test_hubbard():
    _cmp(pm.hubbard(5, 1.0, 4.0), om.hubbard_mpo(5, 1.0, 4.0))


def test_cylinder_bond_dim_24x6():
    assert pm.spin_pairs(144, pm.cylinder_pairs(24, 6)).max_bond() == 26
