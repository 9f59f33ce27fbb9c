"""Host-side layout of the library's MPO and MPS tensors (no GPU): the block
tables that ``to_device``, ``splitblocks`` and the product states hand to
the C ABI, built on CPU torch tensors."""
import numpy as np
import pytest
import torch

from paper_2007_14822_gb300 import models as pm
from paper_2007_14822_gb300 import tnh


@pytest.fixture(autouse=True)
def cpu_tensors(monkeypatch):
    # the binding allocates on CUDA by default; these checks only need the
    # host layout, so allocate on the CPU
    init = tnh.Tensor.__init__

    def on_cpu(self, *a, **k):
        k["device"] = "cpu"
        init(self, *a, **k)
    monkeypatch.setattr(tnh.Tensor, "__init__", on_cpu)


def dense_of(T):
    """The full array of a block-sparse tensor from its block table."""
    dims = [i.dim for i in T.inds]
    out = np.zeros(dims)
    host = T.data.numpy()
    for key, off in zip(T.blocks, T.offsets):
        shp = T.block_shape(key)
        sl = []
        for ax, sec in enumerate(key):
            o = sum(d for _, d in T.inds[ax].sectors[:sec])
            sl.append(slice(o, o + shp[ax]))
        out[tuple(sl)] += host[off:off + int(np.prod(shp))].reshape(shp)
    return out


def flux_of(T, key):
    f = np.zeros(T.inds[0].nq, dtype=np.int64)
    for ind, sec in zip(T.inds, key):
        f += ind.arrow * np.asarray(ind.sectors[sec][0])
    return tuple(int(x) for x in f)


MODELS = [("heisenberg", lambda: pm.heisenberg(6)), ("j1j2", lambda: pm.j1j2_chain(7)),
          ("hubbard", lambda: pm.hubbard(4)), ("tfim", lambda: pm.tfim(5))]


@pytest.mark.parametrize("name,make", MODELS, ids=[m[0] for m in MODELS])
@pytest.mark.parametrize("qn", [True, False])
def test_to_device_and_splitblocks_hold_the_mpo(name, make, qn):
    host = make()      # (the Ising chain's charges are all zero: its QN layout is one sector per state)
    full = pm.to_device(host, qn=qn)
    split = pm.splitblocks(host, qn=qn)
    for j, W in enumerate(host.W):
        for T in (full[j], split[j]):
            np.testing.assert_array_equal(dense_of(T), W)
            # every stored block carries the tensor's (zero) flux
            assert all(not any(flux_of(T, k)) for k in T.blocks)
        # splitblocks stores the nonzero blocks only, one per link-state pair
        assert all(np.any(dense_of_block(split[j], k) != 0) for k in split[j].blocks)
        assert len(set(split[j].blocks)) == len(split[j].blocks)
    assert sum(T.data.numel() for T in split) <= sum(T.data.numel() for T in full)


def dense_of_block(T, key):
    off = T.offsets[T.blocks.index(key)]
    return T.data.numpy()[off:off + T.block_size(key)]


def test_to_device_refuses_weight_outside_allowed_blocks():
    host = pm.heisenberg(3)
    host.W[1] = host.W[1].copy()
    host.W[1][0, 1] = np.eye(2)          # link charge 0 -> 2 with a charge-0 operator
    with pytest.raises(ValueError):
        pm.to_device(host, qn=True)
    with pytest.raises(ValueError):
        pm.splitblocks(host, qn=True)


def test_product_state_links_carry_the_charge_to_their_left():
    site = pm.site_index(pm.HUB_QN, qn=True)
    states = [1, 2, 3, 0, 1]
    A = pm.product_state(site, states)
    q = np.zeros(2, dtype=np.int64)
    for T, st in zip(A, states):
        assert T.inds[0].sectors == [(tuple(int(x) for x in q), 1)]
        q = q + np.asarray(pm.HUB_QN[st])
        assert T.inds[2].sectors == [(tuple(int(x) for x in q), 1)] and T.inds[2].arrow == -1
        # one stored block: the chosen basis state
        assert T.blocks == [(0, st, 0)]
        np.testing.assert_array_equal(T.data.numpy()[:1], [1.0])
    assert tuple(q) == (5, 1)


def test_product_vectors_are_normalised():
    site = pm.site_index(pm.SPIN_QN, qn=False)
    vecs = [np.array([3.0, 4.0]), np.array([1.0, -1.0])]
    A = pm.product_vectors(site, vecs)
    for T, v in zip(A, vecs):
        np.testing.assert_allclose(T.data.numpy()[:2], v / np.linalg.norm(v), rtol=0, atol=1e-15)
