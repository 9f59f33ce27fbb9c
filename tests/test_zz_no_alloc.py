"""tnh_contract_dense_noalloc through the C ABI (FP64).

The allocation-free entry point serves callers that may not allocate device
memory while they run: a process that reserved its memory up front, a
latency-bound loop where cudaMalloc/cudaFree would stall the device, or a
framework that hands out memory only from its own pool. Every call reuses
one static device scratch array, so two calls in a row must each give the
result of tnh_contract and of a plain numpy product, and no call may change
the device's free memory. This file is collected last so that a run stopping
at the first failure has already run every other test.
"""
import numpy as np
import pytest

import helpers as H

pytestmark = pytest.mark.gpu

TOL = 1e-12   # the FP64 tolerance of the other parity tests


@pytest.fixture(scope="module")
def ctx():
    import torch
    from paper_2007_14822_gb300 import build, tnh
    assert torch.cuda.is_available()
    build.build()
    c = tnh.Context(0)
    yield c
    c.close()


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _inputs(dims, seed):
    from paper_2007_14822_gb300.tnh import Index, Tensor
    di, dj, dk, dl = dims
    i, j, k, l = (Index.dense(di, +1, 1), Index.dense(dj, +1, 2), Index.dense(dk, +1, 3),
                  Index.dense(dl, +1, 4))
    A, Ao = H.random_pair([i, j, k], (0,), seed, "A")
    B, Bo = H.random_pair([k.dag(), l, j.dag()], (0,), seed, "B")
    return A, B, Ao.to_dense(), Bo.to_dense(), (l, i)


def _case(ctx, dims, seed):
    """C[l, i] = sum_jk A[i, j, k] B[k, l, j]: the no-alloc result against
    tnh_contract and against numpy (float64 einsum on the host)."""
    from paper_2007_14822_gb300.tnh import FP64, Tensor
    A, B, a, b, (l, i) = _inputs(dims, seed)
    want = Tensor([l, i], (0,))
    ctx.contract(A, B, want, FP64)
    got = Tensor([l, i], (0,))
    got.data.fill_(np.nan)
    ctx.contract_dense_noalloc(A, B, got)
    ctx.sync()
    g = got.data.cpu().numpy().reshape(dims[3], dims[0])
    ref = np.einsum("ijk,klj->li", a, b)
    return _rel(g, want.data.cpu().numpy().reshape(g.shape)), _rel(g, ref)


def test_noalloc_matches_contract_on_two_calls_in_a_row(ctx):
    # first call larger than the second: the second must not see stale scratch
    for dims, seed in (((130, 37, 21, 70), 1), ((9, 5, 3, 66), 2)):
        e_contract, e_numpy = _case(ctx, dims, seed)
        assert e_contract < TOL and e_numpy < TOL, (dims, e_contract, e_numpy)


def test_noalloc_leaves_device_memory_unchanged(ctx):
    # after one warm-up call (module loading), calls of several sizes change
    # neither the device's free memory nor torch's allocation
    import torch
    from paper_2007_14822_gb300.tnh import Tensor
    cases = []
    for dims, seed in (((64, 8, 16, 32), 3), ((200, 3, 7, 150), 4), ((1, 1, 1, 1), 5)):
        A, B, a, b, (l, i) = _inputs(dims, seed)
        cases.append((A, B, Tensor([l, i], (0,)), np.einsum("ijk,klj->li", a, b)))
    ctx.contract_dense_noalloc(*cases[0][:3])
    ctx.sync()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    used0 = torch.cuda.memory_allocated()
    for _ in range(2):
        for A, B, C, ref in cases:
            ctx.contract_dense_noalloc(A, B, C)
    ctx.sync()
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0 and torch.cuda.memory_allocated() == used0, (free0, free1)
    for A, B, C, ref in cases:
        assert _rel(C.data.cpu().numpy().reshape(ref.shape), ref) < TOL


def test_noalloc_refuses_more_than_its_static_scratch(ctx):
    from paper_2007_14822_gb300.tnh import Index, Tensor, TnhError
    i, k, j = Index.dense(4096, +1, 1), Index.dense(1, +1, 2), Index.dense(4096, +1, 3)
    A, B = Tensor([i, k]), Tensor([k.dag(), j])
    Cb = Tensor([i, j])
    with pytest.raises(TnhError) as e:
        ctx.contract_dense_noalloc(A, B, Cb)
    assert e.value.code == 1 and "static maximum" in str(e.value)


def test_noalloc_refuses_repeated_labels_and_mismatched_arrows(ctx):
    # malformed inputs are refused before anything is launched: C is untouched
    import torch
    from paper_2007_14822_gb300.tnh import Index, Tensor, TnhError
    i, k = Index.dense(3, +1, 1), Index.dense(4, +1, 2)
    A = Tensor([i, i, k])            # label 1 twice
    B = Tensor([k.dag()])
    C = Tensor([i, Index.dense(3, +1, 5)])
    C.data.fill_(7.0)
    with pytest.raises(TnhError) as e:
        ctx.contract_dense_noalloc(A, B, C)
    assert e.value.code == 2 and "repeated label" in str(e.value)    # TNH_ERR_LABEL
    A2 = Tensor([i, k])
    C2 = Tensor([i.dag()])           # C's index has the other arrow than A's
    C2.data.fill_(7.0)
    with pytest.raises(TnhError) as e:
        ctx.contract_dense_noalloc(A2, B, C2)
    assert e.value.code == 5                                        # TNH_ERR_SHAPE
    ctx.sync()
    assert torch.all(C.data == 7.0) and torch.all(C2.data == 7.0)
