"""tnh_contract_dense_noalloc against tnh_contract (FP64), through the C ABI.

The allocation-free entry point serves callers that may not allocate device
memory while they run (memory reserved up front, latency-bound loops,
framework-owned pools). It must give the result of tnh_contract on every
call, even though every call reuses the same static device scratch. This
file is collected last so that a run stopping at the first failure has
already run every other test.
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
    a = a.cpu().numpy()
    b = b.cpu().numpy()
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _case(ctx, dims, seed):
    from paper_2007_14822_gb300.tnh import FP64, Index, Tensor
    di, dj, dk, dl = dims
    i, j, k, l = (Index.dense(di, +1, 1), Index.dense(dj, +1, 2), Index.dense(dk, +1, 3),
                  Index.dense(dl, +1, 4))
    A, _ = H.random_pair([i, j, k], (0,), seed, "A")
    B, _ = H.random_pair([k.dag(), l, j.dag()], (0,), seed, "B")
    want = Tensor([l, i], (0,))
    ctx.contract(A, B, want, FP64)
    got = Tensor([l, i], (0,))
    got.data.fill_(np.nan)
    ctx.contract_dense_noalloc(A, B, got)
    ctx.sync()
    return _rel(got.data, want.data)


def test_noalloc_matches_contract_on_two_calls_in_a_row(ctx):
    # first call larger than the second: the second must not see stale scratch
    assert _case(ctx, (130, 37, 21, 70), 1) < TOL
    assert _case(ctx, (9, 5, 3, 66), 2) < TOL


def test_noalloc_refuses_more_than_its_static_scratch(ctx):
    from paper_2007_14822_gb300.tnh import Index, Tensor, TnhError
    i, k, j = Index.dense(4096, +1, 1), Index.dense(1, +1, 2), Index.dense(4096, +1, 3)
    A, B = Tensor([i, k]), Tensor([k.dag(), j])
    Cb = Tensor([i, j])
    with pytest.raises(TnhError) as e:
        ctx.contract_dense_noalloc(A, B, Cb)
    assert e.value.code == 1 and "static maximum" in str(e.value)
