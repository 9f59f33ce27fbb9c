"""Dense matrix products through tnh_contract: the FP64 SIMT GEMM and the
tcgen05 split-bf16 GEMM against numpy float64, over ragged shapes."""
import numpy as np
import pytest

import helpers as H

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2007_14822_gb300 import build, tnh
    build.build()
    c = tnh.Context(0)
    yield c
    c.close()


def _mm(ctx, M, K, N, p, seed=0):
    from paper_2007_14822_gb300.tnh import Index, Tensor, PRECISION
    i, k, j = Index.dense(M, +1, 1), Index.dense(K, +1, 2), Index.dense(N, +1, 3)
    A, Ao = H.random_pair([i, k], (0,), seed, "A")
    B, Bo = H.random_pair([k.dag(), j], (0,), seed, "B")
    Cm = Tensor([i, j], (0,))
    ctx.contract(A, B, Cm, PRECISION[p])
    got = Cm.data.cpu().numpy()[:M * N].reshape(M, N)
    want = Ao.to_dense() @ Bo.to_dense()
    return np.linalg.norm(got - want) / np.linalg.norm(want)


@pytest.mark.parametrize("M,K,N", [(1, 1, 1), (128, 64, 128), (130, 70, 129), (300, 1000, 257), (64, 4096, 64)])
def test_fp64(ctx, M, K, N):
    assert _mm(ctx, M, K, N, "fp64") < 1e-14


@pytest.mark.parametrize("M,K,N", [(1, 1, 1), (128, 64, 128), (130, 70, 129), (300, 1000, 257), (64, 4096, 64)])
def test_bf16x6(ctx, M, K, N):
    assert _mm(ctx, M, K, N, "bf16x6") < 1e-6


def test_split_precision_error_vs_k(ctx):
    errs = {}
    for K in (64, 256, 1024, 4096, 16384):
        errs[K] = {p: _mm(ctx, 128, K, 128, p) for p in ("bf16", "bf16x3", "bf16x6")}
    print("split-precision relative error by K:", errs)
    for K, e in errs.items():
        assert e["bf16x6"] < 1e-6 and e["bf16x3"] < 1e-4 and e["bf16"] < 1e-2
