"""Failure detection without a GPU fault: every failure below is made on the
host (an allocation that a countdown fails, a start vector of zeros) or by a
bounded device wait that nothing completes; each must come back as its
status code with the context still usable."""
import numpy as np
import pytest
import torch

import helpers as H
from oracle import dmrg as D

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2007_14822_gb300 import build, tnh
    build.build()
    c = tnh.Context(0)
    yield c
    c.close()


def _heff_ok(ctx, p="bf16x6"):
    """A small H_eff product still matches the oracle (the context is usable)."""
    from paper_2007_14822_gb300 import tnh
    d = H.heff_inputs(24, None, 5, nsect=5, maxd=8)
    plan = ctx.heff_plan(d["L"], d["W"], d["W"], d["R"], d["psi"], tnh.PRECISION[p])
    y = torch.zeros_like(d["psi"].data)
    plan.apply(d["psi"].data, y)
    yt = d["psi"].with_inds(d["psi"].inds)
    yt.data = y
    want = D.heff_apply(d["Lo"], d["Wo"], d["Wo"], d["Ro"], d["psio"])
    assert H.rel_err(H.to_oracle(yt), want) < 1e-6
    plan.free()


def test_bounded_wait_gives_timeout_and_context_stays_usable(ctx):
    from paper_2007_14822_gb300.tnh import TnhError
    for limit in (2_000, 1_000_000):          # 2 us and 1 ms
        with pytest.raises(TnhError) as e:
            ctx.debug_wait_timeout(limit)
        assert e.value.code == 8 and "site 100" in str(e.value)
        # the flag was cleared: the next calls succeed and compute correctly
        ctx.sync()
        _heff_ok(ctx)
    with pytest.raises(TnhError) as e:
        ctx.debug_wait_timeout(10)           # below the allowed range
    assert e.value.code == 1


@pytest.mark.parametrize("method", ["lanczos", "davidson"])
def test_zero_or_nan_start_vector_gives_numeric_error(ctx, method):
    from paper_2007_14822_gb300 import tnh
    from paper_2007_14822_gb300.tnh import TnhError
    d = H.heff_inputs(12, None, 13, nsect=1, symmetric=True)
    plan = ctx.heff_plan(d["L"], d["W"], d["W"], d["R"], d["psi"], tnh.FP64)
    for bad in (torch.zeros_like(d["psi"].data), torch.full_like(d["psi"].data, float("nan"))):
        with pytest.raises(TnhError) as e:
            plan.eigsolve(bad, krylov_dim=16, tol=1e-10, method=method)
        assert e.value.code == 9, str(e.value)
    # the same plan still solves from a proper start vector
    Hm = D.heff_dense_matrix(d["Lo"], d["Wo"], d["Wo"], d["Ro"], d["psio"])
    w = np.linalg.eigvalsh(0.5 * (Hm + Hm.T))
    psi = d["psi"].data.clone()
    E, r, k = plan.eigsolve(psi, krylov_dim=48, tol=1e-10, method=method)
    assert abs(E - w[0]) < 1e-9 * abs(w[0])


def test_failed_allocation_gives_oom_and_leaks_nothing(ctx):
    # fail the k-th device allocation of an H_eff plan (and of a contraction)
    # for several k: each call returns TNH_ERR_OOM and the pool holds as much
    # as before the call; a call after the failures works
    from paper_2007_14822_gb300 import tnh
    from paper_2007_14822_gb300.tnh import Tensor, TnhError
    d = H.heff_inputs(24, None, 5, nsect=5, maxd=8)
    ctx.sync()
    base = ctx.debug_pool_used()
    failed = 0
    for k in (1, 2, 3, 5, 8, 13, 21):
        ctx.debug_fail_alloc(k)
        try:
            plan = ctx.heff_plan(d["L"], d["W"], d["W"], d["R"], d["psi"], tnh.BF16x6)
            plan.free()                      # k beyond the plan's allocations
        except TnhError as e:
            assert e.code == 6 and "injected failure" in str(e), str(e)
            failed += 1
        ctx.debug_fail_alloc(0)
        assert ctx.debug_pool_used() == base, k
    assert failed >= 5
    # theta = A1 A2 over the shared link c (labels: a 1, s1 2, c 3, s2 4, b 5)
    from paper_2007_14822_gb300.tnh import Index
    a, s = d["psi"].inds[0], d["psi"].inds[1]
    ia, s1, c, s2, b = (Index(a.sectors, +1, 1), Index(s.sectors, +1, 2), Index(a.sectors, +1, 3),
                        Index(s.sectors, +1, 4), Index(a.sectors, +1, 5))
    A1, _ = H.random_pair([ia, s1, c.dag()], None, 3, "A")
    A2, _ = H.random_pair([c, s2, b.dag()], None, 4, "B")
    C = Tensor([ia, s1, s2, b.dag()])
    ctx.debug_fail_alloc(1)
    with pytest.raises(TnhError) as e:
        ctx.contract(A1, A2, C)
    assert e.value.code == 6
    ctx.debug_fail_alloc(0)
    assert ctx.debug_pool_used() == base
    _heff_ok(ctx)
