"""The benchmark's algorithmic flop count against the contractions that the
oracle performs: every labelled contraction of the step (theta, the H_eff
products, the environment update) is counted as 2 M N K per block pair while
it runs on dense storage, and the total must equal ``bench.step_flops``."""
import numpy as np
import pytest

import bench
from oracle import blocksparse as B
from oracle import dmrg as D
from oracle import models as om
from oracle.blocksparse import OUT, BlockTensor, trivial_index
from test_oracle_dmrg import dense_site_mpo


@pytest.fixture
def counted(monkeypatch):
    total = [0]
    contract = B.contract

    def counting(A, Bt, out_labels=None):
        common = [l for l in A.labels if l in Bt.labels]
        ia = [A.labels.index(l) for l in common]
        ib = [Bt.labels.index(l) for l in common]
        for ka, va in A.blocks.items():
            for kb, vb in Bt.blocks.items():
                if all(ka[p] == kb[q] for p, q in zip(ia, ib)):
                    K = int(np.prod([va.shape[p] for p in ia]))
                    total[0] += 2 * (va.size // K) * (vb.size // K) * K
        return contract(A, Bt, out_labels)
    monkeypatch.setattr(D, "contract", counting)
    return total


@pytest.mark.parametrize("m", [1, 3, 6])
def test_step_flops_equal_the_counted_contractions(counted, m):
    d, w, k = bench.D, bench.W_DIM, bench.K_LANCZOS
    mpo = dense_site_mpo(om.heisenberg_mpo(4))
    W = mpo.W[1]
    assert W.shape == (w, w, d, d)
    a, s = trivial_index(m, OUT), trivial_index(d, OUT)
    rng = np.random.default_rng(m)
    A1 = BlockTensor.from_dense(rng.standard_normal((m, d, m)), [a, s, a.dag()])
    A2 = BlockTensor.from_dense(rng.standard_normal((m, d, m)), [a, s, a.dag()])
    L = BlockTensor.from_dense(rng.standard_normal((m, w, m)), [a.dag(), W.inds[0].dag(), a])
    R = BlockTensor.from_dense(rng.standard_normal((m, w, m)), [a, W.inds[1].dag(), a.dag()])
    th = D.theta(A1, A2)
    for _ in range(k + 1):            # k Lanczos products and the FP64 energy product
        D.heff_apply(L, W, W, R, th)
    D.env_left(L, A1, W)
    total, heff = bench.step_flops(m=m)
    assert counted[0] == total
    # one product alone
    counted[0] = 0
    D.heff_apply(L, W, W, R, th)
    assert counted[0] == heff


def test_bench_workload_flops():
    # dense m=256, w=5, d=2: 1.39 GFLOP per product, 13.37 GFLOP per step
    total, heff = bench.step_flops()
    assert heff == 1_394_606_080
    assert total == 13_369_868_288


@pytest.mark.parametrize("kind,m,recipe", [("heis", 24, (5, 8)), ("hub", 30, (3, 6)), ("cyl", 20, (5, 6))])
def test_chain_flops_equal_the_counted_heff_contractions(counted, kind, m, recipe):
    # the headline's flop count (block pairs of S1..S4 on block-sparse
    # storage) against the contractions of one oracle H_eff product
    L, W1, W2, R, psi = bench.qn_oracle_inputs(kind, m, recipe, 3)
    f = bench.chain_flops(L, W1, W2, R, psi)
    D.heff_apply(L, W1, W2, R, psi)
    assert counted[0] == f and f > 0


def test_kernel_traffic_is_keyed_on_code_not_comments(tmp_path, monkeypatch):
    """The stored DRAM traffic of a kernel stays valid across comment edits of
    its sources and is dropped (None) after a change to their code."""
    src = tmp_path / "paper_2007_14822_gb300" / "csrc"
    src.mkdir(parents=True)
    code = "// a kernel\nint f(int x) {\n    return x + 1;   /* one */\n}\n"
    (src / "k.cu").write_text(code)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setitem(bench.KERNEL_SOURCES, "kern", ["k.cu"])
    monkeypatch.setitem(bench.TRAFFIC, "kern_x", {"bytes_per_launch": 123.0,
                                                  "source_sha": bench.source_sha(["k.cu"])})
    assert bench.kernel_traffic("kern_x") == 123.0
    (src / "k.cu").write_text("// the kernel, reworded\n\nint f(int x) {\n    return x + 1;\n}   // end\n")
    assert bench.kernel_traffic("kern_x") == 123.0
    (src / "k.cu").write_text(code.replace("x + 1", "x + 2"))
    assert bench.kernel_traffic("kern_x") is None
