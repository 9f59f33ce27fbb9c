"""Test-side glue: build matching device tensors and oracle tensors from the
same seeded generator, and compare them."""
import numpy as np

from oracle.blocksparse import BlockTensor, QNIndex
from paper_2007_14822_gb300 import synth


def or_index(pi):
    return QNIndex(pi.sectors, pi.arrow)


def py_index(oi, label=0):
    from paper_2007_14822_gb300.tnh import Index
    return Index(oi.sectors, oi.arrow, label)


def random_pair(inds, flux, seed, tag):
    """Device tnh.Tensor and oracle BlockTensor with identical seeded blocks."""
    from paper_2007_14822_gb300.tnh import Tensor
    T = Tensor(inds, flux)
    fn = lambda k, s: synth.block_gaussian(seed, tag, k, s)
    T.fill(fn)
    O = BlockTensor.from_blocks_fn([or_index(i) for i in inds], flux, fn)
    assert sorted(T.blocks) == sorted(O.blocks), "library and oracle disagree on the allowed blocks"
    return T, O


def to_oracle(T):
    return BlockTensor([or_index(i) for i in T.inds], T.flux, T.block_arrays())


def rel_err(got, want):
    """|got - want| / |want| over all blocks (norm-wise, float64)."""
    num = den = 0.0
    for k, w in want.blocks.items():
        g = got.blocks.get(k, np.zeros_like(w))
        num += float(np.sum((g - w) ** 2))
        den += float(np.sum(w * w))
    for k, g in got.blocks.items():
        if k not in want.blocks:
            num += float(np.sum(g * g))
    return np.sqrt(num) / max(np.sqrt(den), 1e-300)


def link_index(m, nsect, maxd, arrow, step=2):
    """QN link with a Gaussian sector profile, charges ... -2, 0, 2 ... (2Sz)."""
    from paper_2007_14822_gb300.tnh import Index
    if nsect == 1:
        return Index([((0,), m)], arrow)
    dims = synth.gaussian_sectors(m, nsect, maxd)
    qs = [step * (k - (nsect - 1) // 2) for k in range(nsect)]
    return Index([((q,), d) for q, d in zip(qs, dims)], arrow)


def heff_inputs(m, w_qn, seed, nsect=1, maxd=None, symmetric=False):
    """L, R, psi (device + oracle) around the Heisenberg bulk MPO.

    ``nsect == 1`` gives dense storage (one trivial sector per index).
    With ``symmetric`` the environments have the symmetry of environments
    built from a real MPS (channel S+ is the transpose of channel S-, the
    others symmetric), which makes H_eff symmetric.
    """
    from paper_2007_14822_gb300 import models as pm
    from paper_2007_14822_gb300.tnh import Index, Tensor
    from oracle import models as om
    qn = nsect > 1
    a = link_index(m, nsect, maxd or m, +1)
    mpo_p = pm.to_device(pm.heisenberg(3), qn=qn)
    W = mpo_p[1]
    wl, wr, sd, s = W.inds
    Lin = [a.dag(), wl.dag(), a]
    Rin = [a, wr.dag(), a.dag()]
    psin = [a, s, s, a.dag()]
    L, Lo = random_pair(Lin, None, seed, "L")
    R, Ro = random_pair(Rin, None, seed, "R")
    if symmetric:
        for T, To in ((L, Lo), (R, Ro)):
            dense = To.to_dense()                       # [a, w, a']
            sym = dense.copy()
            for ch in (0, 3, 4):
                sym[:, ch, :] = 0.5 * (dense[:, ch, :] + dense[:, ch, :].T)
            sym[:, 2, :] = dense[:, 1, :].T
            sym = BlockTensor.from_dense(sym, To.inds, To.flux, atol=np.inf)
            # the symmetrised tensor keeps only allowed blocks
            To.blocks = sym.blocks
            T.fill(lambda k, shp, To=To: To.blocks[k])
    psi, psio = random_pair(psin, None, seed, "psi")
    om_W = om.heisenberg_mpo(3).W[1]
    if not qn:
        from test_oracle_dmrg import dense_site_mpo
        om_W = dense_site_mpo(om.heisenberg_mpo(3)).W[1]
    return dict(L=L, R=R, W=W, psi=psi, Lo=Lo, Ro=Ro, Wo=om_W, psio=psio)


# -------------------------------------------------------- per-block parity
# Element-wise bound: |got - want| <= ELEM_TOL * scale, where scale is the
# same contraction evaluated by the oracle on the absolute values of every
# input (the sum of |terms| that bounds the rounding error of each output
# element). A missed or misplaced K piece, a wrong block or a block written
# twice changes an element by a sizeable fraction of that sum and fails it.
ELEM_TOL = {"fp64": 1e-12, "bf16x6": 2e-5}
# per-block relative error (norm of the block's error over the block's norm)
BLOCK_TOL = {"fp64": 1e-11, "bf16x6": 1e-5}


def abs_tensor(T):
    """Oracle BlockTensor with every element replaced by its absolute value."""
    return BlockTensor(T.inds, T.flux, {k: np.abs(v) for k, v in T.blocks.items()})


def block_report(got, want, scale):
    """Worst per-block relative error and worst element error over its scale.

    Blocks of ``got`` that ``want`` does not hold must be zero. A block whose
    norm is below 1e-2 of its scale's norm (cancellation: a one-element block
    whose sum happens to be small) is measured against that floor instead of
    its own norm.
    """
    worst_blk, worst_el, where_blk, where_el = 0.0, 0.0, None, None
    keys = set(want.blocks) | set(got.blocks)
    for k in keys:
        w = want.blocks.get(k)
        g = got.blocks.get(k)
        s = scale.blocks.get(k)
        if w is None:
            w = np.zeros_like(g)
        if g is None:
            g = np.zeros_like(w)
        if s is None:
            s = np.zeros_like(w)
        d = np.abs(g - w)
        if d.size == 0:
            continue
        nw, ns = float(np.linalg.norm(w)), float(np.linalg.norm(s))
        den = max(nw, 1e-2 * ns, 1e-300)
        rb = float(np.linalg.norm(d)) / den
        if rb > worst_blk:
            worst_blk, where_blk = rb, k
        re = float(np.max(d / np.maximum(s, 1e-300)))
        if re > worst_el:
            worst_el, where_el = re, k
    return dict(block=worst_blk, block_key=where_blk, elem=worst_el, elem_key=where_el)


def assert_parity(got, want, scale, p, norm_tol):
    """Norm-wise error below ``norm_tol``, every block below BLOCK_TOL[p],
    every element below ELEM_TOL[p] of its absolute-value scale."""
    err = rel_err(got, want)
    rep = block_report(got, want, scale)
    assert err < norm_tol, ("norm-wise", err, rep)
    assert rep["block"] < BLOCK_TOL[p], ("per block", rep)
    assert rep["elem"] < ELEM_TOL[p], ("per element", rep)
    return err, rep
