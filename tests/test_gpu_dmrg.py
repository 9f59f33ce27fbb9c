"""GPU two-site DMRG sweeps against the oracle's sweeps and exact energies."""
import numpy as np
import pytest

import helpers as H
from oracle import dmrg as D
from oracle import ed, models as om
from paper_2007_14822_gb300 import models as pm
from paper_2007_14822_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2007_14822_gb300 import build, tnh
    build.build()
    c = tnh.Context(0)
    yield c
    c.close()


def device_product_vectors(site, vecs):
    return pm.product_vectors(site, vecs)


def device_product_basis(site, states):
    return pm.product_state(site, states)


def run_both(ctx, host_mpo, oracle_mpo, qn, init, sweeps, prec="fp64", krylov=64, tol=1e-10):
    from paper_2007_14822_gb300 import tnh
    W = pm.to_device(host_mpo, qn=qn)
    site = W[0].inds[3]
    if init[0] == "vec":
        A = device_product_vectors(site, init[1])
        Ao = D.product_mps_vectors(oracle_mpo.site_index, init[1])
    else:
        A = device_product_basis(site, init[1])
        Ao = D.product_mps_basis(oracle_mpo.site_index, init[1], site.nq)
    maxd = [m for m, _ in sweeps]
    cut = [c for _, c in sweeps]
    E, stats = ctx.dmrg(W, A, host_mpo.start, host_mpo.done, maxd, cut, krylov_dim=krylov, tol=tol,
                        prec=tnh.PRECISION[prec])
    Eo, _, sto = D.dmrg(oracle_mpo, Ao, sweeps, krylov, tol)
    return E, stats, Eo, sto


def test_dmrg_heisenberg_dense(ctx):
    from test_oracle_dmrg import dense_site_mpo
    N = 10
    sweeps = [(8, 1e-12), (16, 1e-12), (32, 1e-13), (32, 1e-13)]
    E, st, Eo, sto = run_both(ctx, pm.heisenberg(N), dense_site_mpo(om.heisenberg_mpo(N)), False,
                              ("vec", synth.product_spinors(1, N, 2)), sweeps)
    e_ed = ed.ground_energy(N, 2, om.spin_pair_terms(om.heisenberg_pairs(N)))
    assert abs(E - Eo) < 1e-9 * abs(Eo)
    assert abs(E - e_ed) < 1e-9 * abs(e_ed)
    assert st[-1]["maxlink"] == sto[-1]["maxdim"]


@pytest.mark.parametrize("prec", ["fp64", "bf16x6"])
def test_dmrg_heisenberg_qn(ctx, prec):
    N = 12
    sweeps = [(8, 1e-12), (32, 1e-12), (64, 1e-13), (64, 1e-13)]
    E, st, Eo, sto = run_both(ctx, pm.heisenberg(N), om.heisenberg_mpo(N), True, ("basis", [0, 1] * (N // 2)),
                              sweeps, prec=prec, tol=1e-10 if prec == "fp64" else 1e-7)
    e_ed = ed.ground_energy(N, 2, om.spin_pair_terms(om.heisenberg_pairs(N)), om.SPIN_QN, (0,))
    assert abs(E - Eo) < 1e-9 * abs(Eo), (E, Eo)
    assert abs(E - e_ed) < 1e-9 * abs(e_ed)


def test_dmrg_hubbard_qn(ctx):
    N = 6
    sweeps = [(16, 1e-12), (64, 1e-13), (128, 1e-13)]
    E, st, Eo, sto = run_both(ctx, pm.hubbard(N, 1.0, 4.0), om.hubbard_mpo(N, 1.0, 4.0), True,
                              ("basis", [1, 2] * (N // 2)), sweeps)
    e_ed = ed.ground_energy(N, 4, om.hubbard_terms(N, 1.0, 4.0), om.HUB_QN, (N, 0))
    assert abs(E - Eo) < 1e-9 * abs(Eo)
    assert abs(E - e_ed) < 1e-9 * abs(e_ed)


def test_dmrg_majumdar_ghosh(ctx):
    N = 12
    sweeps = [(8, 1e-12), (32, 1e-12), (64, 1e-13), (64, 1e-13)]
    E, st, Eo, sto = run_both(ctx, pm.j1j2_chain(N, 1.0, 0.5),
                              om.heisenberg_like_mpo(N, om.j1j2_chain_pairs(N, 1.0, 0.5)), True,
                              ("basis", [0, 1] * (N // 2)), sweeps)
    assert abs(E + 3 * N / 8) < 1e-9 * 3 * N / 8


def test_dmrg_config1_random_product(ctx):
    # plain FP64 two-site DMRG, Heisenberg N=20, d=2, w=5, dense, m=32,
    # cutoff 1e-10, 5 sweeps, random product-state MPS from seed 1
    from test_oracle_dmrg import dense_site_mpo
    N = 20
    sweeps = [(32, 1e-10)] * 5
    E, st, Eo, sto = run_both(ctx, pm.heisenberg(N), dense_site_mpo(om.heisenberg_mpo(N)), False,
                              ("vec", synth.product_spinors(1, N, 2)), sweeps)
    e_ed = ed.ground_energy(N, 2, om.spin_pair_terms(om.heisenberg_pairs(N)), om.SPIN_QN, (0,))
    assert abs(E - Eo) < 1e-9 * abs(Eo), (E, Eo)
    assert E >= e_ed - 1e-10
    assert E - e_ed < 1e-4 * abs(e_ed)


def test_dmrg_mixed_with_tiny_cutoff_matches_fp64(ctx):
    # BF16x6 matvecs leave noise-level singular values (~1e-7 of the largest)
    # in theta; a cutoff of 1e-14 keeps them, so the factorisation must still
    # return an orthonormal exact side for them (otherwise the MPS stops being
    # canonical and the sweep diverges)
    from paper_2007_14822_gb300 import tnh
    N = 24
    mpo = pm.heisenberg(N)
    sweeps = [(16, 1e-14), (64, 1e-14), (256, 1e-14), (256, 1e-14)]
    out = {}
    for name, prec, tol in (("mix", tnh.BF16x6, 1e-7), ("fp64", tnh.FP64, 1e-10)):
        W = pm.to_device(mpo, qn=True)
        A = pm.product_state(W[0].inds[3], [0, 1] * (N // 2))
        out[name], st = ctx.dmrg(W, A, mpo.start, mpo.done, [m for m, _ in sweeps], [c for _, c in sweeps],
                                 krylov_dim=16, tol=tol, prec=prec)
    assert abs(out["mix"] - out["fp64"]) < 1e-9 * abs(out["fp64"]), out
