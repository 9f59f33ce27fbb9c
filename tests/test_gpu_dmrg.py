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


@pytest.mark.parametrize("N,prec", [(6, "fp64"), (6, "bf16x6"), (8, "bf16x6")])
def test_dmrg_hubbard_qn(ctx, N, prec):
    # U(1) x U(1) (N, 2Sz) Hubbard chain, U/t = 4, half filling, d = 4: the
    # sweeps in FP64 and with BF16x6 matvecs against the oracle's sweeps at the
    # same settings and exact diagonalisation (the last maxdim is the exact
    # bond dimension 4^(N/2), so the sweeps converge to the ground state)
    sweeps = [(16, 1e-12), (64, 1e-13), (4 ** (N // 2), 1e-13), (4 ** (N // 2), 1e-13)]
    E, st, Eo, sto = run_both(ctx, pm.hubbard(N, 1.0, 4.0), om.hubbard_mpo(N, 1.0, 4.0), True,
                              ("basis", [1, 2] * (N // 2)), sweeps, prec=prec,
                              tol=1e-10 if prec == "fp64" else 1e-7)
    e_ed = ed.ground_energy(N, 4, om.hubbard_terms(N, 1.0, 4.0), om.HUB_QN, (N, 0))
    assert abs(E - Eo) < 1e-9 * abs(Eo), (E, Eo)
    assert abs(E - e_ed) < 1e-9 * abs(e_ed), (E, e_ed)


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


def test_dmrg_config1_converged_vs_ed(ctx):
    # the same chain and start at maxdim 256, cutoff 1e-12: the exact ground
    # energy (sparse Lanczos over the 184 756 states of Sz=0) to 1e-9
    from test_oracle_dmrg import dense_site_mpo
    N = 20
    sweeps = [(16, 1e-12), (64, 1e-12), (256, 1e-12), (256, 1e-12)]
    E, st, Eo, sto = run_both(ctx, pm.heisenberg(N), dense_site_mpo(om.heisenberg_mpo(N)), False,
                              ("vec", synth.product_spinors(1, N, 2)), sweeps)
    e_ed = ed.ground_energy(N, 2, om.spin_pair_terms(om.heisenberg_pairs(N)), om.SPIN_QN, (0,))
    assert abs(E - Eo) < 1e-9 * abs(Eo), (E, Eo)
    assert abs(E - e_ed) < 1e-9 * abs(e_ed), (E, e_ed)
    assert E >= e_ed - 1e-12 * abs(e_ed)


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


# ------------------------------------------- sums of MPOs, excited states
@pytest.mark.parametrize("prec", ["fp64", "bf16x6"])
def test_dmrg_sum_of_mpos_j1j2(ctx, prec):
    # H = H_J1 + H_J2 given as two MPOs, against the oracle's sum of terms and
    # the Majumdar-Ghosh energy -3N/8
    from paper_2007_14822_gb300 import tnh
    N = 12
    nn = [(i, i + 1, 1.0) for i in range(N - 1)]
    nnn = [(i, i + 2, 0.5) for i in range(N - 2)]
    hosts = [pm.spin_pairs(N, nn), pm.spin_pairs(N, nnn)]
    Ws = [pm.to_device(h, qn=True) for h in hosts]
    site = Ws[0][0].inds[3]
    sweeps = [(8, 1e-12), (32, 1e-12), (64, 1e-13), (64, 1e-13)]
    A = pm.product_state(site, [0, 1] * (N // 2))
    E, st = ctx.dmrg(Ws, A, [h.start for h in hosts], [h.done for h in hosts], [m for m, _ in sweeps],
                     [c for _, c in sweeps], krylov_dim=64, tol=1e-10 if prec == "fp64" else 1e-7,
                     prec=tnh.PRECISION[prec])
    ao = D.product_mps_basis(om.heisenberg_mpo(N).site_index, [0, 1] * (N // 2), 1)
    Eo, _, _ = D.dmrg([om.heisenberg_like_mpo(N, nn), om.heisenberg_like_mpo(N, nnn)], ao, sweeps, 64, 1e-10)
    assert abs(E - Eo) < 1e-9 * abs(Eo), (E, Eo)
    assert abs(E + 3 * N / 8) < 1e-9 * 3 * N / 8


def test_dmrg_sum_of_mpos_tfim_dense(ctx):
    # dense storage: bond and field parts of the TFIM as two MPOs
    from test_oracle_models import tfim_closed_form
    N, J, h = 10, 1.0, 1.3
    hosts = [pm.tfim(N, J, 0.0), pm.tfim(N, 0.0, h)]
    Ws = [pm.to_device(x, qn=False) for x in hosts]
    vecs = synth.product_spinors(3, N, 2)
    A = pm.product_vectors(Ws[0][0].inds[3], vecs)
    sweeps = [(8, 1e-12), (24, 1e-13), (32, 1e-13)]
    E, st = ctx.dmrg(Ws, A, [x.start for x in hosts], [x.done for x in hosts], [m for m, _ in sweeps],
                     [c for _, c in sweeps], krylov_dim=64, tol=1e-10)
    terms = [om.tfim_mpo(N, J, 0.0), om.tfim_mpo(N, 0.0, h)]
    Eo, _, _ = D.dmrg(terms, D.product_mps_vectors(terms[0].site_index, vecs), sweeps, 64, 1e-10)
    assert abs(E - Eo) < 1e-9 * abs(Eo), (E, Eo)
    assert abs(E - tfim_closed_form(N, J, h)) < 1e-9 * abs(E)


@pytest.mark.parametrize("prec", ["fp64", "bf16x6"])
def test_dmrg_excited_states_tfim(ctx, prec):
    # ground state, then the two lowest states above it with the projectors
    # of the earlier ones; levels of the open TFIM in closed form
    from paper_2007_14822_gb300 import tnh
    from test_oracle_dmrg import tfim_levels
    N, J, h = 8, 1.0, 1.5
    levels = tfim_levels(N, J, h)
    host = pm.tfim(N, J, h)
    W = pm.to_device(host, qn=False)
    site = W[0].inds[3]
    sweeps = [(8, 1e-13), (32, 1e-14), (32, 1e-14), (32, 1e-14), (32, 1e-14), (32, 1e-14)]
    kw = dict(krylov_dim=64, tol=1e-10 if prec == "fp64" else 1e-7, prec=tnh.PRECISION[prec])
    states, energies = [], []
    for k in range(3):
        A = pm.product_vectors(site, synth.product_spinors(4 + k, N, 2))
        E, st = ctx.dmrg(W, A, host.start, host.done, [m for m, _ in sweeps], [c for _, c in sweeps],
                         ortho=list(states), weight=20.0, **kw)
        energies.append(E)
        states.append(ctx.dmrg_mps(site))
    for E, ex in zip(energies, levels):
        assert abs(E - ex) < 1e-9 * abs(ex), (energies, levels)
    # the oracle's overlap of the device states (read back through the ABI)
    ost = [[H.to_oracle(T) for T in s] for s in states]
    for a in range(3):
        assert abs(D.mps_overlap(ost[a], ost[a]) - 1.0) < 1e-9
        for b in range(a):
            assert abs(D.mps_overlap(ost[a], ost[b])) < 1e-6


def test_dmrg_excited_state_qn_matches_oracle(ctx):
    N = 8
    host = pm.heisenberg(N)
    W = pm.to_device(host, qn=True)
    site = W[0].inds[3]
    sweeps = [(8, 1e-13), (16, 1e-14), (16, 1e-14), (16, 1e-14), (16, 1e-14), (16, 1e-14)]
    md, co = [m for m, _ in sweeps], [c for _, c in sweeps]
    E0, _ = ctx.dmrg(W, pm.product_state(site, [0, 1] * (N // 2)), host.start, host.done, md, co, krylov_dim=64)
    psi0 = ctx.dmrg_mps(site)
    E1, _ = ctx.dmrg(W, pm.product_state(site, [1, 0] * (N // 2)), host.start, host.done, md, co, krylov_dim=64,
                     ortho=[psi0], weight=5.0)
    # the oracle's run from the device ground state
    omp = om.heisenberg_mpo(N)
    Eo1, Ao1, _ = D.dmrg(omp, D.product_mps_basis(omp.site_index, [1, 0] * (N // 2), 1), sweeps,
                         ortho=[[H.to_oracle(T) for T in psi0]], weight=5.0)
    e_ed = ed.ground_energy(N, 2, om.spin_pair_terms(om.heisenberg_pairs(N)), om.SPIN_QN, (0,), k=2)
    assert abs(E0 - e_ed[0]) < 1e-9 * abs(e_ed[0])
    assert abs(E1 - Eo1) < 1e-9 * abs(Eo1), (E1, Eo1)
    assert abs(E1 - e_ed[1]) < 1e-9 * abs(e_ed[1])


def test_dmrg_checkpoint_resume(ctx):
    # two sweeps, read the MPS back, two more sweeps from it: the same
    # energies as four sweeps in one run (same inputs, deterministic kernels)
    N = 16
    host = pm.heisenberg(N)
    W = pm.to_device(host, qn=True)
    site = W[0].inds[3]
    sweeps = [(8, 1e-12), (16, 1e-12), (32, 1e-12), (48, 1e-12)]
    md, co = [m for m, _ in sweeps], [c for _, c in sweeps]
    start = pm.product_state(site, [0, 1] * (N // 2))
    E4, st4 = ctx.dmrg(W, start, host.start, host.done, md, co, krylov_dim=32)
    E2, st2 = ctx.dmrg(W, pm.product_state(site, [0, 1] * (N // 2)), host.start, host.done, md[:2], co[:2],
                       krylov_dim=32)
    ck = ctx.dmrg_mps(site)
    # the checkpoint is the state of sweep 2
    assert abs(E2 - st4[1]["energy"]) < 1e-12 * abs(E2)
    ck_host = [T.block_arrays() for T in ck]
    Er, str_ = ctx.dmrg(W, ck, host.start, host.done, md[2:], co[2:], krylov_dim=32)
    assert abs(Er - E4) < 1e-12 * abs(E4), (Er, E4)
    assert [s["maxlink"] for s in str_] == [s["maxlink"] for s in st4[2:]]
    # the checkpoint tensors were read, not modified
    for T, h in zip(ck, ck_host):
        for k, v in T.block_arrays().items():
            np.testing.assert_array_equal(v, h[k])


@pytest.mark.parametrize("prec", ["fp64", "bf16x6"])
def test_dmrg_davidson_heisenberg_qn(ctx, prec):
    # the sweeps with the Davidson eigensolver reach the oracle's / ED energy
    from paper_2007_14822_gb300 import tnh
    N = 12
    host = pm.heisenberg(N)
    W = pm.to_device(host, qn=True)
    A = pm.product_state(W[0].inds[3], [0, 1] * (N // 2))
    sweeps = [(8, 1e-12), (32, 1e-12), (64, 1e-13), (64, 1e-13)]
    E, st = ctx.dmrg(W, A, host.start, host.done, [m for m, _ in sweeps], [c for _, c in sweeps], krylov_dim=32,
                     tol=1e-10 if prec == "fp64" else 1e-7, prec=tnh.PRECISION[prec], eigensolver="davidson")
    e_ed = ed.ground_energy(N, 2, om.spin_pair_terms(om.heisenberg_pairs(N)), om.SPIN_QN, (0,))
    assert abs(E - e_ed) < 1e-9 * abs(e_ed), (E, e_ed)


@pytest.mark.parametrize("qn", [False, True])
def test_dmrg_splitblocks_mpo(ctx, qn):
    # the sparse (split) MPO stores only nonzero blocks and gives the same sweeps
    N = 10
    host = pm.heisenberg(N)
    Ws = pm.splitblocks(host, qn=qn)
    Wd = pm.to_device(host, qn=qn)
    assert sum(int(w.data.numel()) for w in Ws) < sum(int(w.data.numel()) for w in Wd)
    site = Ws[0].inds[3]
    sweeps = [(8, 1e-12), (16, 1e-12), (32, 1e-13), (32, 1e-13)]
    if qn:
        mk = lambda: pm.product_state(site, [0, 1] * (N // 2))
    else:
        vecs = synth.product_spinors(1, N, 2)
        mk = lambda: pm.product_vectors(site, vecs)
    md, co = [m for m, _ in sweeps], [c for _, c in sweeps]
    Es, _ = ctx.dmrg(Ws, mk(), host.start, host.done, md, co, krylov_dim=64)
    Ed, _ = ctx.dmrg(Wd, mk(), host.start, host.done, md, co, krylov_dim=64)
    e_ed = ed.ground_energy(N, 2, om.spin_pair_terms(om.heisenberg_pairs(N)))
    assert abs(Es - Ed) < 1e-12 * abs(Ed), (Es, Ed)
    assert abs(Es - e_ed) < 1e-9 * abs(e_ed)


@pytest.mark.parametrize("stop,every", [(37, 1), (30, 0), (52, 7)])
def test_dmrg_checkpoint_file_resume_inside_a_sweep(ctx, tmp_path, stop, every):
    # a run that stops after `stop` bond updates (inside sweep 1, at the end of
    # sweep 0, or inside the right-to-left pass of sweep 1), having written its
    # checkpoint file, is resumed by a new context from that file: the energies
    # of every sweep equal those of the uninterrupted run (FP64, deterministic
    # kernels), the stopped run reports where it stopped, and the file holds
    # the MPS, the environments and the position
    from paper_2007_14822_gb300 import tnh
    N = 16
    host = pm.heisenberg(N)
    W = pm.to_device(host, qn=True)
    site = W[0].inds[3]
    sweeps = [(8, 1e-12), (16, 1e-12), (32, 1e-12), (48, 1e-12)]
    md, co = [m for m, _ in sweeps], [c for _, c in sweeps]
    mk = lambda: pm.product_state(site, [0, 1] * (N // 2))
    E4, st4 = ctx.dmrg(W, mk(), host.start, host.done, md, co, krylov_dim=32)
    path = tmp_path / "run.ckpt"
    c1 = tnh.Context(0)
    c1.dmrg_checkpoint(path, every=every, stop_after=stop)
    c1.dmrg(W, mk(), host.start, host.done, md, co, krylov_dim=32)
    sw, pas, step, fin = c1.dmrg_position()
    bonds_per_sweep = 2 * (N - 1)
    assert not fin and sw == stop // bonds_per_sweep
    rest = stop % bonds_per_sweep
    assert (pas, step) == ((0, rest) if rest < N - 1 else (1, rest - (N - 1)))
    assert path.exists() and path.read_bytes()[:8] == b"TNHCKPT1"
    c1.close()
    c2 = tnh.Context(0)
    Er, str_ = c2.dmrg(W, None, host.start, host.done, md, co, krylov_dim=32, resume=path)
    assert c2.dmrg_position()[3]
    assert abs(Er - E4) < 1e-12 * abs(E4), (Er, E4)
    for a, b in zip(str_, st4):
        assert abs(a["energy"] - b["energy"]) < 1e-12 * abs(b["energy"]), (a, b)
        assert a["maxlink"] == b["maxlink"]
    c2.close()


def test_dmrg_checkpoint_refuses_a_mismatched_problem(ctx, tmp_path):
    from paper_2007_14822_gb300 import tnh
    from paper_2007_14822_gb300.tnh import TnhError
    N = 8
    host = pm.heisenberg(N)
    W = pm.to_device(host, qn=True)
    site = W[0].inds[3]
    path = tmp_path / "a.ckpt"
    c1 = tnh.Context(0)
    c1.dmrg_checkpoint(path, every=3, stop_after=5)
    c1.dmrg(W, pm.product_state(site, [0, 1] * (N // 2)), host.start, host.done, [8, 8], [1e-12] * 2)
    c1.close()
    other = pm.to_device(pm.j1j2_chain(N, 1.0, 0.5), qn=True)    # another MPO link space
    with pytest.raises(TnhError) as e:
        ctx.dmrg(other, None, host.start, host.done, [8, 8], [1e-12] * 2, resume=path)
    assert e.value.code == 5
    bad = tmp_path / "junk.ckpt"
    bad.write_bytes(b"not a checkpoint at all")
    with pytest.raises(TnhError) as e:
        ctx.dmrg(W, None, host.start, host.done, [8, 8], [1e-12] * 2, resume=bad)
    assert e.value.code == 1


@pytest.mark.parametrize("model", ["heisenberg", "hubbard"])
def test_dmrg_split_environments_with_fp64_final_energy(ctx, model):
    # BF16x6 matvecs and BF16x6 environment updates, the FP64 energy product
    # only at each sweep's last bond (energy_mode 1) and the final energy
    # evaluated with FP64 environments rebuilt from the final MPS: the same
    # energy as plain FP64 sweeps and exact diagonalisation to 1e-9; in FP64,
    # energy_mode 1 returns the energy of energy_mode 0
    from paper_2007_14822_gb300 import tnh
    if model == "heisenberg":
        N, d, host = 12, 2, pm.heisenberg(12)
        states = [0, 1] * (N // 2)
        sweeps = [(8, 1e-12), (32, 1e-12), (64, 1e-13), (64, 1e-13)]
        e_ed = ed.ground_energy(N, 2, om.spin_pair_terms(om.heisenberg_pairs(N)), om.SPIN_QN, (0,))
    else:
        N, d, host = 6, 4, pm.hubbard(6, 1.0, 4.0)
        states = [1, 2] * (N // 2)
        sweeps = [(16, 1e-12), (64, 1e-13), (64, 1e-13), (64, 1e-13)]
        e_ed = ed.ground_energy(N, 4, om.hubbard_terms(N, 1.0, 4.0), om.HUB_QN, (N, 0))
    W = pm.to_device(host, qn=True)
    site = W[0].inds[3]
    md, co = [m for m, _ in sweeps], [c for _, c in sweeps]
    run = lambda **kw: ctx.dmrg(W, pm.product_state(site, states), host.start, host.done, md, co,
                                krylov_dim=64, **kw)
    E0, st0 = run(tol=1e-10)
    E1, st1 = run(tol=1e-10, energy_mode=1)
    assert abs(E1 - E0) < 1e-13 * abs(E0), (E0, E1)
    assert [s["maxlink"] for s in st1] == [s["maxlink"] for s in st0]
    E2, st2 = run(tol=1e-7, prec=tnh.BF16x6, env_prec=tnh.BF16x6, energy_mode=1)
    assert abs(E2 - E0) < 1e-9 * abs(E0), (E2, E0)
    assert abs(E2 - e_ed) < 1e-9 * abs(e_ed), (E2, e_ed)
    assert st2[-1]["energy"] == E2
