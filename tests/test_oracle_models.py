"""Pins of the oracle's models and exact diagonalisation against closed forms."""
import math

import numpy as np
import pytest

from oracle import ed, models
from oracle.blocksparse import block_flux


def mpo_full(mpo):
    """Contract an MPO chain into its full matrix (site 0 slowest), test side."""
    W = [w.to_dense() for w in mpo.W]                # [wl, wr, s, s']
    op = np.transpose(W[0][mpo.start], (0, 2, 1))    # [wr, out, in]
    for Wj in W[1:]:
        t = np.einsum("lab,lrcd->radbc", op, Wj)
        D = t.shape[1] * t.shape[2]
        op = t.reshape(t.shape[0], D, D)
    return op[mpo.done]


@pytest.mark.parametrize("N,E", [(2, -0.75), (3, -1.0), (4, -0.75 - math.sqrt(3) / 2)])
def test_heisenberg_small_closed_forms(N, E):
    terms = models.spin_pair_terms(models.heisenberg_pairs(N))
    assert abs(ed.ground_energy(N, 2, terms) - E) < 1e-12


def test_sector_restriction_matches_full():
    N = 8
    terms = models.spin_pair_terms(models.heisenberg_pairs(N))
    e_full = ed.ground_energy(N, 2, terms)
    e_sec = ed.ground_energy(N, 2, terms, models.SPIN_QN, (0,))
    assert abs(e_full - e_sec) < 1e-12


def tfim_closed_form(N, J, h):
    M = np.diag([h] * N) + np.diag([J] * (N - 1), 1)
    return -float(np.sum(np.linalg.svd(M, compute_uv=False)))


def test_tfim_closed_form_checks():
    assert abs(tfim_closed_form(1, 1.0, 0.7) + 0.7) < 1e-15
    assert abs(tfim_closed_form(2, 1.0, 1.0) + math.sqrt(5)) < 1e-14


@pytest.mark.parametrize("N", [2, 3, 5, 8])
@pytest.mark.parametrize("h", [0.5, 1.0, 1.7])
def test_tfim_ed_free_fermion(N, h):
    e = ed.ground_energy(N, 2, models.tfim_terms(N, 1.0, h))
    assert abs(e - tfim_closed_form(N, 1.0, h)) < 1e-11


@pytest.mark.parametrize("N", [2, 4, 6])
def test_hubbard_u0_free_fermions(N):
    t = 1.0
    want = 2 * sum(-2 * t * math.cos(math.pi * k / (N + 1)) for k in range(1, N // 2 + 1))
    e = ed.ground_energy(N, 4, models.hubbard_terms(N, t, 0.0), models.HUB_QN, (N, 0))
    assert abs(e - want) < 1e-11


@pytest.mark.parametrize("U", [1.0, 4.0, 8.0])
def test_hubbard_dimer_closed_form(U):
    t = 1.0
    want = 0.5 * (U - math.sqrt(U * U + 16 * t * t))
    e = ed.ground_energy(2, 4, models.hubbard_terms(2, t, U), models.HUB_QN, (2, 0))
    assert abs(e - want) < 1e-12


@pytest.mark.parametrize("N", [4, 6, 8, 10])
def test_majumdar_ghosh(N):
    terms = models.spin_pair_terms(models.j1j2_chain_pairs(N, 1.0, 0.5))
    assert abs(ed.ground_energy(N, 2, terms) + 3 * N / 8) < 1e-11


def _check_mpo(mpo, N, d, terms):
    H = ed.hamiltonian_dense(N, d, terms)
    np.testing.assert_allclose(mpo_full(mpo), H, atol=1e-13, rtol=0)
    for W in mpo.W:
        for key in W.blocks:
            assert block_flux(W.inds, key) == W.flux


def test_heisenberg_bulk_mpo_matches_terms():
    N = 5
    mpo = models.heisenberg_mpo(N)
    assert mpo.W[1].inds[0].dim == 5          # Sec. 7.1: exact MPO has w = 5
    _check_mpo(mpo, N, 2, models.spin_pair_terms(models.heisenberg_pairs(N)))


def test_fsa_heisenberg_mpo_matches_terms():
    N = 5
    mpo = models.heisenberg_like_mpo(N, models.heisenberg_pairs(N))
    assert mpo.max_bond() == 5
    _check_mpo(mpo, N, 2, models.spin_pair_terms(models.heisenberg_pairs(N)))


def test_tfim_mpo_matches_terms():
    N = 5
    _check_mpo(models.tfim_mpo(N, 1.0, 0.8), N, 2, models.tfim_terms(N, 1.0, 0.8))


def test_j1j2_chain_mpo_matches_terms():
    N = 6
    pairs = models.j1j2_chain_pairs(N, 1.0, 0.5)
    mpo = models.heisenberg_like_mpo(N, pairs)
    assert mpo.max_bond() == 8
    _check_mpo(mpo, N, 2, models.spin_pair_terms(pairs))


def test_cylinder_mpo_matches_terms():
    pairs = models.j1j2_cylinder_pairs(2, 3, 1.0, 0.5)
    N = 6
    _check_mpo(models.heisenberg_like_mpo(N, pairs), N, 2, models.spin_pair_terms(pairs))


def test_cylinder_bond_counts():
    Lx, Ly = 24, 6
    pairs = models.j1j2_cylinder_pairs(Lx, Ly)
    nn = sum(1 for p in pairs if p[2] == 1.0)
    nnn = sum(1 for p in pairs if p[2] == 0.5)
    assert nn == Lx * Ly + (Lx - 1) * Ly
    assert nnn == 2 * (Lx - 1) * Ly
    assert max(j - i for i, j, _ in pairs) == 2 * Ly - 1
    # snake order: consecutive sites are nearest neighbours, so the chain of
    # sites is a path through the lattice
    J = {(i, j): c for i, j, c in pairs}
    assert all(J.get((i, i + 1)) == 1.0 for i in range(Lx * Ly - 1))


def test_hubbard_mpo_matches_terms():
    N = 3
    mpo = models.hubbard_mpo(N, 1.0, 4.0)
    assert mpo.max_bond() == 6
    _check_mpo(mpo, N, 4, models.hubbard_terms(N, 1.0, 4.0))


def test_hubbard_approaches_lieb_wu():
    # Bethe-ansatz ground-state energy per site of the half-filled Hubbard
    # chain (Lieb and Wu): e(U) = -4t int_0^inf J0(w) J1(w) / (w (1 + e^(wU/2))) dw,
    # -0.57373 at U/t = 4. The slopes of the open-chain ED energies E0(N)
    # approach it from above as N grows (a loose check: the remainder
    # falls off like 1/N^2)
    from scipy import integrate, special
    t, U = 1.0, 4.0

    def f(w):
        return special.j0(w) * special.j1(w) / (w * (1.0 + math.exp(min(w * U / 2, 700.0))))
    e_lw = -4.0 * t * integrate.quad(f, 0.0, 200.0, limit=2000)[0]
    assert abs(e_lw + 0.5737293678984) < 1e-9
    E = {N: ed.ground_energy(N, 4, models.hubbard_terms(N, t, U), models.HUB_QN, (N, 0)) for N in (6, 8, 10)}
    s1, s2 = (E[8] - E[6]) / 2, (E[10] - E[8]) / 2
    assert e_lw < s2 < s1
    assert s2 - e_lw < 2e-3
