"""Planted mistakes in the oracle, on the CPU: each one must fail a pin.

Every case edits one line of an oracle module's source: a wrong coefficient,
sign or index, a transposed operand, a dropped sum or a wrong boundary rule.
The edited module is loaded beside the original, every binding of the
original's functions, classes and arrays (in the oracle and in the pin
modules) is pointed at the edited ones for the duration of the case, and the
pin that should catch the mistake is run. Nothing is changed on disk.

Edits that leave every result the same are not listed, because no pin can
see them:
- the three-term Lanczos coefficients: the full reorthogonalisation, applied
  twice, removes the same components again;
- dropping S from the next site in a left-to-right step: only the Lanczos
  start vector of the next bond changes, and the MPS stays canonical;
- the sign of J or h in the transverse-field Ising chain: the spectrum is
  unchanged under a spin flip on every other site (J) or on every site (h);
- the order of the Kronecker factors when ED sums the charges of a basis
  state: a total charge does not depend on the order of its terms;
- Lanczos without the reorthogonalisation: in exact arithmetic the
  three-term recurrence already gives an orthogonal basis, and at the sizes
  of the pins the lowest Ritz pair still converges; the reorthogonalisation
  is a safeguard against lost orthogonality, which the outputs do not show.
"""
import importlib
import inspect
import math
import sys
import types

import numpy as np
import pytest

import test_oracle_blocksparse as TB
import test_oracle_dmrg as TD
import test_oracle_models as TM

# (case id, oracle module, original line(s), planted line(s), pin, pin args)
CASES = [
    ("spin operators as Pauli matrices", "oracle.models",
     "SZ = np.array([[0.5, 0.0], [0.0, -0.5]])", "SZ = np.array([[1.0, 0.0], [0.0, -1.0]])",
     TM.test_heisenberg_small_closed_forms, (4, -0.75 - math.sqrt(3) / 2)),
    ("bulk MPO: S-S+ coefficient", "oracle.models",
     "    W[4, 1] = (0.5 * SM).T", "    W[4, 1] = (1.0 * SM).T",
     TM.test_heisenberg_bulk_mpo_matches_terms, ()),
    ("bulk MPO: SzSz sign", "oracle.models",
     "    W[4, 3] = SZ.T", "    W[4, 3] = -SZ.T",
     TM.test_heisenberg_bulk_mpo_matches_terms, ()),
    ("exchange terms: S+S- without its conjugate's coefficient", "oracle.models",
     "        terms.append((0.5 * J, [(i, SP), (j, SM)]))", "        terms.append((1.0 * J, [(i, SP), (j, SM)]))",
     TM.test_heisenberg_small_closed_forms, (4, -0.75 - math.sqrt(3) / 2)),
    ("Hubbard hopping: conjugate with the wrong sign", "oracle.models",
     "            terms.append((t, [(i, c @ F_SITE), (i + 1, cd)]))",
     "            terms.append((-t, [(i, c @ F_SITE), (i + 1, cd)]))",
     TM.test_hubbard_u0_free_fermions, (4,)),
    ("Hubbard: Jordan-Wigner parity dropped", "oracle.models",
     "F_SITE = np.diag([1.0, -1.0, -1.0, 1.0])", "F_SITE = np.diag([1.0, 1.0, 1.0, 1.0])",
     TM.test_hubbard_u0_free_fermions, (4,)),
    ("Hubbard: interaction on one spin species", "oracle.models",
     "    terms += [(U, [(i, N_UP @ N_DN)]) for i in range(N)]", "    terms += [(U, [(i, N_UP)]) for i in range(N)]",
     TM.test_hubbard_dimer_closed_form, (4.0,)),
    ("J1-J2 chain: next-nearest bonds dropped", "oracle.models",
     "           [(i, i + 2, J2) for i in range(N - 2)]", "           [(i, i + 2, J2) for i in range(0)]",
     TM.test_majumdar_ghosh, (6,)),
    ("H_eff: R transposed", "oracle.dmrg",
     '    R = R.relabel(["b", "w2", "bp"])\n    psi', '    R = R.relabel(["bp", "w2", "b"])\n    psi',
     TD.test_heff_equals_projected_hamiltonian, ("heis",)),
    ("H_eff: W1 applied transposed", "oracle.dmrg",
     '    W1 = W1.relabel(["w", "w1", "s1", "s1p"])', '    W1 = W1.relabel(["w", "w1", "s1p", "s1"])',
     TD.test_heff_equals_projected_hamiltonian, ("heis",)),
    ("H_eff: L transposed", "oracle.dmrg",
     '    L = L.relabel(["a", "w", "ap"])\n    W1', '    L = L.relabel(["ap", "w", "a"])\n    W1',
     TD.test_heff_equals_projected_hamiltonian, ("heis",)),
    ("left environment: W transposed", "oracle.dmrg",
     '    Wt = W.relabel(["w", "w1", "s", "sp"])\n    Ab = dag(A).relabel(["ap", "sp", "bp"])\n    X = contract(L, Ak)',
     '    Wt = W.relabel(["w", "w1", "sp", "s"])\n    Ab = dag(A).relabel(["ap", "sp", "bp"])\n    X = contract(L, Ak)',
     TD.test_heff_hermitian_and_matches_chain_energy, ()),
    ("Lanczos: Ritz vector with a wrong sign", "oracle.dmrg",
     "    x = scale(q[0], s[0])", "    x = scale(q[0], -s[0])",
     TD.test_lanczos_matches_eigh, ()),
    ("truncation: strict cutoff boundary", "oracle.dmrg",
     "        if tail[k - 1] <= cutoff:", "        if tail[k - 1] < cutoff:",
     TD.test_truncation_count_rule, ()),
    ("truncation: absolute instead of relative error", "oracle.dmrg",
     "    tail = np.concatenate([np.cumsum(s2[::-1])[::-1], [0.0]]) / total",
     "    tail = np.concatenate([np.cumsum(s2[::-1])[::-1], [0.0]])",
     TD.test_truncation_count_rule, ()),
    ("truncation: maxdim ignored", "oracle.dmrg",
     "    keep = min(keep, maxdim, n)", "    keep = min(keep, n)",
     TD.test_truncation_count_rule, ()),
    ("SVD: V rows out of order", "oracle.dmrg",
     "            Vt_.blocks[(ci,) + ck] = Vt[idx, coff[ck]:coff[ck] + cc].reshape((len(idx),) + shp)",
     "            Vt_.blocks[(ci,) + ck] = Vt[idx[::-1], coff[ck]:coff[ck] + cc].reshape((len(idx),) + shp)",
     TD.test_svd_trunc_eckart_young_and_predicted_count, ()),
    ("flux rule: arrows ignored", "oracle.blocksparse",
     "        f = qn_add(f, qn_scale(ind.arrow, ind.qn(s)))", "        f = qn_add(f, ind.qn(s))",
     TB.test_allowed_blocks_equals_filtered_full_product, ()),
    ("contraction: block pairs overwrite instead of sum", "oracle.blocksparse",
     "            C.blocks[kc] = C.blocks[kc] + prod", "            C.blocks[kc] = prod",
     TB.test_blocksparse_contract_equals_dense, ()),
    ("allowed blocks: arrow of the last index ignored", "oracle.blocksparse",
     "        need = qn_scale(last.arrow, qn_sub(flux, f))", "        need = qn_sub(flux, f)",
     TB.test_allowed_blocks_equals_filtered_full_product, ()),
    ("finite-state MPO: pass-through identity dropped", "oracle.models",
     "                put(st, st, np.eye(d))", "                pass",
     TM.test_j1j2_chain_mpo_matches_terms, ()),
    ("finite-state MPO: on-site term doubled", "oracle.models",
     '            put("start", "done", onsite[j])', '            put("start", "done", 2 * onsite[j])',
     TM.test_hubbard_mpo_matches_terms, ()),
    ("finite-state MPO: link charge with the wrong sign", "oracle.models",
     "        return tuple(-x for x in op_charge(first_op[st], site_qn))",
     "        return tuple(x for x in op_charge(first_op[st], site_qn))",
     TM.test_fsa_heisenberg_mpo_matches_terms, ()),
    ("Ising MPO: XX bond as XZ", "oracle.models",
     "        bulk[2, 1] = (-J * PX).T", "        bulk[2, 1] = (-J * PZ).T",
     TM.test_tfim_mpo_matches_terms, ()),
    ("Hubbard: down creator built from the up mode", "oracle.models",
     "CD_UP, CD_DN = C_UP.T.copy(), C_DN.T.copy()", "CD_UP, CD_DN = C_UP.T.copy(), C_UP.T.copy()",
     TM.test_hubbard_u0_free_fermions, (4,)),
    ("cylinder: column order instead of snake order", "oracle.models",
     "    return x * Ly + (y if x % 2 == 0 else Ly - 1 - y)", "    return x * Ly + y",
     TM.test_cylinder_bond_counts, ()),
    ("cylinder: one diagonal of J2 dropped", "oracle.models",
     "                add(s, snake_site(x + 1, (y - 1) % Ly, Ly), J2)", "                pass",
     TM.test_cylinder_bond_counts, ()),
    ("H_eff: W2 applied transposed", "oracle.dmrg",
     '    W2 = W2.relabel(["w1", "w2", "s2", "s2p"])', '    W2 = W2.relabel(["w1", "w2", "s2p", "s2"])',
     TD.test_heff_equals_projected_hamiltonian, ("heis",)),
    ("right environment: W transposed", "oracle.dmrg",
     '    Wt = W.relabel(["w", "w1", "s", "sp"])\n    Ab = dag(A).relabel(["ap", "sp", "bp"])\n    X = contract(Ak, R)',
     '    Wt = W.relabel(["w", "w1", "sp", "s"])\n    Ab = dag(A).relabel(["ap", "sp", "bp"])\n    X = contract(Ak, R)',
     TD.test_heff_hermitian_and_matches_chain_energy, ()),
    ("overlap: output indices swapped", "oracle.dmrg",
     '    return contract(contract(LO, Pb), Ak, out_labels=["pb", "b"])',
     '    return contract(contract(LO, Pb), Ak, out_labels=["b", "pb"])',
     TD.test_mps_overlap_and_projected_state_match_full_vectors, ()),
    ("SVD: pooled values ranked ascending", "oracle.dmrg",
     "    pool.sort()", "    pool.sort(reverse=True)",
     TD.test_svd_trunc_eckart_young_and_predicted_count, ()),
    ("singular values divided out instead of multiplied in", "oracle.dmrg",
     "        out.blocks[key] = v * sv.reshape(shp)", "        out.blocks[key] = v / sv.reshape(shp)",
     TD.test_svd_trunc_eckart_young_and_predicted_count, ()),
    ("energy without the norm of the vector", "oracle.dmrg",
     "    E = y.vdot(x) / nx2", "    E = y.vdot(x)",
     TD.test_energy_residual_rayleigh_quotient, ()),
    ("chain expectation without the norm of the MPS", "oracle.dmrg",
     "    return num / n2", "    return num",
     TD.test_heff_hermitian_and_matches_chain_energy, ()),
    ("left boundary selects the start state twice over", "oracle.dmrg",
     "            T.blocks[key][0, pos, 0] = 1.0\n    return T\n\n\ndef right_boundary",
     "            T.blocks[key][0, pos, 0] = 2.0\n    return T\n\n\ndef right_boundary",
     TD.test_heff_equals_projected_hamiltonian, ("heis",)),
    ("right overlap: output indices swapped", "oracle.dmrg",
     '    return contract(contract(Pb, RO), Ak, out_labels=["pa", "a"])',
     '    return contract(contract(Pb, RO), Ak, out_labels=["a", "pa"])',
     TD.test_mps_overlap_and_projected_state_match_full_vectors, ()),
    ("projected state: second site taken from the first", "oracle.dmrg",
     '    t = contract(t, dag(P2).relabel(["pc", "s2", "pb"]))',
     '    t = contract(t, dag(P1).relabel(["pc", "s2", "pb"]))',
     TD.test_mps_overlap_and_projected_state_match_full_vectors, ()),
    ("product state: link charges subtracted", "oracle.dmrg",
     "        q = qn_add(q, qs)", "        q = qn_add(q, tuple(-x for x in qs))",
     TD.test_dmrg_hubbard_vs_ed, ()),
    ("theta: second tensor joined at its right link", "oracle.dmrg",
     '    A2 = A2.relabel(["c", "s2", "b"])', '    A2 = A2.relabel(["b", "s2", "c"])',
     TD.test_dmrg_heisenberg_dense_vs_ed, ()),
    ("sweep: right-to-left step drops S from the new centre", "oracle.dmrg",
     "                A[j] = scale_link(U, S, 2)", "                A[j] = U",
     TD.test_dmrg_excited_states_tfim, ()),
    ("sweep: every sweep truncated to the first sweep's maxdim", "oracle.dmrg",
     "            U, S, V, err = svd_trunc(th, 2, cutoff, maxdim, mindim)",
     "            U, S, V, err = svd_trunc(th, 2, cutoff, sweeps[0][0], mindim)",
     TD.test_dmrg_heisenberg_dense_vs_ed, ()),
    ("residual: E x added instead of subtracted", "oracle.dmrg",
     "    r = y.axpy(-E, x).norm()", "    r = y.axpy(E, x).norm()",
     TD.test_energy_residual_rayleigh_quotient, ()),
    ("ED: highest eigenvalue returned", "oracle.ed",
     "        w = np.linalg.eigh(H.toarray())[0]\n        return w[:k] if k > 1 else float(w[0])",
     "        w = np.linalg.eigh(H.toarray())[0]\n        return w[:k] if k > 1 else float(w[-1])",
     TM.test_heisenberg_small_closed_forms, (4, -0.75 - math.sqrt(3) / 2)),
    ("ED: sector test on any one charge component", "oracle.ed",
     "np.all(ch == np.asarray(sector)[None, :], axis=1)", "np.any(ch == np.asarray(sector)[None, :], axis=1)",
     TD.test_dmrg_hubbard_vs_ed, ()),
    ("permutation: block keys moved, data not transposed", "oracle.blocksparse",
     "        blocks = {tuple(k[p] for p in perm): np.transpose(v, perm)",
     "        blocks = {tuple(k[p] for p in perm): v",
     TB.test_index_order_independence, ()),
    ("contraction: free sectors of B before those of A", "oracle.blocksparse",
     "            kc = tuple(ka[p] for p in fa) + tuple(kb[q] for q in fb)",
     "            kc = tuple(kb[q] for q in fb) + tuple(ka[p] for p in fa)",
     TB.test_blocksparse_contract_equals_dense, ()),
    ("contraction: contracted axes paired in reverse", "oracle.blocksparse",
     "            prod = np.tensordot(va, vb, axes=(ia, ib))",
     "            prod = np.tensordot(va, vb, axes=(ia, ib[::-1]))",
     TB.test_blocksparse_contract_equals_dense, ()),
    ("Lanczos: Ritz vector from shifted coefficients", "oracle.dmrg",
     "    for qi, si in zip(q[1:len(s)], s[1:]):", "    for qi, si in zip(q[1:len(s)], s[:-1]):",
     TD.test_lanczos_matches_eigh, ()),
    ("SVD: U columns out of order", "oracle.dmrg",
     "            Ut.blocks[rk + (ci,)] = U[roff[rk]:roff[rk] + rr, idx].reshape(shp + (len(idx),))",
     "            Ut.blocks[rk + (ci,)] = U[roff[rk]:roff[rk] + rr, idx[::-1]].reshape(shp + (len(idx),))",
     TD.test_svd_trunc_eckart_young_and_predicted_count, ()),
    ("SVD: a group's singular values in reverse", "oracle.dmrg",
     "        S[Q] = s[idx]", "        S[Q] = s[idx][::-1]",
     TD.test_svd_trunc_eckart_young_and_predicted_count, ()),
]


def plant(monkeypatch, modname, old, new):
    """Load ``modname`` with ``old`` replaced by ``new`` and rebind, for this
    test only, every reference to the original module's objects."""
    mod = importlib.import_module(modname)
    src = inspect.getsource(mod)
    assert src.count(old) == 1, f"the line to edit is not unique in {modname}"
    mutant = types.ModuleType(modname)
    mutant.__package__ = modname.rsplit(".", 1)[0]
    mutant.__file__ = mod.__file__
    exec(compile(src.replace(old, new), mod.__file__, "exec"), mutant.__dict__)
    repl = {}
    for name, val in mod.__dict__.items():
        if name.startswith("__") or name not in mutant.__dict__:
            continue
        own = getattr(val, "__module__", None) == modname
        if ((inspect.isfunction(val) or inspect.isclass(val)) and own) or isinstance(val, np.ndarray):
            repl[id(val)] = mutant.__dict__[name]
    for mname, module in list(sys.modules.items()):
        if module is None or not (mname == "oracle" or mname.startswith("oracle.") or mname.startswith("test_")
                                  or mname == "helpers"):
            continue
        for k, v in list(vars(module).items()):
            if id(v) in repl:
                monkeypatch.setattr(module, k, repl[id(v)])


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_pin_passes_on_the_unchanged_oracle(case, monkeypatch):
    # the loader itself changes nothing: the same source, reloaded, passes
    _, modname, old, _, pin, args = case
    plant(monkeypatch, modname, old, old)
    pin(*args)


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_planted_mistake_fails_its_pin(case, monkeypatch):
    _, modname, old, new, pin, args = case
    plant(monkeypatch, modname, old, new)
    # the pin's assertion, or the oracle's own shape, label and block checks
    # (the same pin passes on the unchanged source, above)
    with pytest.raises((AssertionError, ValueError, KeyError)):
        pin(*args)
