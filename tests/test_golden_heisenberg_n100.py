"""Pins of the stored oracle energy of the N=100 Heisenberg sweeps.

tests/golden/heisenberg_n100_dmrg.json is written by
tests/golden/make_heisenberg_n100.py, which runs the oracle's two-site DMRG
(Sec. 7.2) on the benchmark's schedule; bench.py reports the GPU energies
against it. The checks here tie the stored number to the benchmark's run and
to the Bethe-ansatz ground-state energy of the open chain.
"""
import math

import bench


def test_golden_run_is_the_benchmark_run():
    ref = bench.sweep_reference()
    assert [tuple(x) for x in ref["schedule"]] == bench.SWEEP_SCHEDULE
    assert ref["krylov_dim"] == 16
    assert f"N={bench.SWEEP_N}" in ref["model"]
    assert ref["energy"] == ref["sweeps"][-1]["energy"]
    assert len(ref["sweeps"]) == len(bench.SWEEP_SCHEDULE)
    assert all(s["maxdim"] <= m for s, (m, _) in zip(ref["sweeps"], bench.SWEEP_SCHEDULE))


def test_golden_energy_is_variational():
    # each sweep lowers the energy (two-site DMRG with growing maxdim)
    es = [s["energy"] for s in bench.sweep_reference()["sweeps"]]
    assert all(b <= a + 1e-10 for a, b in zip(es, es[1:]))
    # the last two sweeps (maxdim 256 both) agree: converged
    assert abs(es[-1] - es[-2]) < 1e-8 * abs(es[-1])


def test_golden_energy_matches_bethe_ansatz_open_chain():
    # open S=1/2 XXX chain of N sites: E0(N) = N e_inf + e_surface + O(1/N),
    # e_inf = 1/4 - ln 2 and e_surface = (pi - 1 - 2 ln 2) / 4 from the Bethe
    # ansatz; the O(1/N) remainder is a few 1e-3 at N = 100
    N = bench.SWEEP_N
    e_inf = 0.25 - math.log(2.0)
    e_surf = (math.pi - 1.0 - 2.0 * math.log(2.0)) / 4.0
    E = bench.sweep_reference()["energy"]
    assert abs(E - (N * e_inf + e_surf)) < 5e-3
