#!/usr/bin/env python3
"""Write heisenberg_n100_dmrg.json: the oracle's two-site DMRG energy of the
S=1/2 Heisenberg chain, N=100, open ends, U(1) (total Sz) conserving, from the
Neel state, maxdim 32, 64, 128, 256, 256 with cutoff 1e-12 and at most 16
Lanczos steps per bond (tolerance 1e-9): the schedule of the benchmark's
N=100 sweeps (Sec. 7.2 for the method). Calls only oracle/.

    python tests/golden/make_heisenberg_n100.py
"""
import json
import os
import platform
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import dmrg as D, models as om  # noqa: E402

N = 100
SCHEDULE = [(32, 1e-12), (64, 1e-12), (128, 1e-12), (256, 1e-12), (256, 1e-12)]
KRYLOV, TOL = 16, 1e-9


def main():
    mpo = om.heisenberg_mpo(N)
    A = D.product_mps_basis(mpo.site_index, [0, 1] * (N // 2), 1)
    marks = [time.perf_counter()]
    stats = []

    def observer(st):
        marks.append(time.perf_counter())
        stats.append(st)
        print(f"sweep {st['sweep']}: E {st['energy']:.12f} maxdim {st['maxdim']} "
              f"truncerr {st['truncerr']:.2e} ({marks[-1] - marks[-2]:.1f} s)", flush=True)

    E, _, _ = D.dmrg(mpo, A, SCHEDULE, KRYLOV, TOL, observer=observer)
    out = {
        "_source": "oracle two-site DMRG (numpy float64), written by tests/golden/make_heisenberg_n100.py",
        "model": f"S=1/2 Heisenberg chain N={N}, open ends, U(1), Neel start",
        "schedule": SCHEDULE, "krylov_dim": KRYLOV, "tol": TOL,
        "energy": E,
        "sweeps": [{"sweep": s["sweep"], "energy": s["energy"], "maxdim": s["maxdim"],
                    "truncerr": s["truncerr"], "matvecs": s["matvecs"],
                    "seconds": marks[i + 1] - marks[i]} for i, s in enumerate(stats)],
        "host": f"{platform.machine()}, {os.cpu_count()} cores",
    }
    with open(os.path.join(HERE, "heisenberg_n100_dmrg.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
