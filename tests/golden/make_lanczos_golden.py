"""Write lanczos_workload1.txt: the oracle's Lanczos ground-state energy for workload 1.

Workload 1 is the periodic Heisenberg chain L = 20, N = 10 (J = 1, delta = 1, n_sub = 2) with
its seeded start vector. The value is what the plain CPU oracle computes (full
re-orthogonalisation, 100 steps, the recurrence of Sec. 4.4 / App. D), so the GPU Lanczos driver
started from the same vector must reproduce it. Only the oracle and the seeded input generator
are called. About a minute of CPU time.

    python tests/golden/make_lanczos_golden.py
"""

import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import OracleSector, lanczos, matvec, most_equal_partition, sector_dim  # noqa: E402
from paper_2407_14591_gb300 import workloads as wl  # noqa: E402

STEPS = 100


def main():
    w, _ = wl.workload(1, draw_vector=False)
    D = sector_dim(w.L, w.Q, w.N)
    w, x = wl.workload(1, D=D)
    o = OracleSector(w.L, w.Q, w.N, partition=most_equal_partition(w.L, w.n_sub, w.Q))
    res = lanczos(lambda v: matvec(o, w.terms, v), x, STEPS)
    with open(os.path.join(HERE, "lanczos_workload1.txt"), "w") as f:
        f.write("# Lanczos ground-state energy of workload 1 (periodic Heisenberg chain L=20, N=10,\n")
        f.write("# J=1, delta=1, n_sub=2) from its seeded start vector, 100 steps with full\n")
        f.write("# re-orthogonalisation, as computed by the CPU oracle (Sec. 4.4, App. D recurrence).\n")
        f.write("# Written by tests/golden/make_lanczos_golden.py.\n")
        f.write(f"L {w.L}\nN {w.N}\ndim {D}\nsteps {res['steps_done']}\nE0 {res['E0']!r}\n")
    print(res["E0"], res["steps_done"])


if __name__ == "__main__":
    main()
