"""Writes tgv_16c_p4_curves.txt next to this file: the Sec. III.C diagnostics E_k, eps_s and
eps_c of the Taylor-Green run of workload tgv_16c_p4 (16^3 cells, p = 4, Ma 0.5, Re 1600,
Courant number 4; the constant-temperature initial condition of Sec. III.C) at step 0 and
every 20 steps up to 200, computed by the FP64 oracle alone (oracle.init_fields,
oracle.tgv_fields, oracle.step, oracle.diag).  The time step and mu_inf come from the workload
definition (inputs.Workload.dt, inputs.Workload.mu_inf); the GPU test passes the same values.

    python tests/golden/make_tgv_curves.py        (about ten minutes on eight cores)
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_2012_05537_gb300 import inputs as I  # noqa: E402

STEPS, EVERY = 200, 20


def main():
    w = I.WORKLOADS["tgv_16c_p4"]
    g = O.Grid(cells=w.cells, p=w.p, dt=w.dt(), mu_inf=w.mu_inf, gamma=w.gamma, Pr=w.Pr)
    pop = O.init_fields(g, *O.tgv_fields(g, w.U0))
    rows = [(0, O.diag(g, pop, 1.0, w.Re, w.U0))]
    for k in range(EVERY, STEPS + 1, EVERY):
        pop = O.step(g, pop, EVERY)
        rows.append((k, O.diag(g, pop, 1.0, w.Re, w.U0)))
        print(k, rows[-1][1], flush=True)
    with open(os.path.join(HERE, "tgv_16c_p4_curves.txt"), "w") as f:
        f.write("# E_k, eps_s, eps_c (Sec. III.C, volume averages in units of U0) of the Taylor-Green run\n")
        f.write(f"# tgv_16c_p4: 16^3 cells, p = 4, Ma {w.Ma}, Re {w.Re}, dt {w.dt()!r}, mu_inf {w.mu_inf!r};\n")
        f.write("# written by tests/golden/make_tgv_curves.py from the FP64 oracle only\n")
        f.write("# step Ek eps_s eps_c\n")
        for k, d in rows:
            f.write(f"{k} {d[0]:.17e} {d[1]:.17e} {d[2]:.17e}\n")


if __name__ == "__main__":
    main()
