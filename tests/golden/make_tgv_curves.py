"""Writes the Taylor-Green diagnostics files next to this file: the Sec. III.C quantities
E_k, eps_s and eps_c of a Taylor-Green run (constant-temperature initial condition of
Sec. III.C), computed by the FP64 oracle alone (oracle.init_fields, oracle.tgv_fields,
oracle.step, oracle.diag).  The time step, mu_inf and the Prandtl-term flag come from the
workload definition (inputs.Workload); the GPU tests pass the same values.

* tgv_16c_p4_curves.txt: workload tgv_16c_p4 (16^3 cells, p = 4, Ma 0.5, Re 1600, Courant
  number 4), step 0 and every 20 steps up to 200 (about ten minutes on eight cores);
* tgv_16c_p4_c2_curves.txt: workload tgv_16c_p4_c2 (the same mesh at Courant number 2, the
  time step of the 128^3-node throughput workload, Prandtl term on), step 0 and every 50
  steps up to 2000 (about three hours on eight cores).  Rows are written as the run goes;
  the oracle's diagnostic sums are reduced in parallel, so two runs agree to about 1e-13
  relative, not bit for bit.

    python tests/golden/make_tgv_curves.py [tgv_16c_p4 | tgv_16c_p4_c2]
"""
import math
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_2012_05537_gb300 import inputs as I  # noqa: E402

RUNS = {"tgv_16c_p4": (200, 20), "tgv_16c_p4_c2": (2000, 50)}


def main(name: str = "tgv_16c_p4"):
    steps, every = RUNS[name]
    w = I.WORKLOADS[name]
    g = O.Grid(cells=w.cells, p=w.p, dt=w.dt(), mu_inf=w.mu_inf, gamma=w.gamma, Pr=w.Pr,
               pr_correction=w.pr_correction)
    pop = O.init_fields(g, *O.tgv_fields(g, w.U0))
    with open(os.path.join(HERE, f"{name}_curves.txt"), "w") as f:
        f.write("# E_k, eps_s, eps_c (Sec. III.C, volume averages in units of U0) of the Taylor-Green run\n")
        f.write(f"# {name}: {w.cells[0]}^3 cells, p = {w.p}, Ma {w.Ma}, Re {w.Re}, dt {w.dt()!r}, "
                f"mu_inf {w.mu_inf!r}, Prandtl term {'on' if w.pr_correction else 'off'};\n")
        f.write("# written by tests/golden/make_tgv_curves.py from the FP64 oracle only\n")
        f.write("# step Ek eps_s eps_c\n")
        d = O.diag(g, pop, 1.0, w.Re, w.U0)
        f.write(f"0 {d[0]:.17e} {d[1]:.17e} {d[2]:.17e}\n")
        for k in range(every, steps + 1, every):
            pop = O.step(g, pop, every)
            d = O.diag(g, pop, 1.0, w.Re, w.U0)
            if not all(math.isfinite(v) for v in d):
                print(k, "non-finite: stopping", flush=True)
                break
            f.write(f"{k} {d[0]:.17e} {d[1]:.17e} {d[2]:.17e}\n")
            f.flush()
            print(k, d, flush=True)


if __name__ == "__main__":
    main(*sys.argv[1:2])
