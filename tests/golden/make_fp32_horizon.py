"""Write the FP64 oracle's 1000-step observable records of the two horizon workloads
(tests/_util.py: horizon_molecule, horizon_cell) to fp32_horizon_<name>.txt.

The records are the reference of the 1000-step complex64 checks in tests/test_gpu_horizon.py
(the dipole, or the current of the periodic cell, within 1e-4 of its peak after 1000 steps).
Only the oracle computes them: the Taylor-4 propagator of Sec. "New propagators for real-time
TDDFT" with the observables of the record (norm, energy, dipole or current).  Run from the
repository root:  python tests/golden/make_fp32_horizon.py [molecule|cell ...]
"""
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1912_07921_gb300 import inputs as I  # noqa: E402
from tests._util import HORIZON_CASES  # noqa: E402


def main(names):
    for name in names:
        spec = HORIZON_CASES[name](I.PREC_C128)
        inp = I.make_inputs(spec)
        t0 = time.time()
        _, rec = oracle.System(spec, inp).propagate(inp.psi0, 0.0, spec.dt, spec.n_steps, spec.substeps)
        path = os.path.join(HERE, f"fp32_horizon_{name}.txt")
        with open(path + ".tmp", "w") as f:
            f.write(f"# FP64 oracle, Taylor-4 propagator: {spec.describe()}\n")
            f.write("# written by tests/golden/make_fp32_horizon.py (oracle only)\n")
            f.write("# step t norm energy E_x o_x o_y o_z field  (o = dipole, or current in a periodic cell)\n")
            for s, r in enumerate(rec):
                f.write(f"{s} " + " ".join(f"{x:.17g}" for x in r) + "\n")
        os.replace(path + ".tmp", path)
        print(f"{name}: {spec.n_steps} steps in {time.time() - t0:.0f} s -> {path}")


if __name__ == "__main__":
    main(sys.argv[1:] or sorted(HORIZON_CASES))
