"""Write oracle_small.txt: the FP64 oracle's forces and energies on a 16-atom system.

A regression fixture for the oracle itself (it calls only ``oracle`` and the seeded
generator).  The paper prints no force or energy value, so nothing here is the
paper's; the oracle is pinned to closed forms and invariants by
tests/test_oracle_pins.py, and this file only guards it against unnoticed change.
Run from the repository root:  python tests/golden/make_oracle_fixture.py
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1611_04474_gb300 import workloads as W  # noqa: E402

SPEC = dict(n=16, box=(7.0, 7.5, 8.0), rc=3.4, seed=2024)


def compute():
    s = W.small_random(SPEC["n"], SPEC["box"], rc=SPEC["rc"], seed=SPEC["seed"])
    res = oracle.forces_cells(s.pos.astype(np.float64), s.q, s.type, s.box,
                              oracle.ForceField.from_system(s))
    return s, res


if __name__ == "__main__":
    s, res = compute()
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_small.txt")
    with open(path, "w") as f:
        f.write("# oracle forces on small_random(n=16, box=(7,7.5,8), rc=3.4, seed=2024)\n")
        f.write("# written by tests/golden/make_oracle_fixture.py (calls only oracle/)\n")
        f.write(f"npairs {res.npairs}\n")
        f.write("energy " + " ".join(f"{v:.17g}" for v in res.energy) + "\n")
        for i in range(s.n):
            f.write("F " + " ".join(f"{v:.17g}" for v in res.F[i]) + "\n")
    print("wrote", path)
