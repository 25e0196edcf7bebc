"""Writes the stored expected values under tests/golden/.

The paper (arXiv 1008.2801) prints no worked example for its Poisson solve,
so the stored values come from the oracle alone (this script imports nothing
but the oracle, numpy and the seeded input generator, which holds no solver
arithmetic).  Run from the repository root:  python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1008_2801_gb300 import inputs  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def main():
    # a ragged box with a coarsest level of 6 cells and a stellar beta
    nx, ny, nz = 12, 4, 8
    d = inputs.stellar((nx, ny, nz), 77)
    phi, info = oracle.solve(d["beta"], d["f"], d["dx"], tol=1e-14)
    assert info["status"] == "ok"
    with open(os.path.join(HERE, "stellar_12x4x8.txt"), "w") as fh:
        fh.write("# oracle solution of div(beta grad phi) = f, stellar input seed 77, "
                 "(nx, ny, nz) = (12, 4, 8), dx = 1/12, tol 1e-14\n")
        fh.write("# written by tests/golden/make_golden.py; C order (nz, ny, nx)\n")
        for v in phi.ravel():
            fh.write(f"{v:.17e}\n")


if __name__ == "__main__":
    main()
