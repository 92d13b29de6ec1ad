"""Writes the stored expected values under tests/golden/ by calling only the
CPU oracle (package ``oracle``) on seeded inputs from the workload generators.

The paper prints no worked numerical example (its figures are plots and its
only table is timings), so every stored value here is the oracle's, pinned by
the closed-form, quadrature, lattice and invariance tests in tests/.

Run from the repository root:  python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1306_2258_gb300 import workloads as wl  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def main():
    w = wl.c1_plain_fp64()
    I, kap = oracle.profile(w.mol.coords, w.mol.types, w.coef, w.q, with_kappa=True)
    np.savetxt(os.path.join(HERE, "globule1000_q51_profile.txt"), np.stack([w.q, I, kap], 1),
               fmt="%.17g", header="1,000-atom globule (seeded random walk, R = 30 A, 5 types), "
               "q = 0..0.5 A^-1, 51 points; columns: q, I(q) (oracle, FP64), kappa(q)")


if __name__ == "__main__":
    main()
