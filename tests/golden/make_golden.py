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


def small_case():
    """The 300-atom inputs of the per-atom, gradient and histogram fixtures."""
    mol = wl.random_walk_globule(300, 4, 4401)
    coef = wl.form_factor_coefficients(4, 4402)
    q = wl.q_grid(0.0, 0.6, 21)
    ff = wl.atomic_form_factor_table(mol.n, q, 4403)
    gI = np.linspace(-1.0, 2.0, q.size)
    return mol, coef, q, ff, gI


def main():
    w = wl.c1_plain_fp64()
    I, kap = oracle.profile(w.mol.coords, w.mol.types, w.coef, w.q, with_kappa=True)
    np.savetxt(os.path.join(HERE, "globule1000_q51_profile.txt"), np.stack([w.q, I, kap], 1),
               fmt="%.17g", header="1,000-atom globule (seeded random walk, R = 30 A, 5 types), "
               "q = 0..0.5 A^-1, 51 points; columns: q, I(q) (oracle, FP64), kappa(q)")
    mol, coef, q, ff, gI = small_case()
    Ia = oracle.profile_atomic(mol.coords, ff, q)
    np.savetxt(os.path.join(HERE, "globule300_q21_atomic_profile.txt"), np.stack([q, Ia], 1), fmt="%.17g",
               header="300-atom globule (seed 4401), per-atom form-factor table (seed 4403), q = 0..0.6 A^-1, "
               "21 points; columns: q, I(q) (oracle, FP64)")
    g = oracle.vjp(mol.coords, mol.types, coef, q, gI)
    ga = oracle.vjp_atomic(mol.coords, ff, q, gI)
    np.savetxt(os.path.join(HERE, "globule300_q21_vjp.txt"), np.concatenate([g, ga], 1), fmt="%.17g",
               header="300-atom globule (seed 4401, 4 types, coefficients seed 4402), q = 0..0.6 A^-1 x 21, "
               "grad_I = linspace(-1, 2, 21); columns: sum_q grad_I dI/dx (x, y, z) with the typed form "
               "factors, then with the per-atom table (seed 4403) (oracle, FP64)")
    h, dropped = oracle.pair_histogram(mol.coords.astype(np.float32), mol.types, 4, 64, 40.0)
    np.savetxt(os.path.join(HERE, "globule300_hist64_r40.txt"), h, fmt="%d",
               header=f"300-atom globule (seed 4401, 4 types) as float32, 64 bins to 40 A; rows: type pairs "
               f"a <= b in row-major order; dropped pairs: {dropped}")


if __name__ == "__main__":
    main()
