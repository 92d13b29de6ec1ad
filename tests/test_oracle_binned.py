"""Pins of the binned Debye sum (oracle/binned.py), the learned surrogate's baseline: Eq. 2 with every
pair distance replaced by its histogram bin centre.  It equals the exact sum when every pair sits at
a bin centre, gives the closed form (sum_i f_i(0))^2 at q = 0, and converges to the exact profile
as the bins shrink (pairs sit at random offsets inside bins of width w: the error falls about as w)."""
import numpy as np
import pytest

import oracle
from oracle import binned
from paper_1306_2258_gb300 import workloads as wl

N_BINS, R_MAX = 256, 120.0


def _tetrahedron(side):
    """Four atoms, six pair distances all equal to `side`."""
    v = np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]], dtype=np.float64)
    return v * (side / (2.0 * np.sqrt(2.0)))


def test_binned_profile_is_the_debye_sum_when_pairs_sit_at_bin_centres():
    """Two regular tetrahedra (side at the centres of bins 37 and 90, types mixed): the histogram puts
    all six pairs of each in its bin, and the binned sum equals the exact profile."""
    w = R_MAX / N_BINS
    coef = wl.form_factor_coefficients(3, 5)
    q = wl.q_grid(0.0, 0.5, 101)
    for k, types in ((37, [0, 1, 2, 1]), (90, [2, 2, 0, 1])):
        x = _tetrahedron((k + 0.5) * w)
        types = np.array(types, dtype=np.int32)
        h, dropped = oracle.pair_histogram(x.astype(np.float32), types, 3, N_BINS, R_MAX)
        assert dropped == 0 and h[:, k].sum() == 6 and h.sum() == 6
        I_bin = binned.profile(h[None], np.bincount(types, minlength=3), coef, q, N_BINS, R_MAX)[0]
        I_ref = oracle.profile(x, types, coef, q)
        assert np.max(np.abs(I_bin - I_ref) / I_ref) <= 1e-12


def test_binned_profile_at_q0_is_the_squared_sum_of_form_factors():
    mol = wl.random_walk_globule(400, 5, 83).as_f32()
    coef = wl.form_factor_coefficients(5, 84)
    h, dropped = oracle.pair_histogram(mol.coords, mol.types, 5, N_BINS, R_MAX)
    assert dropped == 0
    I0 = binned.profile(h[None], np.bincount(mol.types, minlength=5), coef, np.array([0.0]), N_BINS, R_MAX)[0, 0]
    f0 = oracle.form_factors(mol.types, coef, np.array([0.0]))[:, 0]
    assert I0 == pytest.approx(np.sum(f0) ** 2, rel=1e-13)


def test_binned_profile_converges_to_the_exact_profile_as_bins_shrink():
    """On a chain with 0.5 Å jitter (no repeated distance: the 3.8 Å bonds of a plain walk all sit at
    one offset inside their bin whatever its width)."""
    mol = wl.perturbed(wl.random_walk_globule(300, 4, 85), 0.5, 87).as_f32()
    coef = wl.form_factor_coefficients(4, 86)
    q = wl.q_grid(0.0, 0.5, 26)
    ref = oracle.profile(mol.coords, mol.types, coef, q)
    nt = np.bincount(mol.types, minlength=4)
    errs = []
    for n_bins in (256, 1024, 4096):
        h, dropped = oracle.pair_histogram(mol.coords, mol.types, 4, n_bins, R_MAX)
        assert dropped == 0
        errs.append(np.max(np.abs(binned.profile(h[None], nt, coef, q, n_bins, R_MAX)[0] - ref) / ref))
    assert errs[2] < errs[1] < errs[0]
    assert errs[2] <= 5e-4
