"""Host-side parts of the surrogate pipeline on CPU: the Debye sum over a distance histogram with
every pair at its bin centre (the method without the network, against which the network's gain is
reported), the pair totals and the normalised features.  Pinned to the FP64 oracle."""
import numpy as np

import oracle
from paper_1306_2258_gb300 import workloads as wl
from paper_1306_2258_gb300.surrogate import N_BINS, R_MAX, binned_sinc_profiles, histogram_features, pair_totals


def _tetrahedron(side):
    """Four atoms, six pair distances all equal to `side`."""
    v = np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]], dtype=np.float64)
    return v * (side / (2.0 * np.sqrt(2.0)))


def test_binned_profile_is_the_debye_sum_when_pairs_sit_at_bin_centres():
    """Two regular tetrahedra (side at the centres of bins 37 and 90, types mixed): the histogram puts
    all six pairs of each in its bin, and the binned Debye sum equals the oracle's profile of the
    exact geometry."""
    w = R_MAX / N_BINS
    coef = wl.form_factor_coefficients(3, 5)
    q = wl.q_grid(0.0, 0.5, 101)
    for k, types in ((37, [0, 1, 2, 1]), (90, [2, 2, 0, 1])):
        x = _tetrahedron((k + 0.5) * w)
        types = np.array(types, dtype=np.int32)
        h, dropped = oracle.pair_histogram(x.astype(np.float32), types, 3, N_BINS, R_MAX)
        assert dropped == 0 and h[:, k].sum() == 6 and h.sum() == 6
        I_bin = binned_sinc_profiles(h[None], types, coef, q)[0]
        I_ref = oracle.profile(x, types, coef, q)
        assert np.max(np.abs(I_bin - I_ref) / I_ref) <= 1e-12


def test_pair_totals_and_features_normalise_each_type_pair():
    mol = wl.random_walk_globule(500, 4, 81).as_f32()
    h, dropped = oracle.pair_histogram(mol.coords, mol.types, 4)
    tot = pair_totals(mol.types, 4)
    assert dropped == 0
    np.testing.assert_array_equal(h.sum(axis=1), tot)
    f = histogram_features(h[None], tot)
    assert f.shape == (1, tot.size * N_BINS)
    np.testing.assert_allclose(f.reshape(tot.size, N_BINS).sum(axis=1), 1.0, rtol=1e-12)
