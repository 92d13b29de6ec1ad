"""Host-side parts of the surrogate pipeline on CPU: the pair totals and the normalised features,
against the FP64 oracle's histograms."""
import numpy as np

import oracle
from paper_1306_2258_gb300 import workloads as wl
from paper_1306_2258_gb300.surrogate import N_BINS, histogram_features, pair_totals


def test_pair_totals_and_features_normalise_each_type_pair():
    mol = wl.random_walk_globule(500, 4, 81).as_f32()
    h, dropped = oracle.pair_histogram(mol.coords, mol.types, 4)
    tot = pair_totals(mol.types, 4)
    assert dropped == 0
    np.testing.assert_array_equal(h.sum(axis=1), tot)
    f = histogram_features(h[None], tot)
    assert f.shape == (1, tot.size * N_BINS)
    np.testing.assert_allclose(f.reshape(tot.size, N_BINS).sum(axis=1), 1.0, rtol=1e-12)
