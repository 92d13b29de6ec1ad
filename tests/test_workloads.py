"""The seeded synthetic inputs: deterministic for a seed, and shaped as stated (sizes, bond lengths,
confinement, type ranges, lengths, per-atom form-factor ranges).  CPU only."""
import numpy as np
import pytest

from paper_1306_2258_gb300 import workloads as wl


def test_same_seed_same_molecule_and_different_seed_different_molecule():
    a = wl.random_walk_globule(500, 5, 11)
    b = wl.random_walk_globule(500, 5, 11)
    c = wl.random_walk_globule(500, 5, 12)
    assert np.array_equal(a.coords, b.coords) and np.array_equal(a.types, b.types)
    assert not np.array_equal(a.coords, c.coords)


@pytest.mark.parametrize("n", [1000, 10000])
def test_globule_bonds_confinement_and_types(n):
    m = wl.random_walk_globule(n, 5, wl.seed_for(2, n))
    assert m.coords.shape == (n, 3) and m.types.shape == (n,)
    assert m.types.min() >= 0 and m.types.max() < 5
    bonds = np.linalg.norm(np.diff(m.coords, axis=0), axis=1)
    np.testing.assert_allclose(bonds, 3.8, rtol=1e-9)
    R = wl.globule_radius(n)
    assert np.linalg.norm(m.coords, axis=1).max() <= R + 3.8
    assert abs(wl.globule_radius(1000) - 30.0) < 1e-12


def test_rod_and_sparse_chain_shapes():
    rod = wl.c3_rod().mol
    assert rod.n == 30000
    ext = rod.coords.max(axis=0) - rod.coords.min(axis=0)
    assert 4500 < ext.max() < 5600                       # ~5,100 A long
    radial = np.sort(ext)[:2]
    assert radial.max() < 25                             # radius ~10 A
    chain = wl.free_chain(2000, 3, 5)
    np.testing.assert_allclose(np.linalg.norm(np.diff(chain.coords, axis=0), axis=1), 6.0, rtol=1e-9)
    assert set(np.unique(chain.types)) <= {0, 1, 2}


def test_refinement_and_ensemble_shapes():
    c4 = wl.c4_refinement(n=600, batch=3)
    assert c4["conformers"].shape == (3, 600, 3) and c4["conformers"].dtype == np.float32
    assert c4["q"][0] == 0.01 and c4["q"][-1] == 0.5 and c4["q"].size == 101
    d = np.linalg.norm(c4["conformers"][0] - c4["base"].coords, axis=1)
    assert 0.5 < np.sqrt(np.mean(d ** 2) / 3) < 1.5    # N(0, 1 A^2) displacements
    c5 = wl.c5_ensemble(n_conf=4, n=300)
    assert c5["conformers"].shape == (4, 300, 3) and c5["q"].size == 101 and c5["q"][0] == 0.0


def test_form_factor_coefficient_ranges():
    c = wl.form_factor_coefficients(16, 3)
    assert c.shape == (16, 9)
    assert np.all((c[:, 0:4] >= 0.5) & (c[:, 0:4] <= 3.0))
    assert np.all((c[:, 4:8] >= 0.5) & (c[:, 4:8] <= 40.0))
    assert np.all((c[:, 8] >= 0.0) & (c[:, 8] <= 0.5))


def test_atomic_form_factor_table_shape_and_ranges():
    q = wl.q_grid(0.0, 1.0, 21)
    ff = wl.atomic_form_factor_table(800, q, 7)
    assert ff.shape == (21, 800) and ff.flags["C_CONTIGUOUS"] and np.all(np.isfinite(ff))
    # at q = 0: a + c + d with a in [1, 8], c in [-0.3, 0.3], d in [-1, 1.5] on the shell atoms
    assert ff[0].min() >= 1.0 - 0.3 - 1.0 and ff[0].max() <= 8.0 + 0.3 + 1.5
    # at q = 1 the Gaussians have decayed at most to a e^-0.5 and d e^-0.6
    assert ff[-1].min() >= 1.0 * np.exp(-0.5) - 0.3 - 1.0 and ff[-1].max() <= 8.0 + 0.3 + 1.5
    np.testing.assert_array_equal(ff, wl.atomic_form_factor_table(800, q, 7))


def test_q_grid_endpoints():
    q = wl.q_grid(0.0, 1.0, 201)
    assert q[0] == 0.0 and q[-1] == 1.0 and q.size == 201
    np.testing.assert_allclose(np.diff(q), 0.005, rtol=1e-9)


def test_cubic_lattice_and_spherical_shell_shapes():
    lat = wl.cubic_lattice(5, 6.5, 5, 3)
    assert lat.n == 125 and lat.types.min() >= 0 and lat.types.max() < 5
    np.testing.assert_allclose(lat.coords.mean(axis=0), 0.0, atol=1e-12)
    d2 = np.sum((lat.coords[:, None] - lat.coords[None]) ** 2, axis=-1) / 6.5 ** 2
    np.testing.assert_allclose(d2, np.round(d2), atol=1e-9)       # squared distances on the integer lattice
    shell = wl.spherical_shell(2000, 100.0, 5, 4)
    np.testing.assert_allclose(np.linalg.norm(shell.coords, axis=1), 100.0, rtol=1e-12)
    assert np.linalg.norm(shell.coords.mean(axis=0)) < 10.0       # uniform over the sphere
    assert np.array_equal(shell.coords, wl.spherical_shell(2000, 100.0, 5, 4).coords)
