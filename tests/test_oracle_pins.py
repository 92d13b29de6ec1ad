"""Pins of the FP64 CPU oracle against what the physics and the mathematics fix.

None of these retypes the oracle's double loop: each checks it against a closed
form, a special case that reduces to a library routine, an independent route
(the orientation average of Eq. 1 by quadrature, integer pair counts on a
lattice), brute force, or an invariance.  A dropped diagonal, a missing factor
of two, a wrong (q/4pi) scaling, a wrong sign or a transposed index fails at
least one of them.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1306_2258_gb300 import workloads as wl


def _coef_simple(T=1):
    """Coefficients with a1 = 1, b1 = 16 pi^2 (so exp(-b1 (q/4pi)^2) = exp(-q^2)), rest 0, c = 0.25."""
    c = np.zeros((T, 9))
    c[:, 0] = 1.0
    c[:, 4] = 16.0 * math.pi ** 2
    c[:, 8] = 0.25
    return c


# ---------------------------------------------------------------- form factors

def test_form_factor_closed_forms():
    q = np.array([0.0, 0.3, 1.0, 2.0])
    f = oracle.form_factors([0], _coef_simple(), q)[0]
    np.testing.assert_allclose(f, np.exp(-q * q) + 0.25, rtol=0, atol=1e-15)
    coef = wl.form_factor_coefficients(5, 7)
    f0 = oracle.form_factors(np.arange(5), coef, [0.0])[:, 0]
    np.testing.assert_allclose(f0, coef[:, 0:4].sum(1) + coef[:, 8], rtol=1e-15)   # f(0) = sum a + c
    finf = oracle.form_factors(np.arange(5), coef, [1e4])[:, 0]
    np.testing.assert_allclose(finf, coef[:, 8], rtol=1e-15)                          # f(inf) = c


# ---------------------------------------------------------------- closed forms

@pytest.mark.parametrize("r", [0.0, 1e-7, 3.8, 100.0, 5000.0])
def test_two_atoms_closed_form(r):
    coef = wl.form_factor_coefficients(2, 11)
    q = wl.q_grid(0.0, 1.0, 41)
    xyz = np.array([[0.3, -1.2, 2.0], [0.3 + r, -1.2, 2.0]])
    types = np.array([0, 1])
    I = oracle.profile(xyz, types, coef, q)
    f = oracle.form_factors(types, coef, q)
    x = q * r
    s = np.where(x == 0, 1.0, np.sin(x) / np.where(x == 0, 1.0, x))
    expect = f[0] ** 2 + f[1] ** 2 + 2 * f[0] * f[1] * s
    np.testing.assert_allclose(I, expect, rtol=1e-14, atol=0)


def test_two_atoms_at_zeros_of_sinc():
    """q r = m pi makes the cross term vanish: I = f1^2 + f2^2."""
    coef = wl.form_factor_coefficients(2, 12)
    r = 7.25
    q = np.arange(1, 30) * math.pi / r
    xyz = np.array([[0, 0, 0], [0, 0, r]], dtype=float)
    I = oracle.profile(xyz, [0, 1], coef, q)
    f = oracle.form_factors([0, 1], coef, q)
    np.testing.assert_allclose(I, f[0] ** 2 + f[1] ** 2, rtol=1e-13)


def test_single_atom_and_empty():
    coef = wl.form_factor_coefficients(3, 13)
    q = wl.q_grid(0, 1, 11)
    I1 = oracle.profile(np.array([[1.0, 2.0, 3.0]]), [2], coef, q)
    np.testing.assert_allclose(I1, oracle.form_factors([2], coef, q)[0] ** 2, rtol=1e-15)
    I0 = oracle.profile(np.zeros((0, 3)), np.zeros(0, np.int32), coef, q)
    assert np.all(I0 == 0.0)


def test_zero_q_is_square_of_total_form_factor():
    mol = wl.random_walk_globule(300, 5, 21)
    coef = wl.form_factor_coefficients(5, 22)
    q = np.array([0.0, 0.1])
    I = oracle.profile(mol.coords, mol.types, coef, q)
    f = oracle.form_factors(mol.types, coef, q)
    assert I[0] == pytest.approx(f[:, 0].sum() ** 2, rel=1e-14)


def test_coincident_atoms():
    """All atoms at one point: I(q) = (sum_i f_i(q))^2 at every q."""
    coef = wl.form_factor_coefficients(4, 23)
    types = np.array([0, 1, 2, 3, 1, 0, 2])
    xyz = np.tile([[5.0, -2.0, 1.0]], (types.size, 1))
    q = wl.q_grid(0, 1, 21)
    I = oracle.profile(xyz, types, coef, q)
    f = oracle.form_factors(types, coef, q)
    np.testing.assert_allclose(I, f.sum(0) ** 2, rtol=1e-14)


def test_single_type_powder_form_with_library_sinc():
    """T = 1: I = f^2 (N + 2 sum_{i<j} sinc(q r_ij)), the identical-atom form; the
    sinc sum is taken with numpy.sinc over scipy's pdist distances."""
    from scipy.spatial.distance import pdist
    mol = wl.random_walk_globule(150, 1, 24)
    coef = wl.form_factor_coefficients(1, 25)
    q = wl.q_grid(0.0, 1.0, 26)
    I = oracle.profile(mol.coords, mol.types, coef, q)
    f = oracle.form_factors([0], coef, q)[0]
    d = pdist(mol.coords)
    ssum = np.array([np.sum(np.sinc(qq * d / math.pi)) for qq in q])
    np.testing.assert_allclose(I, f * f * (mol.n + 2 * ssum), rtol=1e-12)


# ---------------------------------------------------------------- independent routes

def _eq1_quadrature(xyz, f_atoms, q, n_theta=72, n_phi=144):
    """<|sum_j f_j exp(i q.r_j)|^2> over the sphere (Eq. 1): Gauss-Legendre in cos(theta)
    times the uniform rule in phi.  Exact to rounding for band-limited integrands."""
    x, w = np.polynomial.legendre.leggauss(n_theta)
    phi = 2 * math.pi * np.arange(n_phi) / n_phi
    st = np.sqrt(1 - x * x)
    u = np.stack([st[:, None] * np.cos(phi)[None, :], st[:, None] * np.sin(phi)[None, :],
                  np.broadcast_to(x[:, None], (n_theta, n_phi))], -1).reshape(-1, 3)
    wt = np.repeat(w / 2.0, n_phi) / n_phi
    out = np.empty(q.size)
    proj = u @ xyz.T                                   # [dirs, atoms]
    for k, qq in enumerate(q):
        amp = np.exp(1j * qq * proj) @ f_atoms[:, k]
        out[k] = np.sum(wt * np.abs(amp) ** 2)
    return out


@pytest.mark.parametrize("seed", [31, 32, 33])
def test_eq2_matches_eq1_orientation_average(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(2, 13))
    xyz = rng.uniform(-8, 8, size=(n, 3))           # diameter <= ~28 A
    types = rng.integers(0, 3, size=n)
    coef = wl.form_factor_coefficients(3, seed + 100)
    q = wl.q_grid(0.0, 0.5, 11)
    I2 = oracle.profile(xyz, types, coef, q)
    f = oracle.form_factors(types, coef, q)
    I1 = _eq1_quadrature(xyz, f, q)
    np.testing.assert_allclose(I2, I1, rtol=1e-12)


def test_lattice_integer_distance_counts():
    """On a cubic lattice of spacing d every squared distance is d^2 * n with integer n,
    so I(q) = sum_i f_i^2 + 2 sum_{a<=b} f_a f_b sum_n c_ab(n) sinc(q d sqrt n) with exact
    integer counts c_ab(n) from integer arithmetic."""
    rng = np.random.default_rng(41)
    d = 1.7
    ijk = np.unique(rng.integers(-4, 5, size=(90, 3)), axis=0)
    n = ijk.shape[0]
    types = rng.integers(0, 3, size=n)
    coef = wl.form_factor_coefficients(3, 42)
    q = wl.q_grid(0.0, 1.0, 21)
    counts = {}
    for i in range(n):
        for j in range(i + 1, n):
            m = int(np.sum((ijk[i] - ijk[j]) ** 2))
            key = (min(types[i], types[j]), max(types[i], types[j]), m)
            counts[key] = counts.get(key, 0) + 1
    F = oracle.form_factors(np.arange(3), coef, q)
    expect = np.sum(F[types] ** 2, axis=0)
    for (a, b, m), c in counts.items():
        x = q * d * math.sqrt(m)
        expect = expect + 2 * F[a] * F[b] * c * np.where(x == 0, 1.0, np.sin(x) / np.where(x == 0, 1, x))
    I = oracle.profile(ijk * d, types, coef, q)
    np.testing.assert_allclose(I, expect, rtol=1e-13)


def test_half_sum_equals_full_double_loop():
    mol = wl.random_walk_globule(180, 5, 43)
    coef = wl.form_factor_coefficients(5, 44)
    q = wl.q_grid(0, 1, 31)
    np.testing.assert_allclose(oracle.profile(mol.coords, mol.types, coef, q),
                               oracle.profile_full(mol.coords, mol.types, coef, q), rtol=1e-14)


def test_pair_sums_assemble_profile_and_count_pairs():
    mol = wl.random_walk_globule(220, 4, 45)
    coef = wl.form_factor_coefficients(4, 46)
    q = wl.q_grid(0, 1, 17)
    S = oracle.pair_sums(mol.coords, mol.types, 4, q)
    F = oracle.form_factors(np.arange(4), coef, q)
    nt = np.bincount(mol.types, minlength=4)
    I = np.sum(nt[:, None] * F ** 2, axis=0)
    for a in range(4):
        for b in range(a, 4):
            p = oracle.pair_index(a, b, 4)
            I = I + 2 * F[a] * F[b] * S[p]
            assert S[p, 0] == (nt[a] * (nt[a] - 1) // 2 if a == b else nt[a] * nt[b])
    np.testing.assert_allclose(I, oracle.profile(mol.coords, mol.types, coef, q), rtol=1e-13)


# ---------------------------------------------------------------- per-atom form factors

@pytest.mark.parametrize("seed", [61, 62])
def test_atomic_eq2_matches_eq1_orientation_average(seed):
    """Per-atom f_i(q) of arbitrary sign and shape (no types): Eq. 2 against the orientation
    average of Eq. 1 by quadrature, an independent route."""
    rng = np.random.default_rng(seed)
    n = int(rng.integers(3, 12))
    xyz = rng.uniform(-8, 8, size=(n, 3))
    q = wl.q_grid(0.0, 0.5, 7)
    ff = rng.uniform(-2.0, 6.0, size=(q.size, n))      # [n_q, n]: any value at any q
    I2 = oracle.profile_atomic(xyz, ff, q)
    I1 = _eq1_quadrature(xyz, ff.T.copy(), q)
    np.testing.assert_allclose(I2, I1, rtol=1e-12, atol=1e-12 * np.max(np.abs(I1)))


def test_atomic_two_atoms_closed_form():
    """I = f1^2 + f2^2 + 2 f1 f2 sin(q r)/(q r) with different f1(q), f2(q) at every q."""
    q = np.array([0.0, 0.13, 0.4, 0.77, 1.5])
    ff = np.array([[3.0, -1.25], [2.5, 0.5], [1.75, 2.0], [-0.5, 4.0], [0.25, 0.125]])
    r = 4.3
    xyz = np.array([[0.0, 0.0, 0.0], [r, 0.0, 0.0]])
    x = q * r
    sinc = np.where(x == 0, 1.0, np.sin(x) / np.where(x == 0, 1.0, x))
    expect = ff[:, 0] ** 2 + ff[:, 1] ** 2 + 2 * ff[:, 0] * ff[:, 1] * sinc
    np.testing.assert_allclose(oracle.profile_atomic(xyz, ff, q), expect, rtol=1e-14)


def test_atomic_zero_q_is_square_of_total():
    mol = wl.random_walk_globule(200, 1, 63)
    q = wl.q_grid(0.0, 0.3, 4)
    ff = wl.atomic_form_factor_table(mol.n, q, 64)
    I = oracle.profile_atomic(mol.coords, ff, q)
    assert math.isclose(I[0], math.fsum(ff[0]) ** 2, rel_tol=1e-14)


def test_atomic_quadratic_in_shell_weight_and_types_limit():
    """f_i(q) = f_type(i)(q) + lam g_i(q): I(lam) is a quadratic in lam (equal second
    differences), and at lam = 0 it is the typed profile."""
    mol = wl.random_walk_globule(160, 3, 65)
    coef = wl.form_factor_coefficients(3, 66)
    q = wl.q_grid(0.0, 1.0, 11)
    f0 = oracle.form_factors(mol.types, coef, q).T.copy()          # [n_q, n]
    g = wl.atomic_form_factor_table(mol.n, q, 67) - 4.0
    I = {lam: oracle.profile_atomic(mol.coords, f0 + lam * g, q) for lam in (-1, 0, 1, 2)}
    np.testing.assert_allclose(I[2] - 2 * I[1] + I[0], I[1] - 2 * I[0] + I[-1],
                               rtol=1e-9, atol=1e-9 * np.max(np.abs(I[1])))
    np.testing.assert_allclose(I[0], oracle.profile(mol.coords, mol.types, coef, q), rtol=1e-14)


# ---------------------------------------------------------------- invariances

def _mol_case(n=250, seed=51):
    mol = wl.random_walk_globule(n, 5, seed)
    return mol, wl.form_factor_coefficients(5, seed + 1), wl.q_grid(0, 1, 21)


def test_rotation_invariance():
    mol, coef, q = _mol_case()
    R = wl.random_rotation(52)
    np.testing.assert_allclose(oracle.profile(mol.coords @ R.T, mol.types, coef, q),
                               oracle.profile(mol.coords, mol.types, coef, q), rtol=1e-13)


def test_translation_invariance():
    mol, coef, q = _mol_case()
    shift = np.array([1.0e4, -7.3e3, 2.9e3])
    np.testing.assert_allclose(oracle.profile(mol.coords + shift, mol.types, coef, q),
                               oracle.profile(mol.coords, mol.types, coef, q), rtol=1e-10)


def test_permutation_invariance_and_thread_count():
    mol, coef, q = _mol_case()
    p = np.random.default_rng(53).permutation(mol.n)
    I = oracle.profile(mol.coords, mol.types, coef, q, n_threads=1)
    np.testing.assert_allclose(oracle.profile(mol.coords[p], mol.types[p], coef, q), I, rtol=1e-13)
    assert np.array_equal(oracle.profile(mol.coords, mol.types, coef, q, n_threads=3), I)


def test_kappa_and_bad_type():
    mol, coef, q = _mol_case(120)
    I, kap = oracle.profile(mol.coords, mol.types, coef, q, with_kappa=True)
    assert np.all(kap >= 1.0 - 1e-12)
    assert kap[0] == pytest.approx(1.0, abs=1e-12)            # q = 0: all terms positive
    bad = mol.types.copy()
    bad[3] = 9
    with pytest.raises(ValueError):
        oracle.profile(mol.coords, bad, coef, q)


def test_golden_globule1000_regression():
    """The stored profile (written by tests/golden/make_golden.py from the oracle)
    still matches: guards the oracle and the generators against silent drift."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "globule1000_q51_profile.txt")
    ref = np.loadtxt(path)
    w = wl.c1_plain_fp64()
    np.testing.assert_array_equal(w.q, ref[:, 0])
    np.testing.assert_allclose(oracle.profile(w.mol.coords, w.mol.types, w.coef, w.q), ref[:, 1],
                               rtol=1e-14)


def _golden(name):
    import os
    return os.path.join(os.path.dirname(__file__), "golden", name)


def test_golden_per_atom_profile_vjp_and_histogram_regression():
    """The stored per-atom profile, typed and per-atom VJPs and pair histogram of a 300-atom globule
    (tests/golden/make_golden.py, from the oracle only) still match."""
    import importlib.util
    spec = importlib.util.spec_from_file_location("make_golden", _golden("make_golden.py"))
    mg = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mg)
    mol, coef, q, ff, gI = mg.small_case()
    ref = np.loadtxt(_golden("globule300_q21_atomic_profile.txt"))
    np.testing.assert_array_equal(q, ref[:, 0])
    np.testing.assert_allclose(oracle.profile_atomic(mol.coords, ff, q), ref[:, 1], rtol=1e-14)
    ref = np.loadtxt(_golden("globule300_q21_vjp.txt"))
    for got, want in ((oracle.vjp(mol.coords, mol.types, coef, q, gI), ref[:, :3]),
                      (oracle.vjp_atomic(mol.coords, ff, q, gI), ref[:, 3:])):
        np.testing.assert_allclose(got, want, rtol=0, atol=1e-12 * np.max(np.abs(want)))
    h, _ = oracle.pair_histogram(mol.coords.astype(np.float32), mol.types, 4, 64, 40.0)
    np.testing.assert_array_equal(h, np.loadtxt(_golden("globule300_hist64_r40.txt"), dtype=np.int64))
