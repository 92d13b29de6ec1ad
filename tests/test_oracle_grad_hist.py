"""Pins of the oracle's gradient and histogram.

Gradient: central finite differences of the oracle's own chi^2 (a separate code
path from its analytic adjoint), and the exact translation/rotation identities
sum_i g_i = 0 and sum_i x_i x g_i = 0.
Histogram: exact rational arithmetic on half-integer lattices, edge-exact pairs,
and closed-form pair totals per type pair.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1306_2258_gb300 import workloads as wl


def _refine_case(n=60, seed=61):
    mol = wl.random_walk_globule(n, 3, seed, radius=12.0)
    coef = wl.form_factor_coefficients(3, seed + 1)
    q = wl.q_grid(0.01, 0.5, 25)
    tgt_mol = wl.perturbed(mol, 1.0, seed + 2)
    target = oracle.profile(tgt_mol.coords, mol.types, coef, q)
    w = 1.0 / target ** 2
    return mol, coef, q, target, w


def test_gradient_matches_central_differences():
    mol, coef, q, target, w = _refine_case()
    chi2, g, _ = oracle.chi2_grad(mol.coords, mol.types, coef, q, target, w)
    h = 1e-4
    rng = np.random.default_rng(62)
    picks = [(int(i), int(c)) for i, c in zip(rng.integers(0, mol.n, 48), rng.integers(0, 3, 48))]
    scale = np.max(np.abs(g))
    for i, c in picks:
        xp = mol.coords.copy(); xp[i, c] += h
        xm = mol.coords.copy(); xm[i, c] -= h
        fp = oracle.chi2_grad(xp, mol.types, coef, q, target, w, grad=False)[0]
        fm = oracle.chi2_grad(xm, mol.types, coef, q, target, w, grad=False)[0]
        fd = (fp - fm) / (2 * h)
        assert abs(fd - g[i, c]) <= 1e-6 * scale + 1e-7 * abs(g[i, c]), (i, c, fd, g[i, c])


def test_gradient_rigid_motion_identities():
    mol, coef, q, target, w = _refine_case(80, 63)
    _, g, _ = oracle.chi2_grad(mol.coords, mol.types, coef, q, target, w)
    scale = np.abs(g).sum()
    assert np.all(np.abs(g.sum(0)) <= 1e-12 * scale)
    torque = np.cross(mol.coords, g).sum(0)
    assert np.all(np.abs(torque) <= 1e-11 * np.abs(np.cross(mol.coords, g)).sum())


def test_vjp_unit_vector_is_derivative_of_one_q():
    mol, coef, q, _, _ = _refine_case(40, 64)
    k = 7
    e = np.zeros(q.size); e[k] = 1.0
    g = oracle.vjp(mol.coords, mol.types, coef, q, e)
    h = 1e-4
    for i, c in [(0, 0), (5, 1), (17, 2), (39, 0)]:
        xp = mol.coords.copy(); xp[i, c] += h
        xm = mol.coords.copy(); xm[i, c] -= h
        fd = (oracle.profile(xp, mol.types, coef, q)[k] - oracle.profile(xm, mol.types, coef, q)[k]) / (2 * h)
        assert fd == pytest.approx(g[i, c], rel=1e-6, abs=1e-6 * np.abs(g).max())


def test_gradient_zero_q_and_coincident_atoms_are_finite():
    coef = wl.form_factor_coefficients(2, 65)
    q = np.array([0.0, 0.2, 0.4])
    xyz = np.array([[0, 0, 0], [0, 0, 0], [1.5, 0, 0]], dtype=float)
    g = oracle.vjp(xyz, [0, 1, 0], coef, q, np.array([1.0, 1.0, 1.0]))
    assert np.all(np.isfinite(g))


# ---------------------------------------------------------------- histogram

def test_atomic_vjp_matches_central_differences_of_atomic_profile():
    """Per-atom form factors of either sign (a shell-like table): sum_q gI_q dI(q)/dx against
    central differences of the oracle's per-atom profile, a separate code path."""
    mol, _, q, _, _ = _refine_case(50, 65)
    ff = wl.atomic_form_factor_table(mol.n, q, 66)
    gI = np.random.default_rng(67).standard_normal(q.size)
    g = oracle.vjp_atomic(mol.coords, ff, q, gI)
    h = 1e-4
    scale = np.max(np.abs(g))
    for i, c in [(0, 0), (3, 2), (11, 1), (24, 0), (49, 2)]:
        xp = mol.coords.copy(); xp[i, c] += h
        xm = mol.coords.copy(); xm[i, c] -= h
        fd = gI @ (oracle.profile_atomic(xp, ff, q) - oracle.profile_atomic(xm, ff, q)) / (2 * h)
        assert abs(fd - g[i, c]) <= 1e-6 * scale, (i, c, fd, g[i, c])


def test_atomic_vjp_rigid_motion_and_typed_limit():
    """sum_i g_i = 0 and sum_i x_i x g_i = 0 for any per-atom table; with the table of the typed form
    factors it is the typed product."""
    mol, coef, q, _, _ = _refine_case(70, 68)
    gI = np.random.default_rng(69).standard_normal(q.size)
    g = oracle.vjp_atomic(mol.coords, wl.atomic_form_factor_table(mol.n, q, 70), q, gI)
    assert np.all(np.abs(g.sum(0)) <= 1e-12 * np.abs(g).sum())
    assert np.all(np.abs(np.cross(mol.coords, g).sum(0)) <= 1e-11 * np.abs(np.cross(mol.coords, g)).sum())
    ff_typed = oracle.form_factors(mol.types, coef, q).T          # [n, n_q] -> [n_q, n]
    np.testing.assert_allclose(oracle.vjp_atomic(mol.coords, ff_typed, q, gI),
                               oracle.vjp(mol.coords, mol.types, coef, q, gI), rtol=0, atol=1e-13)


def _exact_bin(r2: Fraction, n_bins: int, w: Fraction):
    """max{k : (k w)^2 <= r2} in exact rationals (None if >= n_bins)."""
    k = 0
    while k + 1 <= n_bins and ((k + 1) * w) ** 2 <= r2:
        k += 1
    return None if k >= n_bins else k


def test_histogram_half_integer_lattice_exact():
    rng = np.random.default_rng(71)
    ijk = rng.integers(-60, 61, size=(70, 3))
    xyz = (ijk * 0.5).astype(np.float32)              # exact in float32; r2 exact too
    types = rng.integers(0, 4, size=70).astype(np.int32)
    n_bins, r_max = 256, 120.0
    w = Fraction(15, 32)
    expect = np.zeros((10, n_bins), np.int64)
    dropped = 0
    for i in range(70):
        for j in range(i + 1, 70):
            r2 = Fraction(int(np.sum((ijk[i] - ijk[j]) ** 2)), 4)
            k = _exact_bin(r2, n_bins, w)
            if k is None:
                dropped += 1
            else:
                expect[oracle.pair_index(types[i], types[j], 4), k] += 1
    h, d = oracle.pair_histogram(xyz, types, 4, n_bins, r_max)
    assert d == dropped
    assert np.array_equal(h, expect)


def test_histogram_pairs_exactly_on_edges():
    ks = np.arange(0, 256)
    xyz = np.zeros((2 * ks.size, 3), np.float32)
    xyz[1::2, 0] = (ks * 15 / 32).astype(np.float32)    # r = e_k exactly
    xyz[0::2, 1] = 1e4 * (np.arange(ks.size) + 1)        # pairs far from each other
    xyz[1::2, 1] = 1e4 * (np.arange(ks.size) + 1)
    types = np.zeros(2 * ks.size, np.int32)
    h, d = oracle.pair_histogram(xyz, types, 1, 256, 120.0)
    assert np.array_equal(h[0], np.ones(256, np.int32))  # one pair at each edge e_k -> bin k
    n = 2 * ks.size
    assert d == n * (n - 1) // 2 - 256


def test_histogram_pair_totals():
    mol = wl.random_walk_globule(400, 5, 72).as_f32()
    h, d = oracle.pair_histogram(mol.coords, mol.types, 5)
    nt = np.bincount(mol.types, minlength=5)
    assert d == 0
    for a in range(5):
        for b in range(a, 5):
            tot = nt[a] * (nt[a] - 1) // 2 if a == b else nt[a] * nt[b]
            assert h[oracle.pair_index(a, b, 5)].sum() == tot
