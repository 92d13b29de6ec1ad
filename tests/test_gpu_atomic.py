"""GPU parity of the Debye profile with per-atom form factors (Section I-A, Eq. 2 without types)
against the FP64 CPU oracle, through the C ABI (sas_profile_atomic).

Tolerances (per q, relative to the oracle's I(q)): mixed precision 1e-5 (FP32 terms weighted by
FP32 form factors, FP64 reductions), all-FP64 kernel 1e-12.  q = 0 is exact up to FP64 rounding of
(sum_i f_i(0))^2.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1306_2258_gb300 import _lib, workloads as wl
from paper_1306_2258_gb300.profile import Profile

pytestmark = pytest.mark.gpu

TOL_MIXED = 1e-5
TOL_FP64 = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    _lib.load()


def _rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return np.max(np.abs(a - b) / np.abs(b))


def _run(coords, ff, q, precision="mixed", coef_types=2, **opts):
    p = Profile(wl.form_factor_coefficients(coef_types, 5), q, precision)
    for k, v in opts.items():
        p.set_option(getattr(_lib, "SAS_OPT_" + k.upper()), v)
    I = p.atomic(torch.as_tensor(coords).cuda(), torch.as_tensor(ff).cuda()).cpu().numpy()
    st = p.stats()
    p.close()
    return I, st


# n, q grid, why: small molecules run the grid in re-seed passes of 32 q; 2,500 atoms at 101 q use
# one pass of the 104-q form (J-ranges of 128); 10,000 atoms at 201 q one pass of the 208-q form
# (J-ranges of 64); 333 atoms leave a ragged last tile.
CASES = [
    (1000, (0.0, 0.5, 51), "re-seed passes, 51 q"),
    (3000, (0.0, 1.0, 201), "re-seed passes, 201 q"),
    (2500, (0.0, 0.5, 101), "one 101-q pass"),
    (10000, (0.0, 1.0, 201), "one 201-q pass"),
    (333, (0.02, 0.62, 31), "ragged tile, offset grid"),
]


@pytest.mark.parametrize("n,grid,why", CASES, ids=[c[2] for c in CASES])
def test_atomic_mixed_matches_oracle(n, grid, why):
    mol = wl.random_walk_globule(n, 1, 700 + n)
    q = wl.q_grid(*grid)
    ff = wl.atomic_form_factor_table(n, q, 800 + n)
    ref = oracle.profile_atomic(mol.coords, ff, q)
    I, st = _run(mol.coords, ff, q)
    assert _rel(I, ref) <= TOL_MIXED, why
    assert st[2] == n * (n - 1) // 2


def test_atomic_fp64_matches_oracle():
    n = 700
    mol = wl.random_walk_globule(n, 1, 711)
    q = wl.q_grid(0.0, 1.0, 61)
    ff = wl.atomic_form_factor_table(n, q, 712)
    ref = oracle.profile_atomic(mol.coords, ff, q)
    I, _ = _run(mol.coords, ff, q, precision="fp64")
    assert _rel(I, ref) <= TOL_FP64


def test_atomic_batch_host_pointers_and_f64_coords():
    """Three conformers with their own form-factor tables, host (NumPy) buffers through the C ABI,
    FP64 coordinates (centred on the device before the FP32 conversion)."""
    n, B = 517, 3
    q = wl.q_grid(0.0, 0.8, 41)
    base = wl.random_walk_globule(n, 1, 720)
    X = np.stack([wl.perturbed(base, 1.0, 721 + b).coords + 500.0 for b in range(B)])
    F = np.stack([wl.atomic_form_factor_table(n, q, 730 + b) for b in range(B)])
    p = Profile(wl.form_factor_coefficients(3, 6), q)
    out = np.full((B, q.size), np.nan)
    _lib.sas_profile_atomic(p._ctx, np.ascontiguousarray(X), _lib.SAS_COORDS_F64, n, B, np.ascontiguousarray(F), out)
    p.close()
    for b in range(B):
        ref = oracle.profile_atomic(X[b], F[b], q)
        assert _rel(out[b], ref) <= TOL_MIXED


def test_atomic_piecewise_grid():
    """A grid of two uniform runs (SAXS then WAXS spacing) is computed run by run."""
    n = 2200
    mol = wl.random_walk_globule(n, 1, 740)
    q = np.concatenate([np.linspace(0.0, 0.3, 31), np.linspace(0.35, 2.0, 34)])
    ff = wl.atomic_form_factor_table(n, q, 741)
    ref = oracle.profile_atomic(mol.coords, ff, q)
    I, _ = _run(mol.coords, ff, q)
    assert _rel(I, ref) <= TOL_MIXED


def test_atomic_types_limit_matches_typed_profile():
    """Per-atom tables built from the type form factors give the typed profile."""
    n, T = 4000, 5
    mol = wl.random_walk_globule(n, T, 750)
    coef = wl.form_factor_coefficients(T, 751)
    q = wl.q_grid(0.0, 0.5, 101)
    ff = oracle.form_factors(mol.types, coef, q).T.copy()      # [n_q, n]
    p = Profile(coef, q)
    x = torch.as_tensor(mol.coords.astype(np.float32)).cuda()
    I_typed = p(x, torch.as_tensor(mol.types).cuda()).cpu().numpy()
    I_atom = p.atomic(x, torch.as_tensor(ff).cuda()).cpu().numpy()
    p.close()
    ref = oracle.profile(mol.coords.astype(np.float32).astype(np.float64), mol.types, coef, q)
    assert _rel(I_typed, ref) <= TOL_MIXED
    assert _rel(I_atom, ref) <= TOL_MIXED


def test_atomic_small_cases_and_zero_q():
    q = np.array([0.0, 0.1, 0.37, 0.9])
    # one atom: f^2
    ff1 = np.array([[2.0], [1.5], [-0.75], [0.5]])
    I1, _ = _run(np.zeros((1, 3), np.float32), ff1, q)
    np.testing.assert_allclose(I1, ff1[:, 0] ** 2, rtol=1e-12)
    # two atoms: closed form (mixed tolerance), q = 0 exact
    r = 5.5
    X2 = np.array([[0.0, 0.0, 0.0], [r, 0.0, 0.0]], np.float32)
    ff2 = np.array([[3.0, -1.0], [2.0, 0.5], [1.0, 2.5], [-0.5, 4.0]])
    x = q * r
    sinc = np.where(x == 0, 1.0, np.sin(x) / np.where(x == 0, 1.0, x))
    expect = ff2[:, 0] ** 2 + ff2[:, 1] ** 2 + 2 * ff2[:, 0] * ff2[:, 1] * sinc
    I2, _ = _run(X2, ff2, q)
    assert _rel(I2, expect) <= TOL_MIXED
    assert I2[0] == (3.0 - 1.0) ** 2
    # coincident atoms: sinc = 1
    I3, _ = _run(np.zeros((2, 3), np.float32), ff2, q)
    assert _rel(I3, (ff2[:, 0] + ff2[:, 1]) ** 2) <= TOL_MIXED
    # no atoms
    I0, _ = _run(np.zeros((0, 3), np.float32), np.zeros((4, 0)), q)
    assert np.all(I0 == 0.0)


def test_atomic_invalid_inputs_leave_output_untouched():
    n = 300
    mol = wl.random_walk_globule(n, 1, 760)
    q = wl.q_grid(0.0, 0.5, 21)
    ff = wl.atomic_form_factor_table(n, q, 761)
    ff[7, 123] = np.nan
    p = Profile(wl.form_factor_coefficients(1, 7), q)
    out = torch.full((1, q.size), -3.0, dtype=torch.float64, device="cuda")
    x = torch.as_tensor(mol.coords.astype(np.float32)).cuda()
    with pytest.raises(_lib.SasError) as e:
        _lib.sas_profile_atomic(p._ctx, x, _lib.SAS_COORDS_F32, n, 1, torch.as_tensor(ff).cuda(), out)
    assert e.value.status == _lib.SAS_ERR_INVALID_ARG and "form factor" in e.value.message
    assert torch.all(out == -3.0)
    with pytest.raises(_lib.SasError) as e:
        _lib.sas_profile_atomic(p._ctx, x, 7, n, 1, torch.as_tensor(ff).cuda(), out)
    assert e.value.status == _lib.SAS_ERR_INVALID_ARG
    p.set_option(_lib.SAS_OPT_SHARD, 2 * 65536 + 1)
    ff[7, 123] = 1.0
    with pytest.raises(_lib.SasError) as e:
        _lib.sas_profile_atomic(p._ctx, x, _lib.SAS_COORDS_F32, n, 1, torch.as_tensor(ff).cuda(), out)
    assert e.value.status == _lib.SAS_ERR_UNSUPPORTED
    p.close()


def test_atomic_globule50k_sampled_q():
    """The 50,000-atom globule at 201 q (one 201-q pass, J-ranges of 64, the launch the benchmark
    times): every q of the GPU grid is computed, and three of them are checked against the oracle
    evaluated at those q alone; q = 0 against (sum f)^2."""
    w = wl.c2_globule(50000)
    q = w.q
    ff = wl.atomic_form_factor_table(w.mol.n, q, 770)
    I, _ = _run(w.mol.coords.astype(np.float32), ff, q)
    ks = [57, 131, 200]
    ref = oracle.profile_atomic(w.mol.coords.astype(np.float32).astype(np.float64), ff[ks], q[ks])
    assert _rel(I[ks], ref) <= TOL_MIXED
    assert abs(I[0] - np.sum(ff[0]) ** 2) <= 1e-12 * np.sum(ff[0]) ** 2


# ---------------------------------------------------------------- gradient (sas_profile_vjp_atomic)

def _grad_ok(g, ref, tol=1e-4):
    g, ref = np.asarray(g, np.float64), np.asarray(ref, np.float64)
    assert np.linalg.norm(g - ref) <= tol * np.linalg.norm(ref), np.linalg.norm(g - ref) / np.linalg.norm(ref)
    assert np.max(np.abs(g - ref)) <= tol * np.max(np.abs(ref))


@pytest.mark.parametrize("n,q_hi,n_q,batch", [(333, 0.5, 101, 1), (1500, 1.0, 201, 2), (129, 0.3, 7, 1),
                                              (2000, 0.5, 53, 1)])
def test_atomic_vjp_matches_oracle(n, q_hi, n_q, batch):
    """Per-atom form factors with a water-layer term, passes of at most 52 q (201 q: four passes, the
    last ragged; 53 q: one full pass and a single q), ragged tiles, a batch of conformers."""
    q = wl.q_grid(0.0, q_hi, n_q)
    rng = np.random.default_rng(n + n_q)
    X = np.stack([wl.random_walk_globule(n, 2, 610 + n + b).coords for b in range(batch)]).astype(np.float32)
    ff = np.stack([wl.atomic_form_factor_table(n, q, 620 + n + b) for b in range(batch)])
    gI = rng.standard_normal((batch, n_q)) / np.stack([oracle.profile_atomic(X[b], ff[b], q) for b in range(batch)])
    p = Profile(wl.form_factor_coefficients(2, 5), q)
    g = p.vjp_atomic(torch.as_tensor(X).cuda(), torch.as_tensor(ff).cuda(), torch.as_tensor(gI).cuda()).cpu().numpy()
    p.close()
    for b in range(batch):
        _grad_ok(g[b], oracle.vjp_atomic(X[b], ff[b], q, gI[b]))


def test_atomic_vjp_rigid_motion_and_types_limit():
    """Sum of the gradient and of its torques vanish (rigid motions leave I unchanged); with every
    atom's form factor equal to its type's, the per-atom VJP equals the typed one (sas_profile_vjp)."""
    mol = wl.random_walk_globule(1200, 4, 631).as_f32()
    coef = wl.form_factor_coefficients(4, 632)
    q = wl.q_grid(0.0, 0.6, 121)
    ff = oracle.form_factors(mol.types, coef, q).T.copy()   # [n_q, n]
    gI = np.random.default_rng(633).standard_normal(q.size) / oracle.profile(mol.coords, mol.types, coef, q)
    x = torch.as_tensor(mol.coords).cuda()
    p = Profile(coef, q)
    ga = p.vjp_atomic(x, torch.as_tensor(ff).cuda(), torch.as_tensor(gI).cuda()).double().cpu().numpy()
    gt = p.vjp(x, mol.types, torch.as_tensor(gI).cuda()).double().cpu().numpy()
    p.close()
    _grad_ok(ga, gt, 1e-5)
    assert np.all(np.abs(ga.sum(0)) <= 1e-4 * np.abs(ga).sum())
    tq = np.cross(mol.coords.astype(np.float64) - mol.coords.mean(0), ga)
    assert np.all(np.abs(tq.sum(0)) <= 1e-4 * np.abs(tq).sum())


def test_atomic_vjp_host_buffers_small_cases_and_unsupported_contexts():
    q = wl.q_grid(0.0, 0.5, 51)
    coef = wl.form_factor_coefficients(2, 5)
    for n in (1, 2, 3, 130):
        mol = wl.random_walk_globule(n, 2, 640 + n).as_f32()
        ff = wl.atomic_form_factor_table(n, q, 650 + n)
        gI = np.random.default_rng(n).standard_normal(q.size)
        out = np.full((1, n, 3), np.nan, np.float32)
        p = Profile(coef, q)
        _lib.sas_profile_vjp_atomic(p._ctx, mol.coords[None], n, 1, ff[None], gI[None], out)
        p.close()
        ref = oracle.vjp_atomic(mol.coords, ff, q, gI)
        if n == 1:
            assert np.all(out == 0.0)
        else:
            _grad_ok(out[0], ref)
    mol = wl.random_walk_globule(50, 2, 660).as_f32()
    ff = torch.as_tensor(wl.atomic_form_factor_table(50, q, 661)).cuda()
    gI = torch.ones(q.size, dtype=torch.float64, device="cuda")
    for kw in ({"precision": "fp64"}, {"deterministic": True}):
        p = Profile(coef, q, **kw)
        with pytest.raises(_lib.SasError) as e:
            p.vjp_atomic(torch.as_tensor(mol.coords).cuda(), ff, gI)
        assert e.value.status == _lib.SAS_ERR_UNSUPPORTED
        p.close()
    p = Profile(coef, q)
    bad = ff.clone()
    bad[3, 7] = float("nan")
    with pytest.raises(_lib.SasError) as e:
        p.vjp_atomic(torch.as_tensor(mol.coords).cuda(), bad, gI)
    assert e.value.status == _lib.SAS_ERR_INVALID_ARG
    p.close()


def test_atomic_vjp_6000_atoms_q101():
    mol = wl.random_walk_globule(6000, 2, 671).as_f32()
    q = wl.q_grid(0.0, 0.5, 101)
    ff = wl.atomic_form_factor_table(6000, q, 672)
    gI = np.random.default_rng(673).standard_normal(q.size) / oracle.profile_atomic(mol.coords, ff, q)
    p = Profile(wl.form_factor_coefficients(2, 5), q)
    g = p.vjp_atomic(torch.as_tensor(mol.coords).cuda(), torch.as_tensor(ff).cuda(), torch.as_tensor(gI).cuda())
    p.close()
    _grad_ok(g.cpu().numpy(), oracle.vjp_atomic(mol.coords, ff, q, gI))
