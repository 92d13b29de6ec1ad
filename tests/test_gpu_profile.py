"""GPU parity of the Debye profile (Section I-A, Eq. 2) against the FP64 CPU oracle.

Tolerances (per q, relative to the oracle's I(q)):
  mixed precision (FP32 pair terms, FP64 reductions)  1e-5
  all-FP64 kernel                                     1e-12
Every call goes through the C ABI (libsas.so) via the ctypes binding.
"""
import functools

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
    return np.max(np.abs(np.asarray(a) - np.asarray(b)) / np.abs(np.asarray(b)))


@functools.lru_cache(maxsize=None)
def _oracle_cached(key):
    kind = key[0]
    if kind == "c1":
        w = wl.c1_plain_fp64()
        return oracle.profile(w.mol.coords, w.mol.types, w.coef, w.q)
    if kind == "c2_10k":
        w = wl.c2_globule(10000)
        return oracle.profile(w.mol.coords, w.mol.types, w.coef, w.q)
    raise KeyError(key)


def _gpu(w_mol, coef, q, precision="mixed", coords=None, **opts):
    p = Profile(coef, q, precision)
    for k, v in opts.items():
        p.set_option(getattr(_lib, "SAS_OPT_" + k.upper()), v)
    x = torch.as_tensor(w_mol.coords if coords is None else coords).cuda()
    I = p(x, torch.as_tensor(w_mol.types).cuda()).cpu().numpy()
    p.close()
    return I


# ---------------------------------------------------------------- configurations

def test_c1_fp64_kernel_matches_oracle_1e12():
    w = wl.c1_plain_fp64()
    ref = _oracle_cached(("c1",))
    I = _gpu(w.mol, w.coef, w.q, "fp64")
    assert _rel(I, ref) <= TOL_FP64


def test_c1_mixed_matches_oracle():
    w = wl.c1_plain_fp64()
    ref = _oracle_cached(("c1",))
    I = _gpu(w.mol, w.coef, w.q, "mixed", coords=w.mol.coords.astype(np.float32))
    ref32 = oracle.profile(w.mol.coords.astype(np.float32), w.mol.types, w.coef, w.q)
    assert _rel(I, ref32) <= TOL_MIXED
    assert _rel(I, ref) <= 1e-4   # float32 rounding of the input itself stays small


@pytest.mark.parametrize("step,reseed", [(2, -1), (2, 0), (2, 32), (2, 64), (4, 32), (4, 0)])
def test_c2_10k_mixed_matches_oracle(step, reseed):
    w = wl.c2_globule(10000)
    ref = _oracle_cached(("c2_10k",))
    I = _gpu(w.mol, w.coef, w.q, "mixed", step=step, reseed=reseed)
    assert _rel(I, ref) <= TOL_MIXED


@pytest.mark.parametrize("variant", [1, 2, 3, 4])
def test_c2_10k_kernel_variants_match_oracle(variant):
    w = wl.c2_globule(10000)
    ref = _oracle_cached(("c2_10k",))
    I = _gpu(w.mol, w.coef, w.q, "mixed", step=2, reseed=0, variant=variant)
    assert _rel(I, ref) <= TOL_MIXED


@pytest.mark.parametrize("case", ["c5_conformers", "c4_conformers", "n1999_q101", "n3000_q201"])
def test_automatic_reseed_rule_cases_match_oracle(case):
    """The automatic re-seed rule on both sides of its boundaries: the 2,000-atom ensemble and the
    5,000-atom refinement conformers (101 q: no re-seeding), 1,999 atoms with 101 q and 3,000 atoms
    with 201 q (re-seeded)."""
    if case == "c5_conformers":
        w = wl.c5_ensemble(n_conf=3)
        coef, q, types = w["coef"], w["q"], w["base"].types
        X = w["conformers"]
    elif case == "c4_conformers":
        w = wl.c4_refinement(batch=2)
        coef, q, types = w["coef"], w["q"], w["base"].types
        X = w["conformers"]
    else:
        n, nq = (1999, 101) if case == "n1999_q101" else (3000, 201)
        m = wl.random_walk_globule(n, 5, 90 + n).as_f32()
        coef, q, types = wl.form_factor_coefficients(5, 91), wl.q_grid(0.0, 0.5 * (nq - 1) / 100, nq), m.types
        X = m.coords[None]
    p = Profile(coef, q, "mixed")
    I = p(torch.as_tensor(X).cuda(), torch.as_tensor(types).cuda()).cpu().numpy()
    p.close()
    for b in range(X.shape[0]):
        ref = oracle.profile(X[b], types, coef, q)
        assert _rel(I[b], ref) <= TOL_MIXED, b


def _shares(mol, coef, q, world, what):
    from paper_1306_2258_gb300.shard import set_shard
    x = torch.as_tensor(mol.coords).cuda()
    t = torch.as_tensor(mol.types).cuda()
    out = []
    for rank in range(world):
        p = Profile(coef, q, "mixed")
        set_shard(p, rank, world)
        if what == "profile":
            out.append((p(x, t).cpu().numpy(), p.partials()))
        elif what == "histogram":
            out.append(p.pair_histogram(x, t)[0].cpu().numpy())
        else:
            gI = torch.as_tensor(np.linspace(1.0, 2.0, q.size)).cuda()
            out.append(p.vjp(x, t, gI).cpu().numpy().astype(np.float64))
        p.close()
    return out


@pytest.mark.parametrize("world", [1, 2, 3, 7])
def test_shards_of_one_molecule_sum_to_the_whole(world):
    """A molecule's work list split over `world` shards, run one after another on this GPU: the
    shares of I(q) and of S_ab(q) summed in rank order equal the unsplit call to rounding of the
    regrouped FP64 item sums; pair histograms add up exactly; VJP shares add up too."""
    w = wl.c2_globule(10000)
    whole = _shares(w.mol, w.coef, w.q, 1, "profile")[0]
    parts = _shares(w.mol, w.coef, w.q, world, "profile")
    I = sum(pp[0] for pp in parts)
    S = sum(pp[1] for pp in parts)
    assert np.max(np.abs(I - whole[0]) / whole[0]) <= 1e-13
    assert np.max(np.abs(S - whole[1])) <= 1e-13 * np.max(np.abs(whole[1]))
    h = sum(_shares(w.mol, w.coef, w.q, world, "histogram"))
    assert np.array_equal(h, _shares(w.mol, w.coef, w.q, 1, "histogram")[0])
    g = sum(_shares(w.mol, w.coef, w.q, world, "vjp"))
    g1 = _shares(w.mol, w.coef, w.q, 1, "vjp")[0]
    assert np.linalg.norm(g - g1) <= 1e-6 * np.linalg.norm(g1)


@pytest.mark.parametrize("precision,world", [("mixed", 2), ("mixed", 3), ("mixed", 7), ("fp64", 3)])
def test_deterministic_shards_reassemble_bit_for_bit(precision, world):
    """SAS_DETERMINISTIC: the exact sums of `world` shards of the 10,000-atom globule, run in turn on
    this GPU and added as 128-bit integers, equal the unsplit call's and assemble to its I(q) bit for
    bit; the shares of I(q) still add up to it to FP64 rounding, and it agrees with a default
    context's profile to 1e-13."""
    from paper_1306_2258_gb300.shard import add_exact, set_shard
    w = wl.c2_globule(10000)
    x = torch.as_tensor(w.mol.coords).cuda()
    t = torch.as_tensor(w.mol.types).cuda()
    p1 = Profile(w.coef, w.q, precision, deterministic=True)
    whole = p1(x, t).cpu().numpy()
    U1 = p1.exact_sums()
    Us, shares = [], []
    for rank in range(world):
        p = Profile(w.coef, w.q, precision, deterministic=True)
        set_shard(p, rank, world)
        shares.append(p(x, t).cpu().numpy())
        Us.append(p.exact_sums())
        p.close()
    U = add_exact(Us).numpy()
    assert np.array_equal(U, U1)
    assert np.array_equal(p1.assemble_exact(U).numpy()[0], whole)
    p1.close()
    assert np.max(np.abs(sum(shares) - whole) / whole) <= 1e-13
    pd = Profile(w.coef, w.q, precision)
    ref = pd(x, t).cpu().numpy()
    pd.close()
    assert np.max(np.abs(whole - ref) / ref) <= 1e-13


def test_exact_sums_need_a_deterministic_context_and_a_profile():
    w = wl.c1_plain_fp64()
    p = Profile(w.coef, w.q, "mixed")
    p(torch.as_tensor(w.mol.coords).cuda(), torch.as_tensor(w.mol.types).cuda())
    with pytest.raises(_lib.SasError) as e:
        p.exact_sums()
    assert e.value.status == _lib.SAS_ERR_UNSUPPORTED
    p.close()
    p = Profile(w.coef, w.q, "mixed", deterministic=True)
    with pytest.raises(_lib.SasError) as e:
        p.exact_sums()
    assert e.value.status == _lib.SAS_ERR_INVALID_ARG
    p.close()


def test_shard_option_validation():
    from paper_1306_2258_gb300.shard import set_shard
    w = wl.c1_plain_fp64()
    p = Profile(w.coef, w.q, "mixed")
    for bad in (0, 65536 * 2 + 2, 65536 * 3 + 5):
        with pytest.raises(_lib.SasError):
            p.set_option(_lib.SAS_OPT_SHARD, bad)
    set_shard(p, 1, 2)
    m = w.mol.as_f32()
    T = np.ones(w.q.size)
    with pytest.raises(_lib.SasError) as e:
        p.chi2_grad(torch.as_tensor(m.coords).cuda(), m.types, T, T)
    assert e.value.status == _lib.SAS_ERR_UNSUPPORTED
    p.close()


def _grid(name):
    if name == "saxs_two_steps":      # fine steps at low q, coarse beyond
        return np.concatenate([np.linspace(0.0, 0.3, 61), np.linspace(0.32, 1.0, 35)])
    if name == "waxs_0_3":            # one uniform run to 3/A, split into two passes
        return np.linspace(0.0, 3.0, 301)
    if name == "scattered":           # irregular points: runs of two
        return np.array([0.011, 0.05, 0.052, 0.2, 0.21, 0.22, 0.23, 0.5, 0.77, 0.9])
    if name == "three_runs_offset":   # three runs, none starting at q = 0
        return np.concatenate([np.linspace(0.02, 0.1, 17), np.linspace(0.11, 0.5, 14), np.linspace(0.6, 2.0, 8)])
    raise KeyError(name)


@pytest.mark.parametrize("grid", ["saxs_two_steps", "waxs_0_3", "scattered", "three_runs_offset"])
@pytest.mark.parametrize("precision,tol", [("mixed", TOL_MIXED), ("fp64", TOL_FP64)])
def test_piecewise_uniform_and_irregular_q_grids_match_oracle(grid, precision, tol):
    """q grids made of uniform runs (each run computed from its own start and step): the oracle
    takes the same q values directly."""
    q = _grid(grid)
    m = wl.random_walk_globule(2000, 5, 95)
    m32 = m.as_f32()
    coef = wl.form_factor_coefficients(5, 96)
    ref = oracle.profile(m32.coords, m32.types, coef, q)
    I = _gpu(m32, coef, q, precision)
    assert _rel(I, ref) <= tol


def test_chi2_gradient_on_a_piecewise_uniform_grid():
    q = _grid("three_runs_offset")
    base = wl.random_walk_globule(1200, 5, 97)
    coef = wl.form_factor_coefficients(5, 98)
    T = oracle.profile(wl.perturbed(base, 1.0, 99).coords, base.types, coef, q)
    w = 1.0 / T ** 2
    x = wl.perturbed(base, 1.0, 100).coords.astype(np.float32)
    p = Profile(coef, q, "mixed")
    chi2, g, _ = p.chi2_grad(torch.as_tensor(x).cuda(), base.types, T, w)
    chi2_ref, g_ref, _ = oracle.chi2_grad(x, base.types, coef, q, T, w)
    p.close()
    assert abs(float(chi2) - chi2_ref) <= 1e-4 * chi2_ref
    g = g.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(g - g_ref) <= 1e-4 * np.linalg.norm(g_ref)


def _variant_case(name):
    if name == "globule10k_q201":
        w = wl.c2_globule(10000)
        return w.mol, w.coef, w.q
    if name == "rod6k_q101":
        w = wl.c3_rod()
        return wl.subsample(w.mol, 6000, 77), w.coef, w.q
    if name == "globule3k_q300_offset":   # two q chunks, neither starting at q = 0
        m = wl.random_walk_globule(3000, 4, 78)
        return m.as_f32(), wl.form_factor_coefficients(4, 79), wl.q_grid(0.05, 1.2, 300)
    if name == "globule3k_q50_from_dq":   # q0 = dq: the start phase is the step phase t
        m = wl.random_walk_globule(3000, 4, 82)
        return m.as_f32(), wl.form_factor_coefficients(4, 83), wl.q_grid(0.02, 1.0, 50)
    if name == "globule3k_q49_from_2dq":   # q0 = 2 dq: the start phase is 2t
        m = wl.random_walk_globule(3000, 4, 84)
        return m.as_f32(), wl.form_factor_coefficients(4, 85), wl.q_grid(0.04, 1.0, 49)
    if name == "n37_q51":
        m = wl.random_walk_globule(37, 3, 80)
        return m.as_f32(), wl.form_factor_coefficients(3, 81), wl.q_grid(0.0, 0.5, 51)
    raise KeyError(name)


@pytest.mark.parametrize("name", ["globule10k_q201", "rod6k_q101", "globule3k_q300_offset", "globule3k_q50_from_dq",
                                  "globule3k_q49_from_2dq", "n37_q51"])
def test_two_pair_kernel_is_bitwise_equal_to_one_pair_kernels(name):
    """Variant 4 (two pairs per step, packed set-up) performs the same operations lane by lane and
    adds pair j before pair j+1 into every accumulator: I(q) and S_ab(q) equal bit for bit."""
    mol, coef, q = _variant_case(name)
    x = torch.as_tensor(mol.coords).cuda()
    t = torch.as_tensor(mol.types).cuda()
    out = {}
    for v in (2, 3, 4):
        p = Profile(coef, q, "mixed")
        p.set_option(_lib.SAS_OPT_RESEED, 0)
        p.set_option(_lib.SAS_OPT_VARIANT, v)
        out[v] = (p(x, t).cpu().numpy(), p.partials())
        p.close()
    for v in (3, 4):
        assert np.array_equal(out[v][0], out[2][0]), v
        assert np.array_equal(out[v][1], out[2][1]), v


def test_c2_10k_fp64_matches_oracle():
    w = wl.c2_globule(10000)
    ref = _oracle_cached(("c2_10k",))
    I = _gpu(w.mol, w.coef, w.q, "fp64")
    assert _rel(I, ref) <= TOL_FP64


def test_c2_50k_subsample_mixed_matches_oracle():
    w = wl.c2_globule(50000)
    sub = wl.subsample(w.mol, 5000, wl.seed_for(2, 5000))
    ref = oracle.profile(sub.coords, sub.types, w.coef, w.q)
    assert _rel(_gpu(sub, w.coef, w.q, "mixed"), ref) <= TOL_MIXED


def test_c2_50k_full_mixed_vs_oracle_on_sampled_q_and_vs_fp64_kernel():
    """The full 50,000-atom profile in the benchmark's configuration: the oracle
    evaluates a few sampled q values over all 1.25e9 pairs; the FP64 kernel all of them."""
    w = wl.c2_globule(50000)
    I = _gpu(w.mol, w.coef, w.q, "mixed")
    I64 = _gpu(w.mol, w.coef, w.q, "fp64")
    assert _rel(I, I64) <= TOL_MIXED
    ks = np.array([0, 37, 100, 163, 200])
    ref = oracle.profile(w.mol.coords, w.mol.types, w.coef, w.q[ks])
    assert _rel(I[ks], ref) <= TOL_MIXED
    assert _rel(I64[ks], ref) <= TOL_FP64


@pytest.mark.parametrize("which", ["rod", "sparse"])
def test_c3_subsamples_mixed_match_oracle(which):
    w = wl.c3_rod() if which == "rod" else wl.c3_sparse()
    sub = wl.subsample(w.mol, 4000, wl.seed_for(3, 40 + (which == "sparse")))
    ref = oracle.profile(sub.coords, sub.types, w.coef, w.q)
    assert _rel(_gpu(sub, w.coef, w.q, "mixed"), ref) <= TOL_MIXED
    assert _rel(_gpu(sub, w.coef, w.q, "fp64"), ref) <= TOL_FP64


# ---------------------------------------------------------------- edges and closed forms

@pytest.mark.parametrize("n", [1, 2, 3, 31, 127, 128, 129, 300])
@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_small_and_ragged_sizes(n, precision):
    mol = wl.random_walk_globule(n, 4, 100 + n).as_f32()
    mol.types[: max(1, n // 3)] = 2          # a big group, and types that may be empty or single
    coef = wl.form_factor_coefficients(4, 7)
    q = wl.q_grid(0.0, 1.0, 101)
    ref = oracle.profile(mol.coords, mol.types, coef, q)
    tol = TOL_MIXED if precision == "mixed" else TOL_FP64
    assert _rel(_gpu(mol, coef, q, precision), ref) <= tol


@pytest.mark.parametrize("precision,tol", [("mixed", TOL_MIXED), ("fp64", TOL_FP64)])
def test_maximum_types_and_q_values_with_absent_types(precision, tol):
    """SAS_MAX_TYPES = 16 types of which three never occur, and SAS_MAX_Q = 1664 q values (eight
    passes of 208)."""
    m = wl.random_walk_globule(1500, 13, 121).as_f32()
    remap = np.array([0, 1, 2, 4, 5, 6, 7, 8, 10, 11, 12, 13, 15], dtype=np.int32)   # 3, 9, 14 unused
    types = remap[m.types]
    coef = wl.form_factor_coefficients(16, 122)
    q = wl.q_grid(0.0, 2.0, _lib.SAS_MAX_Q)
    ref = oracle.profile(m.coords, types, coef, q)
    mol = wl.Molecule(m.coords, types, 16)
    assert _rel(_gpu(mol, coef, q, precision), ref) <= tol


@pytest.mark.parametrize("precision,tol", [("mixed", TOL_MIXED), ("fp64", TOL_FP64)])
def test_many_coincident_atoms(precision, tol):
    """400 atoms at one point (every pair among them has r = 0: sinc = 1) and 100 elsewhere."""
    rng = np.random.default_rng(123)
    x = np.concatenate([np.tile(np.array([[3.0, -2.0, 1.5]]), (400, 1)), rng.uniform(-20, 20, (100, 3))])
    x = x.astype(np.float32)
    types = rng.integers(0, 3, 500).astype(np.int32)
    coef = wl.form_factor_coefficients(3, 124)
    q = wl.q_grid(0.0, 0.6, 61)
    ref = oracle.profile(x, types, coef, q)
    mol = wl.Molecule(x, types, 3)
    assert _rel(_gpu(mol, coef, q, precision), ref) <= tol


def test_empty_molecule_gives_zero():
    p = Profile(wl.form_factor_coefficients(3, 1), wl.q_grid(0, 1, 11))
    I = p(torch.zeros((0, 3), device="cuda"), torch.zeros(0, dtype=torch.int32, device="cuda"))
    assert torch.all(I == 0)


@pytest.mark.parametrize("r", [0.0, 1e-7, 3.8, 100.0, 5000.0])
def test_two_atom_closed_form(r):
    coef = wl.form_factor_coefficients(2, 11)
    q = wl.q_grid(0.0, 1.0, 41)
    mol = wl.Molecule(np.array([[0.5, -1.0, 2.0], [0.5 + r, -1.0, 2.0]], np.float32), np.array([0, 1], np.int32), 2)
    f = oracle.form_factors(mol.types, coef, q)
    rr = float(np.float32(0.5 + r) - np.float32(0.5))
    x = q * rr
    s = np.where(x == 0, 1.0, np.sin(x) / np.where(x == 0, 1.0, x))
    expect = f[0] ** 2 + f[1] ** 2 + 2 * f[0] * f[1] * s
    assert _rel(_gpu(mol, coef, q, "mixed"), expect) <= TOL_MIXED
    assert _rel(_gpu(mol, coef, q, "fp64"), expect) <= TOL_FP64


def test_q_grid_not_from_zero_many_chunks_and_single_q():
    mol = wl.random_walk_globule(700, 3, 5).as_f32()
    coef = wl.form_factor_coefficients(3, 6)
    for q in (wl.q_grid(0.01, 0.5, 101), wl.q_grid(0.0, 2.0, 500), np.array([0.3])):
        ref = oracle.profile(mol.coords, mol.types, coef, q)
        assert _rel(_gpu(mol, coef, q, "mixed"), ref) <= TOL_MIXED
        assert _rel(_gpu(mol, coef, q, "fp64"), ref) <= TOL_FP64


# ---------------------------------------------------------------- invariances and API behaviour

def test_rotation_translation_permutation():
    mol = wl.random_walk_globule(2000, 5, 77)
    coef = wl.form_factor_coefficients(5, 78)
    q = wl.q_grid(0, 1, 201)
    ref = oracle.profile(mol.coords, mol.types, coef, q)
    R = wl.random_rotation(79)
    rot = wl.Molecule(mol.coords @ R.T, mol.types, 5)
    assert _rel(_gpu(rot, coef, q, "mixed", coords=rot.coords), ref) <= TOL_MIXED
    shifted = mol.coords + np.array([1.0e4, -7.0e3, 3.0e3])   # float64 input: centred before rounding
    assert _rel(_gpu(mol, coef, q, "mixed", coords=shifted), ref) <= TOL_MIXED
    assert _rel(_gpu(mol, coef, q, "fp64", coords=shifted), ref) <= 1e-10
    perm = np.random.default_rng(80).permutation(mol.n)
    pm = wl.Molecule(mol.coords[perm], mol.types[perm], 5)
    assert _rel(_gpu(pm, coef, q, "mixed", coords=pm.coords), ref) <= TOL_MIXED


def test_batch_equals_single_calls_bitwise_and_repeatable():
    w = wl.c4_refinement(n=1500, batch=4)
    p = Profile(w["coef"], w["q"])
    p.set_option(_lib.SAS_OPT_JMAX, 512)
    types = torch.as_tensor(w["base"].types).cuda()
    X = torch.as_tensor(w["conformers"]).cuda()
    Ib = p(X, types)
    Ib2 = p(X, types)
    assert torch.equal(Ib, Ib2)
    for b in range(4):
        assert torch.equal(p(X[b], types), Ib[b])
    p.close()


def test_host_and_device_buffers_agree():
    w = wl.c1_plain_fp64()
    p = Profile(w.coef, w.q)
    x32 = w.mol.coords.astype(np.float32)
    Ih = p(x32, w.mol.types)                       # host in, host out (staged)
    Id = p(torch.as_tensor(x32).cuda(), torch.as_tensor(w.mol.types).cuda()).cpu()
    assert torch.equal(Ih, Id)
    p.close()


def test_partials_match_oracle_pair_sums():
    mol = wl.random_walk_globule(1200, 3, 81).as_f32()
    coef = wl.form_factor_coefficients(3, 82)
    q = wl.q_grid(0, 1, 101)
    p = Profile(coef, q, "fp64")
    p(torch.as_tensor(mol.coords).cuda(), torch.as_tensor(mol.types).cuda())
    S = p.partials()[0]
    ref = oracle.pair_sums(mol.coords, mol.types, 3, q)
    np.testing.assert_allclose(S, ref, rtol=1e-11, atol=1e-11 * np.abs(ref).max())
    p.close()


def test_invalid_inputs_leave_output_untouched():
    mol = wl.random_walk_globule(300, 3, 83).as_f32()
    coef = wl.form_factor_coefficients(3, 84)
    q = wl.q_grid(0, 1, 21)
    p = Profile(coef, q)
    x = torch.as_tensor(mol.coords).cuda()
    t = torch.as_tensor(mol.types).cuda()
    out = torch.full((1, 21), 7.0, dtype=torch.float64, device="cuda")
    bad = x.clone()
    bad[17, 1] = float("nan")
    with pytest.raises(_lib.SasError) as e:
        _lib.sas_profile_batch(p._ctx, bad, 0, t, 300, 1, out)
    assert e.value.status == _lib.SAS_ERR_INVALID_ARG
    tb = t.clone()
    tb[5] = 3
    with pytest.raises(_lib.SasError) as e:
        _lib.sas_profile_batch(p._ctx, x, 0, tb, 300, 1, out)
    assert e.value.status == _lib.SAS_ERR_INVALID_ARG
    assert torch.all(out == 7.0)
    _lib.sas_profile_batch(p._ctx, x, 0, t, 300, 1, out)    # the context is still usable
    assert torch.all(torch.isfinite(out))
    p.close()


def test_single_type_long_group_segmented_reduction():
    """One atom type, 30,000 atoms: all items fall in one type-pair group (more than 256 of them), which
    is summed in segments of 256 items and then across segments; three sampled q against the oracle
    evaluated at those q alone."""
    mol = wl.random_walk_globule(30000, 1, 780)
    coef = wl.form_factor_coefficients(1, 781)
    q = wl.q_grid(0.0, 1.0, 201)
    p = Profile(coef, q)
    I = p(torch.as_tensor(mol.coords).cuda(), torch.as_tensor(mol.types).cuda()).cpu().numpy()
    n_items = int(p.stats()[0])
    p.close()
    assert n_items > 256
    ks = [0, 77, 190]
    ref = oracle.profile(mol.coords, mol.types, coef, q[ks])
    assert _rel(I[ks], ref) <= TOL_MIXED


def test_small_molecule_64_atom_tiles_with_ragged_and_empty_groups():
    """2,000 atoms of 16 types (one absent, one with a single atom, fourteen of ~143) at 101 q: the
    automatic two-pair form takes 64-atom tiles (groups padded to 128 would take 3,584 slots, to
    64 about 2,700); mixed against the oracle, single conformer and a batch."""
    rng = np.random.default_rng(790)
    mol = wl.random_walk_globule(2000, 16, 791).as_f32()
    t = rng.integers(0, 14, size=mol.n).astype(np.int32)
    t[7] = 14                                   # a one-atom group; type 15 stays empty
    mol.types = t
    coef = wl.form_factor_coefficients(16, 792)
    q = wl.q_grid(0.0, 0.5, 101)
    ref = oracle.profile(mol.coords, mol.types, coef, q)
    p = Profile(coef, q, "mixed")
    I1 = p(torch.as_tensor(mol.coords).cuda(), torch.as_tensor(mol.types).cuda()).cpu().numpy()
    assert p.stats()[8] == 64
    assert _rel(I1, ref) <= TOL_MIXED
    X = np.stack([wl.perturbed(mol, 0.5, 793 + b).coords for b in range(3)]).astype(np.float32)
    I = p(torch.as_tensor(X).cuda(), torch.as_tensor(mol.types).cuda()).cpu().numpy()
    assert p.stats()[8] == 64
    p.close()
    for b in range(3):
        assert _rel(I[b], oracle.profile(X[b], mol.types, coef, q)) <= TOL_MIXED


def test_profiles_repeat_bit_for_bit_on_any_context():
    """Every work item writes its own partial sums and they are added in a fixed order, so repeated
    calls give identical bits whatever order the items finish in: the mixed and FP64 direct sums,
    the quadrature method and per-atom form factors, with and without SAS_DETERMINISTIC, on a
    molecule of many more items than CTAs."""
    mol = wl.random_walk_globule(12000, 5, 431)
    coef = wl.form_factor_coefficients(5, 432)
    q = wl.q_grid(0.0, 1.0, 201)
    x = torch.as_tensor(mol.coords).cuda()
    t = torch.as_tensor(mol.types).cuda()
    ff = torch.as_tensor(wl.atomic_form_factor_table(mol.n, q, 433)).cuda()
    out = {}
    for precision, det, method in (("mixed", False, 0), ("fp64", False, 0), ("mixed", False, 2),
                                   ("mixed", True, 0)):
        p = Profile(coef, q, precision, deterministic=det)
        p.set_option(_lib.SAS_OPT_METHOD, method)
        a, b = p(x, t), p(x, t)
        assert torch.equal(a, b), (precision, det, method)
        out[(precision, det, method)] = a.cpu().numpy()
        if method == 0 and precision == "mixed" and not det:
            fa, fb = p.atomic(x, ff), p.atomic(x, ff)
            assert torch.equal(fa, fb)
        p.close()
    # the flag changes only how the items' partial sums are added (exactly)
    ref = out[("mixed", False, 0)]
    assert np.max(np.abs(out[("mixed", True, 0)] - ref) / ref) <= 1e-13
