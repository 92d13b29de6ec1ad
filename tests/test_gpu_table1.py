"""GPU parity on the workload of the paper's own timings (Table 1): random-walk globules of
1,000-100,000 atoms and 50-point profiles on 0 < q <= 1 A^-1 (q_k = 0.02 k), a grid that does
not start at q = 0, so every pair is seeded from its phase at the first q.

Tolerances per q as in test_gpu_profile: mixed 1e-5, FP64 1e-12 relative to the oracle's I(q).
The 100,000-atom case is the paper's largest molecule: the FP64 kernel covers all 50 q and the
oracle two sampled ones over all 5e9 pairs.
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
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b)) / np.abs(np.asarray(b))))


def _gpu(w, precision):
    p = Profile(w.coef, w.q, precision)
    try:
        dev = torch.device("cuda:0")
        return p(torch.as_tensor(w.mol.coords, device=dev), torch.as_tensor(w.mol.types, device=dev)).cpu().numpy()
    finally:
        p.close()


def test_grid_is_fifty_points_above_zero():
    w = wl.table1_globule(1000)
    assert w.q.size == 50 and w.q[0] == pytest.approx(0.02) and w.q[-1] == pytest.approx(1.0)
    assert np.allclose(np.diff(w.q), 0.02)


@pytest.mark.parametrize("n", [1000, 4000])
def test_small_globules_match_oracle_on_every_q(n):
    w = wl.table1_globule(n)
    ref = oracle.profile(w.mol.coords, w.mol.types, w.coef, w.q)
    assert _rel(_gpu(w, "mixed"), ref) <= TOL_MIXED
    assert _rel(_gpu(w, "fp64"), ref) <= TOL_FP64


def test_100k_atoms_mixed_vs_fp64_kernel_and_oracle_on_sampled_q():
    w = wl.table1_globule(100000)
    I = _gpu(w, "mixed")
    I64 = _gpu(w, "fp64")
    assert np.all(I64 > 0)
    assert _rel(I, I64) <= TOL_MIXED
    ks = np.array([0, 49])
    ref = oracle.profile(w.mol.coords, w.mol.types, w.coef, w.q[ks])
    assert _rel(I[ks], ref) <= TOL_MIXED
    assert _rel(I64[ks], ref) <= TOL_FP64


def test_coef_option_rejects_bad_values():
    w = wl.table1_globule(1000)
    p = Profile(w.coef, w.q, "mixed")
    try:
        for bad in (-1, 3):
            with pytest.raises(_lib.SasError):
                p.set_option(_lib.SAS_OPT_COEF, bad)
    finally:
        p.close()


def _with_coef(w, coef):
    p = Profile(w.coef, w.q, "mixed")
    try:
        p.set_option(_lib.SAS_OPT_COEF, coef)
        dev = torch.device("cuda:0")
        return p(torch.as_tensor(w.mol.coords, device=dev), torch.as_tensor(w.mol.types, device=dev)).cpu().numpy()
    finally:
        p.close()


def test_coefficient_forms_on_a_coarse_grid():
    """20,000 atoms on Table 1's grid: the step phase 2 dq D passes 0.8 pi, so the automatic choice
    forms the coefficient both ways (the same bits as forcing it) and holds 1e-5; the form
    2 - 4 sin^2 t alone drifts where 2t nears pi."""
    w = wl.table1_globule(20000)
    I64 = _gpu(w, "fp64")
    auto, one, both = _with_coef(w, 0), _with_coef(w, 1), _with_coef(w, 2)
    assert np.array_equal(auto, both)
    assert _rel(both, I64) <= TOL_MIXED
    assert _rel(one, I64) > _rel(both, I64)


def test_per_atom_form_factors_on_a_coarse_grid():
    """Per-atom form factors on Table 1's grid (20,000 atoms): the per-atom pair kernel forms its
    coefficient both ways too (2.4e-5 from the FP64 kernel with the one form)."""
    w = wl.table1_globule(20000)
    ff = wl.atomic_form_factor_table(w.mol.n, w.q, 771)
    dev = torch.device("cuda:0")
    x = torch.as_tensor(w.mol.coords, device=dev)
    out = {}
    for precision in ("mixed", "fp64"):
        p = Profile(w.coef, w.q, precision)
        try:
            out[precision] = p.atomic(x, torch.as_tensor(ff, device=dev)).cpu().numpy()
        finally:
            p.close()
    assert _rel(out["mixed"], out["fp64"]) <= TOL_MIXED
    ks = np.array([0, 49])
    ref = oracle.profile_atomic(w.mol.coords, ff[ks], w.q[ks])
    assert _rel(out["mixed"][ks], ref) <= TOL_MIXED
    assert _rel(out["fp64"][ks], ref) <= TOL_FP64
