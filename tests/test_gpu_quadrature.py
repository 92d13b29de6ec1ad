"""GPU parity of the orientation-average method (Eq. 1 by spherical quadrature) and of the hybrid
that picks it or the direct sum per q (SAS_OPT_METHOD), and of the direct sum's re-seed rule for
molecules whose phase step M dq D approaches pi.  Tolerance: 1e-5 per q relative to the FP64
oracle of Eq. 2.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1306_2258_gb300 import _lib, workloads as wl
from paper_1306_2258_gb300.profile import Profile

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    _lib.load()


def _rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return np.max(np.abs(a - b) / np.abs(b))


def _run(mol, coef, q, method, precision="mixed", **opts):
    p = Profile(coef, q, precision)
    p.set_option(_lib.SAS_OPT_METHOD, method)
    for k, v in opts.items():
        p.set_option(getattr(_lib, "SAS_OPT_" + k.upper()), v)
    I = p(torch.as_tensor(mol.coords).cuda(), torch.as_tensor(mol.types).cuda()).cpu().numpy()
    st = p.stats()
    p.close()
    return I, st


@pytest.mark.parametrize("grid", [(0.0, 0.5, 51), (0.05, 2.0, 40)], ids=["saxs", "waxs_offset"])
def test_quadrature_every_q_matches_oracle(grid):
    mol = wl.random_walk_globule(3000, 5, 910)
    coef = wl.form_factor_coefficients(5, 911)
    q = wl.q_grid(*grid)
    ref = oracle.profile(mol.coords, mol.types, coef, q)
    I, st = _run(mol, coef, q, 2)
    assert st[6] == q.size and st[7] > 0
    assert _rel(I, ref) <= TOL


def test_hybrid_splits_and_matches_oracle_on_both_sides():
    """30,000 atoms at q <= 0.4: the low-q passes go to the quadrature, the rest to the direct sum;
    sampled q on both sides against the oracle."""
    mol = wl.random_walk_globule(30000, 5, 912)
    coef = wl.form_factor_coefficients(5, 913)
    q = wl.q_grid(0.0, 0.4, 81)
    I, st = _run(mol, coef, q, 1)
    split = int(st[6])
    assert 0 < split <= q.size
    ks = sorted({0, 5, split - 1, min(split, q.size - 1), q.size - 1})
    ref = oracle.profile(mol.coords, mol.types, coef, q[ks])
    assert _rel(I[ks], ref) <= TOL


def test_quadrature_batch_and_piecewise_grid():
    base = wl.random_walk_globule(2500, 3, 914)
    coef = wl.form_factor_coefficients(3, 915)
    q = np.concatenate([np.linspace(0.0, 0.3, 31), np.linspace(0.32, 1.0, 18)])
    X = np.stack([wl.perturbed(base, 1.0, 916 + b).coords for b in range(3)])
    p = Profile(coef, q)
    p.set_option(_lib.SAS_OPT_METHOD, 2)
    I = p(torch.as_tensor(X).cuda(), torch.as_tensor(base.types).cuda()).cpu().numpy()
    p.close()
    for b in range(3):
        ref = oracle.profile(X[b], base.types, coef, q)
        assert _rel(I[b], ref) <= TOL


def test_method_option_rules():
    mol = wl.random_walk_globule(1500, 2, 917)
    coef = wl.form_factor_coefficients(2, 918)
    q = wl.q_grid(0.0, 0.5, 21)
    p = Profile(coef, q)
    with pytest.raises(_lib.SasError) as e:
        p.set_option(_lib.SAS_OPT_METHOD, 3)
    assert e.value.status == _lib.SAS_ERR_INVALID_ARG
    p.set_option(_lib.SAS_OPT_METHOD, 1)
    p.set_option(_lib.SAS_OPT_SHARD, 2 * 65536)
    with pytest.raises(_lib.SasError) as e:
        p(torch.as_tensor(mol.coords).cuda(), torch.as_tensor(mol.types).cuda())
    assert e.value.status == _lib.SAS_ERR_UNSUPPORTED
    p.close()
    # an FP64 context always takes the direct sum
    ref = oracle.profile(mol.coords, mol.types, coef, q)
    I, st = _run(mol, coef, q, 2, precision="fp64")
    assert st[6] == 0 and _rel(I, ref) <= 1e-12


def test_direct_reseed_rule_for_ill_conditioned_phase_steps():
    """A 12,000-atom globule (diameter ~140 A) on 0..2.5/A in 201 q: the 2-step phase 2 dq D
    reaches pi, where the recurrence is ill-conditioned; the automatic rule re-seeds and the
    direct sum stays within the tolerance at high q."""
    mol = wl.random_walk_globule(12000, 5, 919)
    coef = wl.form_factor_coefficients(5, 920)
    q = wl.q_grid(0.0, 2.5, 201)
    I, _ = _run(mol, coef, q, 0)
    ks = [60, 120, 160, 199]
    ref = oracle.profile(mol.coords, mol.types, coef, q[ks])
    assert _rel(I[ks], ref) <= TOL
