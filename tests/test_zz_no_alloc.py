"""The allocation-free profile entry point agrees with the context-based one and with the oracle.

sas_profile_static serves callers that may not allocate GPU memory where they need a profile
(a memory budget reserved up front, an allocator that must not be re-entered, loops where
cudaMalloc/cudaFree would synchronize the device).  Its scratch is one fixed __device__ array
shared by all calls, so this test also checks that consecutive calls on different molecules do
not see each other's leftovers (including after a call that failed validation part-way), that
the largest accepted molecule fits, and that a call leaves the device's free memory unchanged.
The file is named so that pytest collects it last.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1306_2258_gb300 import _lib, workloads as wl
from paper_1306_2258_gb300.profile import Profile

pytestmark = pytest.mark.gpu

TOL_MIXED = 1e-5


def _case(n, seed, n_types=5, n_q=201, types=None):
    mol = wl.random_walk_globule(n, n_types, seed).as_f32()
    if types is not None:
        mol.types = types
    coef = wl.form_factor_coefficients(n_types, seed + 1)
    q = wl.q_grid(0.0, 1.0 * (n_q - 1) / 200, n_q)
    x = torch.as_tensor(mol.coords).cuda()
    t = torch.as_tensor(mol.types).cuda()
    p = Profile(coef, q)
    ref = p(x, t).cpu().numpy()
    p.close()
    return x, t, coef, q, ref, mol


def _static(x, t, coef, q, out):
    _lib.sas_profile_static(x, t, x.shape[0], coef.shape[0], coef, q[0], q[1] - q[0], q.size, out)
    return out.cpu().numpy()


def _rel(a, b):
    return float(np.max(np.abs(a - b) / np.abs(b)))


def test_static_profile_matches_sas_profile_and_oracle_on_consecutive_calls():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    big = _case(9000, 9101)      # above the re-seed threshold
    small = _case(3000, 9201)    # below it
    out = torch.full((201,), float("nan"), dtype=torch.float64, device="cuda")
    _static(*big[:4], out)       # first call on this device: set-up
    torch.cuda.synchronize()
    ref_small = oracle.profile(small[5].coords, small[5].types, small[2], small[3])
    ks = np.array([0, 41, 117, 200])
    ref_big = oracle.profile(big[5].coords, big[5].types, big[2], big[3][ks])
    for x, t, coef, q, ref, mol in (big, small, small, big):
        out.fill_(float("nan"))
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        I = _static(x, t, coef, q, out)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
        assert np.all(np.isfinite(I))
        assert _rel(I, ref) <= TOL_MIXED
        if mol.n == 3000:
            assert _rel(I, ref_small) <= TOL_MIXED
        else:
            assert _rel(I[ks], ref_big) <= TOL_MIXED


def test_static_profile_at_its_size_limit_with_16_types_and_single_atom_types():
    """SAS_STATIC_MAX_ATOMS atoms, 16 types (three of them with one atom, so that 16 groups pad to
    whole tiles), 208 q: the largest padding and work list the fixed regions were sized for."""
    n = 16384
    rng = np.random.default_rng(9301)
    types = rng.integers(0, 13, size=n).astype(np.int32)
    types[[5, 777, 16000]] = [13, 14, 15]
    x, t, coef, q, ref, mol = _case(n, 9302, n_types=16, n_q=208, types=types)
    out = torch.full((208,), float("nan"), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    I = _static(x, t, coef, q, out)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert _rel(I, ref) <= TOL_MIXED
    ks = np.array([0, 99, 207])
    assert _rel(I[ks], oracle.profile(mol.coords, mol.types, coef, q[ks])) <= TOL_MIXED


def test_static_profile_empty_molecule_bad_type_and_recovery():
    """n = 0 gives zeros; a type out of range is rejected after the validation kernel has written
    the shared array; the next valid call still gives sas_profile's result."""
    x, t, coef, q, ref, mol = _case(2500, 9401)
    out = torch.full((201,), float("nan"), dtype=torch.float64, device="cuda")
    I0 = _static(x[:0], t[:0], coef, q, out)
    assert np.all(I0 == 0.0)
    bad = t.clone()
    bad[1234] = 5
    out.fill_(7.0)
    with pytest.raises(_lib.SasError) as e:
        _static(x, bad, coef, q, out)
    assert e.value.status == _lib.SAS_ERR_INVALID_ARG
    assert np.all(out.cpu().numpy() == 7.0)
    assert _rel(_static(x, t, coef, q, out), ref) <= TOL_MIXED


def test_static_profile_rejects_oversize_and_host_buffers():
    _lib.load()
    coef = wl.form_factor_coefficients(2, 1)
    out = torch.empty(11, dtype=torch.float64, device="cuda")
    x = torch.zeros((16385, 3), dtype=torch.float32, device="cuda")
    t = torch.zeros(16385, dtype=torch.int32, device="cuda")
    with pytest.raises(_lib.SasError) as e:
        _lib.sas_profile_static(x, t, 16385, 2, coef, 0.0, 0.1, 11, out)
    assert e.value.status == _lib.SAS_ERR_UNSUPPORTED
    with pytest.raises(_lib.SasError) as e:
        _lib.sas_profile_static(x[:10], t[:10], 10, 2, coef, 0.0, 0.1, 209, out)
    assert e.value.status == _lib.SAS_ERR_UNSUPPORTED
    with pytest.raises(_lib.SasError) as e:
        _lib.sas_profile_static(x[:10].cpu(), t[:10], 10, 2, coef, 0.0, 0.1, 11, out)
    assert e.value.status == _lib.SAS_ERR_INVALID_ARG
