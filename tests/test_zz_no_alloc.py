"""The allocation-free profile entry point agrees with the context-based one.

sas_profile_static serves callers that may not allocate GPU memory where they need a profile
(a memory budget reserved up front, an allocator that must not be re-entered, loops where
cudaMalloc/cudaFree would synchronize the device).  Its scratch is one fixed __device__ array
shared by all calls, so this test also checks that consecutive calls on different molecules do
not see each other's leftovers, and that a call leaves the device's free memory unchanged.
The file is named so that pytest collects it last.
"""
import numpy as np
import pytest
import torch

from paper_1306_2258_gb300 import _lib, workloads as wl
from paper_1306_2258_gb300.profile import Profile

pytestmark = pytest.mark.gpu

TOL_MIXED = 1e-5


def _case(n, seed):
    mol = wl.random_walk_globule(n, 5, seed).as_f32()
    coef = wl.form_factor_coefficients(5, seed + 1)
    q = wl.q_grid(0.0, 1.0, 201)
    x = torch.as_tensor(mol.coords).cuda()
    t = torch.as_tensor(mol.types).cuda()
    p = Profile(coef, q)
    ref = p(x, t).cpu().numpy()
    p.close()
    return x, t, coef, q, ref


def _static(x, t, coef, q, out):
    _lib.sas_profile_static(x, t, x.shape[0], coef.shape[0], coef, q[0], q[1] - q[0], q.size, out)
    return out.cpu().numpy()


def test_static_profile_matches_sas_profile_on_consecutive_calls():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    big = _case(9000, 9101)      # above the re-seed threshold
    small = _case(3000, 9201)    # below it
    out = torch.full((201,), float("nan"), dtype=torch.float64, device="cuda")
    _static(*big[:4], out)       # first call on this device: set-up
    torch.cuda.synchronize()
    for x, t, coef, q, ref in (big, small, small, big):
        out.fill_(float("nan"))
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        I = _static(x, t, coef, q, out)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
        assert np.all(np.isfinite(I))
        assert np.max(np.abs(I - ref) / ref) <= TOL_MIXED


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
