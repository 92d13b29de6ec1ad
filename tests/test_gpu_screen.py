"""GPU screening kernels (sas_screen_select, sas_gather_rows) against plain NumPy: the surrogate chi^2
in FP64 (a network's log-profile, a base profile, or the base times the network's correction), the
unique (chi^2, index) order with NaN last, and the row gather."""
import numpy as np
import pytest
import torch

from paper_1306_2258_gb300 import _lib
from paper_1306_2258_gb300.surrogate import gather_conformers

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    _lib.load()


def _check_top(top, topc, chi2, ref, k):
    """The selection against the NumPy chi^2: k distinct indices holding the k smallest values, in
    ascending order with ties by index; where the reference values of neighbours differ by more than
    the kernel's rounding, exactly the reference's order; the reported values are the kernel's chi^2
    of the reported indices."""
    order = np.lexsort((np.arange(ref.size), ref))
    assert len(set(top.tolist())) == k
    np.testing.assert_allclose(ref[top], ref[order[:k]], rtol=1e-12, atol=0)
    r = ref[order[:k + 1]]
    gap = np.diff(r) > 1e-10 * np.abs(r[1:])
    decided = np.ones(k, bool)
    decided[1:] &= gap[:k - 1]
    decided &= gap[:k] if r.size > k else True
    assert np.array_equal(top[decided], order[:k][decided])
    assert np.array_equal(topc, chi2[top])


def _select(z, mean, std, target, w, k, base=None):
    d = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64)).cuda()
    n_conf, n_q = (z if z is not None else base).shape
    zt = torch.as_tensor(z).cuda() if z is not None else None
    bt = d(base) if base is not None else None
    chi2 = torch.empty(n_conf, dtype=torch.float64, device="cuda")
    top = torch.empty(k, dtype=torch.int32, device="cuda")
    topc = torch.empty(k, dtype=torch.float64, device="cuda")
    _lib.sas_screen_select(n_conf, n_q, zt, n_q, d(mean), d(std), bt, n_q, d(target), d(w), k, top, topc, chi2)
    return top.cpu().numpy(), topc.cpu().numpy(), chi2.cpu().numpy()


@pytest.mark.parametrize("n_conf,n_q,k", [(4096, 101, 205), (1, 7, 1), (1000, 51, 1000), (8192, 33, 17)])
def test_screen_select_matches_numpy(n_conf, n_q, k):
    rng = np.random.default_rng(n_conf + n_q)
    z = rng.standard_normal((n_conf, n_q)).astype(np.float32)
    mean, std = rng.uniform(2, 8, n_q), rng.uniform(0.1, 2.0, n_q)
    target = np.exp(mean + rng.standard_normal(n_q) * std)
    w = 1.0 / target ** 2
    top, topc, chi2 = _select(z, mean, std, target, w, k)
    ref = np.sum(w * (np.exp(z.astype(np.float64) * std + mean) - target) ** 2, axis=1)
    assert np.allclose(chi2, ref, rtol=1e-12, atol=0)
    _check_top(top, topc, chi2, ref, k)


@pytest.mark.parametrize("with_z", [True, False])
def test_screen_select_with_a_base_profile_matches_numpy(with_z):
    """P = base * exp(z s + m) (a correction to a base profile) and P = base alone."""
    rng = np.random.default_rng(17)
    n_conf, n_q, k = 3000, 101, 150
    base = np.exp(rng.uniform(2, 8, n_q) + 0.3 * rng.standard_normal((n_conf, n_q)))
    z = (0.05 * rng.standard_normal((n_conf, n_q))).astype(np.float32) if with_z else None
    mean, std = rng.uniform(-0.01, 0.01, n_q), rng.uniform(0.01, 0.1, n_q)
    target = base[11] * 1.01
    w = 1.0 / target ** 2
    top, topc, chi2 = _select(z, mean, std, target, w, k, base=base)
    P = base * (np.exp(z.astype(np.float64) * std + mean) if with_z else 1.0)
    ref = np.sum(w * (P - target) ** 2, axis=1)
    assert np.allclose(chi2, ref, rtol=1e-12, atol=0)
    _check_top(top, topc, chi2, ref, k)


def test_screen_select_ties_by_index_and_nan_last():
    rng = np.random.default_rng(5)
    base = rng.standard_normal((1, 20)).astype(np.float32)
    z = np.repeat(base, 300, axis=0)              # 300 identical rows: equal chi2
    z[7, 3] = np.nan                              # NaN rows rank after every number
    z[100, 0] = np.nan
    z[250] += 0.5                                 # a different row
    mean, std = np.zeros(20), np.ones(20)
    target, w = np.ones(20), np.ones(20)
    top, topc, chi2 = _select(z, mean, std, target, w, 300)
    ref = np.sum(w * (np.exp(z.astype(np.float64) * std + mean) - target) ** 2, axis=1)
    assert np.isnan(chi2[7]) and np.isnan(chi2[100])
    assert list(top[-2:]) == [7, 100]
    # 297 equal rows first (identical arithmetic gives identical chi^2: ties by index), then row 250
    fin = ~np.isnan(ref)
    assert np.allclose(chi2[fin], ref[fin], rtol=1e-12, atol=0) and ref[250] > ref[0]
    assert np.all(chi2[[i for i in range(300) if i not in (7, 100, 250)]] == chi2[0])
    assert list(top[:-2]) == [i for i in range(300) if i not in (7, 100, 250)] + [250]


def test_select_and_gather_limits():
    z = torch.zeros((2, 3), device="cuda")
    d = torch.ones(3, dtype=torch.float64, device="cuda")
    top = torch.empty(2, dtype=torch.int32, device="cuda")
    chi2 = torch.empty(2, dtype=torch.float64, device="cuda")
    b = torch.ones((2, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(_lib.SasError):   # k > n_conf
        _lib.sas_screen_select(2, 3, z, 3, d, d, None, 0, d, d, 3, top, None, chi2)
    with pytest.raises(_lib.SasError):   # host buffer
        _lib.sas_screen_select(2, 3, z, 3, d.cpu(), d, None, 0, d, d, 1, top, None, chi2)
    with pytest.raises(_lib.SasError):   # too many conformers for one CTA
        _lib.sas_screen_select(8193, 3, z, 3, d, d, None, 0, d, d, 1, top, None, chi2)
    with pytest.raises(_lib.SasError):   # neither a log-profile nor a base
        _lib.sas_screen_select(2, 3, None, 0, d, d, None, 0, d, d, 1, top, None, chi2)
    with pytest.raises(_lib.SasError):   # base row stride too short
        _lib.sas_screen_select(2, 3, None, 0, None, None, b, 2, d, d, 1, top, None, chi2)


@pytest.mark.parametrize("shape", [(50, 2000, 3), (7, 3, 3), (1, 1, 1)])
def test_gather_rows(shape):
    rng = np.random.default_rng(sum(shape))
    X = torch.as_tensor(rng.standard_normal(shape).astype(np.float32)).cuda()
    idx_np = rng.integers(0, shape[0], size=2 * shape[0]).astype(np.int32)
    out = gather_conformers(X, torch.as_tensor(idx_np).cuda())
    assert torch.equal(out, X[torch.as_tensor(idx_np, dtype=torch.long).cuda()])
