"""GPU binned Debye sum (sas_binned_profile) against the FP64 oracle (oracle/binned.py) on the same
integer histograms, element by element: histograms of ensemble conformers from the oracle's own
binning, seeded random counts up to 2^24 - 1 (the largest exact in FP32), batches that end in a
ragged CTA, several grids, 16 types, and a cached table reused across calls.

Tolerance: the kernel rounds each table entry to FP32 (one rounding), each product (one) and sums 32
products in FP32 before FP64 (at most 31 roundings of a partial sum), so per q
|I - I_ref| <= 40 * 2^-24 * (sum over terms of |term|).
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import binned
from paper_1306_2258_gb300 import _lib, workloads as wl
from paper_1306_2258_gb300.profile import Profile

pytestmark = pytest.mark.gpu

N_BINS, R_MAX = 256, 120.0


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    _lib.load()


def _abs_terms(hist, nt, coef, q, n_bins, r_max):
    """sum_t n_t f_t^2 + sum_p sum_k h_pk |2 f_a f_b sinc(q r_k)|: the scale of the rounding error."""
    T = coef.shape[0]
    F = oracle.form_factors(np.arange(T, dtype=np.int32), coef, q)
    r = (np.arange(n_bins) + 0.5) * (r_max / n_bins)
    x = q[:, None] * r[None, :]
    s = np.ones_like(x)
    s[x != 0] = np.abs(np.sin(x[x != 0]) / x[x != 0])
    out = np.tile(np.sum(np.asarray(nt, float)[:, None] * F * F, axis=0), (hist.shape[0], 1))
    p = 0
    for a in range(T):
        for b in range(a, T):
            out += np.abs(2 * F[a] * F[b])[None, :] * (hist[:, p, :].astype(np.float64) @ s.T)
            p += 1
    return out


def _check(hist, nt, coef, q, n_bins=N_BINS, r_max=R_MAX, prof=None, on_device=True):
    own = prof is None
    prof = prof or Profile(coef, q)
    h = torch.as_tensor(hist).cuda() if on_device else torch.as_tensor(hist)
    I = prof.binned(h, nt, n_bins, r_max).cpu().numpy()
    if own:
        prof.close()
    ref = binned.profile(hist, nt, coef, q, n_bins, r_max)
    bound = 40 * 2.0 ** -24 * _abs_terms(hist, nt, coef, q, n_bins, r_max)
    assert np.all(np.abs(I - ref) <= bound), float(np.max(np.abs(I - ref) / bound))
    return I, ref


def test_ensemble_histograms_match_oracle():
    w = wl.c5_ensemble(n_conf=21)
    types = w["base"].types
    hist = np.stack([oracle.pair_histogram(c, types, 5, N_BINS, R_MAX)[0] for c in w["conformers"]])
    I, ref = _check(hist, np.bincount(types, minlength=5), w["coef"], w["q"])
    assert np.max(np.abs(I - ref) / ref) <= 1e-5


@pytest.mark.parametrize("batch,n_q,n_bins,T", [(1, 1, 1, 1), (8, 51, 64, 3), (19, 201, 256, 5), (37, 300, 1000, 2),
                                               (9, 101, 128, 16)])
def test_random_counts_match_oracle(batch, n_q, n_bins, T):
    rng = np.random.default_rng(batch * 1000 + n_q)
    P = T * (T + 1) // 2
    hist = rng.integers(0, 2 ** 24, size=(batch, P, n_bins)).astype(np.int32)
    hist[:, :, rng.random(n_bins) < 0.3] = 0
    coef = wl.form_factor_coefficients(T, 7 + T)
    q = wl.q_grid(0.0, 1.0, n_q) if n_q > 1 else np.array([0.37])
    _check(hist, rng.integers(0, 5000, T), coef, q, n_bins, 90.0 + n_bins / 100)


def test_table_is_rebuilt_for_new_bins_and_reused_otherwise_host_buffers():
    rng = np.random.default_rng(5)
    coef = wl.form_factor_coefficients(3, 9)
    q = wl.q_grid(0.0, 0.5, 101)
    prof = Profile(coef, q)
    for n_bins, r_max, on_device in ((256, 120.0, True), (128, 60.0, False), (256, 120.0, True), (256, 100.0, False)):
        hist = rng.integers(0, 1000, size=(11, 6, n_bins)).astype(np.int32)
        _check(hist, [300, 200, 100], coef, q, n_bins, r_max, prof=prof, on_device=on_device)
    prof.close()


def test_binned_profile_rejects_bad_arguments():
    coef = wl.form_factor_coefficients(2, 1)
    prof = Profile(coef, wl.q_grid(0, 0.5, 11))
    h = torch.zeros((2, 3, 16), dtype=torch.int32, device="cuda")
    out = torch.empty((2, 11), dtype=torch.float64, device="cuda")
    for args in ((h, 2, 0, 120.0, [1, 1], out), (h, 2, 16, -1.0, [1, 1], out), (h, 2, 16, 120.0, [1, -1], out),
                 (h, -1, 16, 120.0, [1, 1], out), (None, 2, 16, 120.0, [1, 1], out)):
        with pytest.raises(_lib.SasError) as e:
            _lib.sas_binned_profile(prof._ctx, *args)
        assert e.value.status == _lib.SAS_ERR_INVALID_ARG
    prof.close()
