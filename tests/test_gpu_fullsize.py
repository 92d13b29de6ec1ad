"""Every benchmark row at its full size, in the launch configuration bench.py times, against the
FP64 CPU oracle on sampled outputs it can compute one at a time: sampled q values over all pairs
(rod, sparse chain), sampled conformers of a full batch (refinement gradients, ensemble profiles
and histograms).  Tolerances as elsewhere: profiles 1e-5 per q, gradients 1e-4 (norm and max),
histograms exact.
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


@pytest.mark.parametrize("which,ks", [("rod", [0, 31, 77, 100]), ("sparse", [64])])
def test_c3_full_size_on_sampled_q(which, ks):
    """The 30,000-atom rod and the 200,000-bead sparse chain in full (101 q); the oracle sums all
    pairs at the sampled q values (the sparse chain's 2e10 pairs at one q take ~25 s on 16 cores)."""
    w = wl.c3_rod() if which == "rod" else wl.c3_sparse()
    p = Profile(w.coef, w.q)
    I = p(torch.as_tensor(w.mol.coords).cuda(), torch.as_tensor(w.mol.types).cuda()).cpu().numpy()
    p.close()
    ref = oracle.profile(w.mol.coords, w.mol.types, w.coef, w.q[ks])
    assert _rel(I[ks], ref) <= TOL


def test_c4_full_batch_gradients_on_sampled_conformers():
    """chi^2 and its coordinate gradient for all 64 conformers of 5,000 atoms in one call; two of
    them against the oracle's FP64 chi^2 and gradient."""
    c4 = wl.c4_refinement()
    tt = c4["base"].types
    T = oracle.profile(c4["target"].coords.astype(np.float32).astype(np.float64), tt, c4["coef"], c4["q"])
    wq = 1.0 / T ** 2
    p = Profile(c4["coef"], c4["q"])
    chi2, g, I = p.chi2_grad(torch.as_tensor(c4["conformers"]).cuda(), tt, T, wq)
    p.close()
    assert g.shape[0] == 64
    for b in (0, 45):
        x = c4["conformers"][b]
        c_ref, g_ref, I_ref = oracle.chi2_grad(x, tt, c4["coef"], c4["q"], T, wq)
        assert _rel(I[b].cpu().numpy(), I_ref) <= TOL
        assert abs(chi2[b].item() - c_ref) <= 1e-3 * c_ref
        gg = g[b].cpu().numpy().astype(np.float64)
        assert np.linalg.norm(gg - g_ref) <= 1e-4 * np.linalg.norm(g_ref)
        assert np.max(np.abs(gg - g_ref)) <= 1e-4 * np.max(np.abs(g_ref))


def test_c5_full_ensemble_profiles_and_histograms_on_sampled_conformers():
    """Profiles and pair histograms of all 4,096 conformers of 2,000 atoms in one call each; three
    conformers against the oracle (profiles within 1e-5, histograms identical)."""
    c5 = wl.c5_ensemble()
    X = torch.as_tensor(c5["conformers"]).cuda()
    types = c5["base"].types
    p = Profile(c5["coef"], c5["q"])
    I = p(X, torch.as_tensor(types).cuda()).cpu().numpy()
    assert p.stats()[8] == 64   # five groups of ~400 atoms: 64-atom tiles
    h, d = p.pair_histogram(X, types)
    h = h.cpu().numpy()
    d = d.cpu().numpy()
    p.close()
    assert I.shape == (4096, c5["q"].size) and h.shape[0] == 4096
    for c in (0, 2047, 4095):
        x = c5["conformers"][c]
        assert _rel(I[c], oracle.profile(x, types, c5["coef"], c5["q"])) <= TOL
        hr, dr = oracle.pair_histogram(x, types, 5)
        assert int(d[c]) == dr and np.array_equal(h[c], hr)
