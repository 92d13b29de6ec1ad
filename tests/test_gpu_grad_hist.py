"""GPU adjoint (derivative of Eq. 2) and pair histogram against the CPU oracle.

Gradient tolerances: ||g - g_ref|| <= 1e-4 ||g_ref|| and max |g - g_ref| <= 1e-4 max |g_ref|
(FP32 pair terms, FP64 accumulation).  Histogram counts must be identical.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1306_2258_gb300 import _lib, workloads as wl
from paper_1306_2258_gb300.profile import DebyeFunction, Profile

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    _lib.load()


def _grad_ok(g, ref, tol=1e-4):
    g, ref = np.asarray(g, np.float64), np.asarray(ref, np.float64)
    assert np.linalg.norm(g - ref) <= tol * np.linalg.norm(ref), np.linalg.norm(g - ref) / np.linalg.norm(ref)
    assert np.max(np.abs(g - ref)) <= tol * np.max(np.abs(ref))


def _refine_case(n=1500, batch=3, seed=401):
    base = wl.random_walk_globule(n, 5, seed)
    coef = wl.form_factor_coefficients(5, seed + 1)
    q = wl.q_grid(0.01, 0.5, 101)
    tgt = wl.perturbed(base, 1.0, seed + 2)
    T = oracle.profile(tgt.coords, base.types, coef, q)
    w = 1.0 / T ** 2
    X = np.stack([wl.perturbed(base, 1.0, seed + 10 + b).coords for b in range(batch)]).astype(np.float32)
    return base.types, coef, q, T, w, X


def test_chi2_gradient_matches_oracle_gradient():
    types, coef, q, T, w, X = _refine_case()
    p = Profile(coef, q)
    chi2, g, I = p.chi2_grad(torch.as_tensor(X).cuda(), types, T, w)
    for b in range(X.shape[0]):
        c_ref, g_ref, I_ref = oracle.chi2_grad(X[b], types, coef, q, T, w)
        assert np.max(np.abs(I[b].cpu().numpy() - I_ref) / I_ref) <= 1e-5
        assert abs(chi2[b].item() - c_ref) <= 1e-3 * c_ref
        _grad_ok(g[b].cpu().numpy(), g_ref)
    p.close()


def test_gradient_matches_central_differences_of_fp64_chi2():
    types, coef, q, T, w, X = _refine_case(n=800, batch=1, seed=411)
    x = X[0].astype(np.float64)
    p = Profile(coef, q)
    _, g, _ = p.chi2_grad(torch.as_tensor(X).cuda(), types, T, w)
    g = g[0].cpu().numpy()
    p64 = Profile(coef, q, "fp64")
    tt = torch.as_tensor(types).cuda()

    def chi2(xx):
        I = p64(torch.as_tensor(xx).cuda(), tt).cpu().numpy()
        return float(np.sum(w * (I - T) ** 2))

    h = 1e-4
    rng = np.random.default_rng(412)
    idx = list(zip(rng.integers(0, x.shape[0], 48), rng.integers(0, 3, 48)))
    fd, an = [], []
    for i, c in idx:
        xp = x.copy(); xp[i, c] += h
        xm = x.copy(); xm[i, c] -= h
        fd.append((chi2(xp) - chi2(xm)) / (2 * h))
        an.append(g[i, c])
    fd, an = np.array(fd), np.array(an)
    assert np.linalg.norm(an - fd) <= 1e-4 * np.linalg.norm(fd)
    p.close()
    p64.close()


def test_gradient_rigid_motion_identities():
    types, coef, q, T, w, X = _refine_case(n=1200, batch=2, seed=421)
    p = Profile(coef, q)
    _, g, _ = p.chi2_grad(torch.as_tensor(X).cuda(), types, T, w)
    for b in range(2):
        gb = g[b].double().cpu().numpy()
        xb = X[b].astype(np.float64)
        assert np.all(np.abs(gb.sum(0)) <= 1e-4 * np.abs(gb).sum())
        tq = np.cross(xb - xb.mean(0), gb)
        assert np.all(np.abs(tq.sum(0)) <= 1e-4 * np.abs(tq).sum())
    p.close()


def test_autograd_vjp_matches_oracle():
    mol = wl.random_walk_globule(900, 4, 431).as_f32()
    coef = wl.form_factor_coefficients(4, 432)
    q = wl.q_grid(0.0, 0.8, 161)
    p = Profile(coef, q)
    x = torch.as_tensor(mol.coords).cuda().requires_grad_(True)
    v = np.random.default_rng(433).standard_normal(q.size) / oracle.profile(mol.coords, mol.types, coef, q)
    I = DebyeFunction.apply(x, p, torch.as_tensor(mol.types).cuda())
    (I * torch.as_tensor(v).cuda()).sum().backward()
    ref = oracle.vjp(mol.coords, mol.types, coef, q, v)
    _grad_ok(x.grad.cpu().numpy(), ref)
    p.close()


def test_vjp_batch_host_buffers():
    types, coef, q, T, w, X = _refine_case(n=700, batch=2, seed=441)
    p = Profile(coef, q)
    gI = np.random.default_rng(442).standard_normal((2, q.size)) / T
    out = np.empty((2, 700, 3), np.float32)
    _lib.sas_profile_vjp(p._ctx, X, types.astype(np.int32), 700, 2, gI, out)
    for b in range(2):
        _grad_ok(out[b], oracle.vjp(X[b], types, coef, q, gI[b]))
    p.close()


# ---------------------------------------------------------------- histogram

@pytest.mark.parametrize("n,batch,seed", [(1500, 3, 421), (6000, 1, 423)])
def test_deterministic_context_repeats_gradients_bit_for_bit(n, batch, seed):
    """SAS_DETERMINISTIC: chi^2, gradient, profile and VJP identical bit for bit over repeated calls
    (the 6,000-atom case has J-ranges of several I-tiles, so an atom's totals come from many items),
    the gradient within the oracle tolerance, and the VJP within 1e-5 of the default context's."""
    types, coef, q, T, w, X = _refine_case(n=n, batch=batch, seed=seed)
    x = torch.as_tensor(X).cuda()
    gI = torch.as_tensor(np.random.default_rng(seed).standard_normal((batch, q.size))).cuda()
    p = Profile(coef, q, deterministic=True)
    runs = [p.chi2_grad(x, types, T, w) for _ in range(3)]
    vj = [p.vjp(x, types, gI) for _ in range(3)]
    p.close()
    for c, g, I in runs[1:]:
        assert torch.equal(c, runs[0][0]) and torch.equal(g, runs[0][1]) and torch.equal(I, runs[0][2])
    for v in vj[1:]:
        assert torch.equal(v, vj[0])
    c_ref, g_ref, I_ref = oracle.chi2_grad(X[0], types, coef, q, T, w)
    assert np.max(np.abs(runs[0][2][0].cpu().numpy() - I_ref) / I_ref) <= 1e-5
    assert abs(runs[0][0][0].item() - c_ref) <= 1e-3 * c_ref
    _grad_ok(runs[0][1][0].cpu().numpy(), g_ref)
    p0 = Profile(coef, q)
    v0 = p0.vjp(x, types, gI)
    p0.close()
    for b in range(batch):
        _grad_ok(vj[0][b].cpu().numpy(), v0[b].cpu().numpy(), 1e-5)


@pytest.mark.parametrize("n,seed,T", [(2000, 501, 5), (129, 502, 3), (1, 503, 2), (3000, 504, 1), (2500, 505, 16)])
def test_histogram_exact(n, seed, T):
    mol = wl.random_walk_globule(n, T, seed).as_f32()
    p = Profile(wl.form_factor_coefficients(T, 1), wl.q_grid(0, 0.5, 11))
    h, d = p.pair_histogram(torch.as_tensor(mol.coords).cuda(), mol.types)
    hr, dr = oracle.pair_histogram(mol.coords, mol.types, T)
    assert int(d) == dr
    assert np.array_equal(h.cpu().numpy(), hr)
    p.close()


def test_histogram_lattice_edges_and_drops_exact():
    rng = np.random.default_rng(511)
    ijk = rng.integers(-150, 151, size=(800, 3))
    xyz = (ijk * 0.5).astype(np.float32)          # exact; includes pairs on bin edges and beyond 120 A
    types = rng.integers(0, 4, size=800).astype(np.int32)
    p = Profile(wl.form_factor_coefficients(4, 1), wl.q_grid(0, 0.5, 11))
    for nb, rmax in [(256, 120.0), (100, 50.0)]:
        h, d = p.pair_histogram(torch.as_tensor(xyz).cuda(), types, n_bins=nb, r_max=rmax)
        hr, dr = oracle.pair_histogram(xyz, types, 4, nb, rmax)
        assert int(d) == dr and dr > 0
        assert np.array_equal(h.cpu().numpy(), hr)
    p.close()


def test_histogram_batch_of_conformers():
    w = wl.c5_ensemble(n_conf=6, n=2000)
    p = Profile(w["coef"], w["q"])
    h, d = p.pair_histogram(torch.as_tensor(w["conformers"]).cuda(), w["base"].types)
    for c in range(6):
        hr, dr = oracle.pair_histogram(w["conformers"][c], w["base"].types, 5)
        assert int(d[c]) == dr
        assert np.array_equal(h[c].cpu().numpy(), hr)
    p.close()
