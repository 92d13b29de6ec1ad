"""Pins of the FP64 MLP reference: bfloat16 rounding against torch's conversion, GELU against
known values of the normal CDF, analytic gradients against central finite differences (with
the rounding switched off so the loss is smooth), and the closed-form first Adam step."""
import math

import numpy as np
import pytest
import torch

from oracle import mlp


def test_bf16_rounding_matches_torch():
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.standard_normal(100000).astype(np.float32) * 10.0 ** rng.integers(-20, 20, 100000),
                        np.array([1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -(1.0 + 2 ** -8), 0.0, -0.0, 65504.0],
                                 np.float32)])   # exact ties round to even
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mlp.bf16(x), ref)


def test_gelu_known_values_and_derivative():
    assert mlp.gelu(np.array([0.0]))[0] == 0.0
    assert mlp.gelu(np.array([1.0]))[0] == pytest.approx(0.8413447460685429, rel=1e-15)   # Phi(1)
    assert mlp.gelu(np.array([-1.0]))[0] == pytest.approx(-1.0 + 0.8413447460685429, rel=1e-14)
    assert mlp.gelu(np.array([40.0]))[0] == 40.0
    z = np.linspace(-6, 6, 101)
    h = 1e-6
    fd = (mlp.gelu(z + h) - mlp.gelu(z - h)) / (2 * h)
    np.testing.assert_allclose(mlp.gelu_grad(z), fd, rtol=1e-7, atol=1e-9)


def _tiny(seed=3, n_in=12, h=8, n_out=5, B=7):
    rng = np.random.default_rng(seed)
    p = {"W1": rng.standard_normal((h, n_in)) * 0.5, "b1": rng.standard_normal(h) * 0.1,
         "W2": rng.standard_normal((h, h)) * 0.5, "b2": rng.standard_normal(h) * 0.1,
         "W3": rng.standard_normal((n_out, h)) * 0.5, "b3": rng.standard_normal(n_out) * 0.1}
    return p, rng.standard_normal((B, n_in)), rng.standard_normal((B, n_out))


def test_gradients_match_finite_differences(monkeypatch):
    monkeypatch.setattr(mlp, "bf16", lambda a: np.asarray(a, dtype=np.float64))
    p, x, t = _tiny()
    _, g, _ = mlp.loss_and_grads(p, x, t)
    h = 1e-6
    for k in p:
        flat = p[k].reshape(-1)
        for idx in range(0, flat.size, max(1, flat.size // 7)):
            pp = {kk: vv.copy() for kk, vv in p.items()}
            pm = {kk: vv.copy() for kk, vv in p.items()}
            pp[k].reshape(-1)[idx] += h
            pm[k].reshape(-1)[idx] -= h
            fd = (mlp.loss_and_grads(pp, x, t)[0] - mlp.loss_and_grads(pm, x, t)[0]) / (2 * h)
            assert g[k].reshape(-1)[idx] == pytest.approx(fd, rel=1e-6, abs=1e-9), (k, idx)


def test_first_adam_step_is_minus_lr_sign():
    p, x, t = _tiny(5)
    _, g, _ = mlp.loss_and_grads(p, x, t)
    m = {k: np.zeros_like(v) for k, v in p.items()}
    v = {k: np.zeros_like(v) for k, v in p.items()}
    p0 = {k: vv.copy() for k, vv in p.items()}
    p1, _, _ = mlp.adam_step({k: vv.copy() for k, vv in p.items()}, g, m, v, 1, lr=1e-3, eps=1e-8)
    for k in p:
        step = p1[k] - p0[k]
        np.testing.assert_allclose(step, -1e-3 * g[k] / (np.abs(g[k]) + 1e-8), rtol=1e-12, atol=1e-18)


def test_forward_and_gradients_match_a_float64_torch_chain(monkeypatch):
    """With the bfloat16 rounding switched off, the reference is the plain network: torch's float64
    linear / exact-erf GELU chain and its autograd gradients, at the surrogate's full width."""
    import torch.nn.functional as F
    monkeypatch.setattr(mlp, "bf16", lambda a: np.asarray(a, dtype=np.float64))
    rng = np.random.default_rng(21)
    n_in, h, n_out, B = 3840, 512, 101, 16
    p = {"W1": rng.uniform(-1, 1, (h, n_in)) * math.sqrt(3 / n_in), "b1": rng.standard_normal(h) * 0.1,
         "W2": rng.uniform(-1, 1, (h, h)) * math.sqrt(3 / h), "b2": rng.standard_normal(h) * 0.1,
         "W3": rng.uniform(-1, 1, (n_out, h)) * math.sqrt(3 / h), "b3": rng.standard_normal(n_out) * 0.1}
    x, t = rng.standard_normal((B, n_in)), rng.standard_normal((B, n_out))
    loss, g, y = mlp.loss_and_grads(p, x, t)
    tp = {k: torch.tensor(v, dtype=torch.float64, requires_grad=True) for k, v in p.items()}
    a1 = F.gelu(F.linear(torch.tensor(x), tp["W1"], tp["b1"]), approximate="none")
    a2 = F.gelu(F.linear(a1, tp["W2"], tp["b2"]), approximate="none")
    yt = F.linear(a2, tp["W3"], tp["b3"])
    lt = F.mse_loss(yt, torch.tensor(t))
    lt.backward()
    np.testing.assert_allclose(y, yt.detach().numpy(), rtol=1e-12, atol=1e-13)
    assert loss == pytest.approx(lt.item(), rel=1e-13)
    for k in p:
        np.testing.assert_allclose(g[k], tp[k].grad.numpy(), rtol=1e-10, atol=1e-16), k
