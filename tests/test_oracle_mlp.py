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
