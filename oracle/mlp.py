"""FP64 reference of the surrogate MLP — TEST INFRASTRUCTURE ONLY.

The network maps per-type-pair distance histograms to a standardized log I(q):
    x -> Linear(n_in, h) -> GELU -> Linear(h, h) -> GELU -> Linear(h, n_out) -> y
with the loss L = mean over batch and outputs of (y - t)^2 and Adam on FP32 master weights.

It mirrors the GPU kernels' rounding points so the two can be compared tensor by tensor: every
GEMM operand is rounded to bfloat16 (round to nearest even) exactly where the GPU rounds it,
everything else is float64 here (float32 accumulation on the GPU).  GELU is the exact erf form.
The paper has no learned part; this follows the plain definitions of each step.
"""
from __future__ import annotations

import math

import numpy as np

_erf = np.vectorize(math.erf, otypes=[np.float64])


def bf16(x) -> np.ndarray:
    """Round to bfloat16 (nearest, ties to even) the way the GPU does: the value is a float32
    there, so it is first rounded to float32, then to bfloat16; returned as float64."""
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = a.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    nan = np.isnan(a)
    out = r.astype(np.uint32).view(np.float32).astype(np.float64)
    out[nan] = np.nan
    return out


def gelu(z):
    return 0.5 * z * (1.0 + _erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + _erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


# ---- the steps, each at the GPU's rounding points (GEMM operands in bfloat16) ----

def linear(a_b, W, b):
    """z = a W^T + b for an input already rounded to bfloat16; the weight is rounded here."""
    return a_b @ bf16(W).T + b


def activation(z):
    """bfloat16(GELU(z)): the next layer's GEMM operand."""
    return bf16(gelu(z))


def mse_grad(y, t):
    """dL/dy of L = mean over batch and outputs of (y - t)^2."""
    B, Q = t.shape
    return 2.0 * (y - t) / (B * Q)


def linear_backward(dz, dz_b, a_b, W):
    """Gradients through z = a W^T + b: (dW, db, da), with dz_b = bfloat16(dz) the GEMM operand and
    the bias gradient summed from the unrounded dz."""
    return dz_b.T @ a_b, dz.sum(0), dz_b @ bf16(W)


def activation_backward(da, z):
    """dz = da GELU'(z)."""
    return da * gelu_grad(z)


def forward(params, x):
    """Returns (y, cache).  params: dict W1 [h,n_in], b1, W2 [h,h], b2, W3 [n_out,h], b3 (float32 masters)."""
    xb = bf16(x)
    z1 = linear(xb, params["W1"], params["b1"])
    a1b = activation(z1)
    z2 = linear(a1b, params["W2"], params["b2"])
    a2b = activation(z2)
    y = linear(a2b, params["W3"], params["b3"])
    return y, dict(xb=xb, z1=z1, a1b=a1b, z2=z2, a2b=a2b)


def loss_and_grads(params, x, t):
    """MSE loss and its gradients with the GPU's rounding points (GEMM operands in bfloat16)."""
    y, c = forward(params, x)
    B, Q = t.shape
    d = y - t
    loss = float(np.sum(d * d) / (B * Q))
    dy = mse_grad(y, t)
    g = {}
    g["W3"], g["b3"], da2 = linear_backward(dy, bf16(dy), c["a2b"], params["W3"])
    dz2 = activation_backward(da2, c["z2"])
    g["W2"], g["b2"], da1 = linear_backward(dz2, bf16(dz2), c["a1b"], params["W2"])
    dz1 = activation_backward(da1, c["z1"])
    g["W1"], g["b1"], _ = linear_backward(dz1, bf16(dz1), c["xb"], params["W1"])
    return loss, g, y


def adam_moments(m, v, g, beta1=0.9, beta2=0.999):
    """Adam's moment estimates after one more gradient g (element-wise, float64)."""
    return beta1 * m + (1 - beta1) * g, beta2 * v + (1 - beta2) * g ** 2


def adam_update(p, m, v, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """The parameter after step `step` (counting from 1) given the updated moments m, v."""
    mh = m / (1 - beta1 ** step)
    vh = v / (1 - beta2 ** step)
    return p - lr * mh / (np.sqrt(vh) + eps)


def adam_step(params, grads, m, v, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (bias-corrected), in place on float64 copies; `step` counts from 1."""
    for k in params:
        m[k], v[k] = adam_moments(m[k], v[k], grads[k], beta1, beta2)
        params[k] = adam_update(params[k], m[k], v[k], step, lr, beta1, beta2, eps)
    return params, m, v
