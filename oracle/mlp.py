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


def forward(params, x):
    """Returns (y, cache).  params: dict W1 [h,n_in], b1, W2 [h,h], b2, W3 [n_out,h], b3 (float32 masters)."""
    xb = bf16(x)
    z1 = xb @ bf16(params["W1"]).T + params["b1"]
    a1 = gelu(z1)
    a1b = bf16(a1)
    z2 = a1b @ bf16(params["W2"]).T + params["b2"]
    a2 = gelu(z2)
    a2b = bf16(a2)
    y = a2b @ bf16(params["W3"]).T + params["b3"]
    return y, dict(xb=xb, z1=z1, a1b=a1b, z2=z2, a2b=a2b)


def loss_and_grads(params, x, t):
    """MSE loss and its gradients with the GPU's rounding points (GEMM operands in bfloat16)."""
    y, c = forward(params, x)
    B, Q = t.shape
    d = y - t
    loss = float(np.sum(d * d) / (B * Q))
    dy = 2.0 * d / (B * Q)
    dyb = bf16(dy)
    g = {}
    g["W3"] = dyb.T @ c["a2b"]
    g["b3"] = dy.sum(0)
    da2 = dyb @ bf16(params["W3"])
    dz2 = da2 * gelu_grad(c["z2"])
    dz2b = bf16(dz2)
    g["W2"] = dz2b.T @ c["a1b"]
    g["b2"] = dz2.sum(0)
    da1 = dz2b @ bf16(params["W2"])
    dz1 = da1 * gelu_grad(c["z1"])
    dz1b = bf16(dz1)
    g["W1"] = dz1b.T @ c["xb"]
    g["b1"] = dz1.sum(0)
    return loss, g, y


def adam_step(params, grads, m, v, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (bias-corrected), in place on float64 copies; `step` counts from 1."""
    for k in params:
        m[k] = beta1 * m[k] + (1 - beta1) * grads[k]
        v[k] = beta2 * v[k] + (1 - beta2) * grads[k] ** 2
        mh = m[k] / (1 - beta1 ** step)
        vh = v[k] / (1 - beta2 ** step)
        params[k] = params[k] - lr * mh / (np.sqrt(vh) + eps)
    return params, m, v
