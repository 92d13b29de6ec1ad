"""Element-wise error bounds for the surrogate network's kernels against the FP64 reference
(oracle/mlp.py), shared by the GPU tests of the network.

The reference runs from scratch on a test's own inputs (parameters, batch, optimizer state); every
tensor the kernels write is compared with the reference's one element at a time, within a bound
carried through the layers:
  - GEMM outputs: the FP32 accumulation of the bfloat16 products (1e-6 of |A| |B|^T, the margin the
    tensor-core GEMM tests hold on their own), plus each operand's deviation times the other
    operand's magnitude;
  - bfloat16 roundings (activations, dY, dZ): both sides round nearly the same value; where the
    value's deviation reaches a rounding boundary they may pick neighbours, and the bound becomes
    the gap between the roundings of value - deviation and value + deviation;
  - GELU from erff (a few units of 2^-24), carried with |GELU'| <= 1.13 and |GELU''| <= 0.8;
    dY and dZ in FP32; bias sums within batch * 2^-24 * sum |terms|;
  - Adam: the moments from the gradient's deviation, the parameter from the update's variation over
    the gradient's interval plus a few FP32 roundings.
Two passes: the first carries bounds alone (every bound follows from reference values; they grow
layer by layer as the worst cases add up), the second carries each input's measured deviation once
that input has passed its own bound, so that each step is held to what its own arithmetic adds.
The reference values are the same in both.
"""
import json

import numpy as np

from oracle import mlp as ref
from paper_1306_2258_gb300 import _lib

U = 2.0 ** -24
EPS_GEMM = 1e-6
# the optimizer's constants as the kernel holds them (float32)
B1, B2, EPS = float(np.float32(0.9)), float(np.float32(0.999)), float(np.float32(1e-8))


def _gelu_slack(z):
    # 0.5 z (1 + erff(z / sqrt 2)) in FP32: erff within 2 units of its last place (2^-23 absolute
    # near -1, where 1 + erff is then exact), so 0.5 |z| 2^-23 absolute, plus a few roundings of the
    # result; taken four times over.
    return np.abs(z) * 2.0 ** -22 + np.abs(ref.gelu(z)) * 2.0 ** -20 + 1e-38


def _gelu_grad_slack(z):
    # 0.5 (1 + erff(z/sqrt 2)) + z expf(-z^2/2) / sqrt(2 pi): the first term within ~2^-23, the
    # second within a few roundings plus exp's argument error z^2/2 * 2^-24 (relative)
    phi = np.abs(z) * np.exp(-0.5 * z * z) / np.sqrt(2 * np.pi)
    return 2.0 ** -21 + phi * (2.0 ** -20 + 0.5 * z * z * 2.0 ** -22)


def _gap(v, d):
    """Largest difference between bfloat16 roundings of values within d of v (0 where it is decided)."""
    return ref.bf16(v + d) - ref.bf16(v - d)


def _mm_bound(A, DA, Bm):
    """|A' Bm^T - A Bm^T| for |A' - A| <= DA (Bm exact: a bfloat16 weight or the other operand's
    reference value with its bound folded into DA's side by the caller), plus the FP32 accumulation."""
    return DA @ np.abs(Bm).T + EPS_GEMM * ((np.abs(A) + DA) @ np.abs(Bm).T)


def _mm_bound2(A, DA, Bm, DB):
    """As _mm_bound with both operands uncertain: |A' Bm'^T - A Bm^T| for |A' - A| <= DA, |Bm' - Bm| <= DB."""
    absA, absB = np.abs(A) + DA, np.abs(Bm) + DB
    return DA @ np.abs(Bm).T + absA @ DB.T + EPS_GEMM * (absA @ absB.T)


def reference(P, x, t, got=None):
    """The reference's forward and backward from scratch, with each tensor's bound against the
    kernels' (o: values, D: bounds; G, DG: the gradients and theirs).

    Each step's bound is its own rounding error plus its inputs' deviations carried through it.  With
    got=None the deviations carried are the inputs' bounds, so every bound follows from reference
    values alone (and grows layer by layer as the worst cases add up).  With got (the kernels'
    tensors) the deviation carried is the one measured on the input, once that input has passed
    its own bound: each step is then held to what its own arithmetic can add."""
    o, D = {}, {}

    def carry(key):
        if got is None:
            return D[key]
        within(got[key], o[key], D[key], key)
        return np.abs(np.asarray(got[key], np.float64) - o[key])

    Wb = {k: ref.bf16(P["W" + k]) for k in "123"}
    o["xb"] = ref.bf16(x)
    D["xb"] = np.zeros_like(o["xb"])
    a, Da = o["xb"], carry("xb")
    for k in "12":
        z = ref.linear(a, P["W" + k], P["b" + k])
        o["z" + k], D["z" + k] = z, _mm_bound(a, Da, Wb[k]) + EPS_GEMM * np.abs(P["b" + k])
        Dz = carry("z" + k)
        g = ref.gelu(z)
        o["a" + k], D["a" + k] = ref.bf16(g), _gap(g, _gelu_slack(z) + 1.13 * Dz)
        a, Da = o["a" + k], carry("a" + k)
    y = ref.linear(a, P["W3"], P["b3"])
    o["y"], D["y"] = y, _mm_bound(a, Da, Wb["3"]) + EPS_GEMM * np.abs(P["b3"])
    dy = ref.mse_grad(y, t.astype(np.float64))
    # dY = 2 (Y - T) / (B Q) rounded once to float32: the rounding is relative to the kernel's value,
    # which may sit further from zero than the reference's by the carried deviation
    bound = 2.0 * carry("y") / t.size
    o["dy"], D["dy"] = dy, bound + 2 * U * (np.abs(dy) + bound) + 1e-45
    Ddy = carry("dy")
    o["dyb"], D["dyb"] = ref.bf16(dy), _gap(dy, Ddy)
    G, DG = {}, {}
    dz, Ddz, dzb, Ddzb = o["dy"], Ddy, o["dyb"], carry("dyb")
    for k, a_name in (("3", "a2"), ("2", "a1"), ("1", "xb")):
        a = o[a_name]
        Da = carry(a_name)
        G["W" + k], G["b" + k], da = ref.linear_backward(dz, dzb, a, P["W" + k])
        DG["W" + k] = _mm_bound2(dzb.T, Ddzb.T, a.T, Da.T)
        DG["b" + k] = Ddz.sum(0) + len(t) * U * (np.abs(dz) + Ddz).sum(0)
        if k == "1":
            break
        lo = str(int(k) - 1)
        o["da" + lo], D["da" + lo] = da, _mm_bound(dzb, Ddzb, Wb[k].T)
        Dda = carry("da" + lo)
        z = o["z" + lo]
        gp, Dgp = ref.gelu_grad(z), 0.8 * carry("z" + lo) + _gelu_grad_slack(z)
        dz = ref.activation_backward(da, z)
        bound = Dda * (np.abs(gp) + Dgp) + np.abs(da) * Dgp
        o["dz" + lo], D["dz" + lo] = dz, bound + 2 * U * (np.abs(dz) + bound) + 1e-45
        Ddz = carry("dz" + lo)
        o["dzb" + lo], D["dzb" + lo] = ref.bf16(dz), _gap(dz, Ddz)
        dzb, Ddzb = o["dzb" + lo], carry("dzb" + lo)
    if got is not None:
        for k in G:
            within(got["G_" + k], G[k], DG[k], "G_" + k)
            DG[k] = np.abs(np.asarray(got["G_" + k], np.float64) - G[k])
    return o, D, G, DG


def adam_reference(p, m, v, g, Dg, step, lr):
    """One Adam step of the reference from (p, m, v) and gradient g, with the bounds of the kernel's
    moments and parameter when its gradient lies within Dg of g."""
    m1, v1 = ref.adam_moments(m, v, g, B1, B2)
    p1 = ref.adam_update(p, m1, v1, step, lr, B1, B2, EPS)
    Dm = (1 - B1) * Dg + 3 * U * (B1 * np.abs(m) + (1 - B1) * (np.abs(g) + Dg)) + 1e-45
    Dv = (1 - B2) * (2 * np.abs(g) + Dg) * Dg + 6 * U * (B2 * np.abs(v) + (1 - B2) * (np.abs(g) + Dg) ** 2) + 1e-45
    # the update's variation over the gradient's interval (smooth and tiny there, so its values at
    # the ends and the midpoints, with half as much again), and FP32 roundings of the step
    dev = np.zeros_like(p)
    for f in (-1.0, -0.5, 0.5, 1.0):
        mm, vv = ref.adam_moments(m, v, g + f * Dg, B1, B2)
        dev = np.maximum(dev, np.abs(ref.adam_update(p, mm, vv, step, lr, B1, B2, EPS) - p1))
    Dp = 1.5 * dev + 2 * U * np.abs(p1) + 12 * U * np.abs(p1 - p) + 1e-45
    return (p1, m1, v1), (Dp, Dm, Dv)


def within(got, exact, bound, what):
    got = np.asarray(got, np.float64)
    bad = np.abs(got - exact) > bound
    assert not bad.any(), (what, int(bad.sum()), float(np.max(np.abs(got - exact) - bound)))


BUFFERS = (("xb", "XB"), ("z1", "Z1"), ("a1", "A1B"), ("z2", "Z2"), ("a2", "A2B"), ("y", "Y"), ("dy", "DY"),
           ("dyb", "DYB"), ("da2", "DA2"), ("dz2", "DZ2"), ("dzb2", "DZ2B"), ("da1", "DA1"), ("dz1", "DZ1"),
           ("dzb1", "DZ1B"))


def check_pass(net, P, x, t, g_gpu):
    got = {key: net.read_buffer(getattr(_lib, "SAS_MLP_BUF_" + buf), len(x)) for key, buf in BUFFERS}
    got.update({"G_" + k: v for k, v in net.unpack(g_gpu).items()})
    # bounds from reference values alone
    o, D, G, DG = reference(P, x, t)
    for key, _ in BUFFERS:
        within(got[key], o[key], D[key], key)
    for k in G:
        within(got["G_" + k], G[k], DG[k], "G_" + k)
    # the loss, mean (Y - T)^2 (FP64 sums of the kernel's Y, rounded to float32), within what Y's
    # bound allows
    e = np.abs(o["y"] - t)
    loss_ref = float(np.sum(e * e)) / t.size
    loss_bound = float(np.sum(2 * e * D["y"] + D["y"] ** 2)) / t.size + 2 * U * loss_ref
    # each step held to its own arithmetic (the deviation of its inputs measured, each input within
    # its bound above); the reference values are the same
    o, D, G, DG = reference(P, x, t, got)
    # how much of each bfloat16 tensor is checked exactly: its rounding is decided wherever the
    # carried deviation cannot reach a rounding boundary (D = 0), and there the kernel's value must
    # be the reference's rounding; the rest may take either neighbour
    keys = ("a1", "a2", "dyb", "dzb2", "dzb1")
    stats = {key: {"open": float(np.mean(D[key] > 0)), "differ": float(np.mean(got[key] != o[key]))} for key in keys}
    print(json.dumps({"batch": len(x), "bfloat16_roundings": stats}))
    for key in keys:
        assert stats[key]["open"] < 0.5, (key, stats[key])
    return o, G, DG, loss_ref, loss_bound


def adam_steps(net, inputs, lr, seed):
    """Adam steps from the parameters init_params(seed) and zero moments, one per (x, t) of inputs:
    before each step the reference's state (float32, the precision the network holds it in) is
    loaded into the network, so both sides start from the same values; the pass's tensors, the
    gradients, and the new parameters and moments are checked element by element."""
    p32 = net.unpack(net.init_params(seed))
    state = ({k: v.astype(np.float64) for k, v in p32.items()},
             {k: np.zeros(v.shape) for k, v in p32.items()}, {k: np.zeros(v.shape) for k, v in p32.items()})
    for step, (x, t) in enumerate(inputs, start=1):
        p, m, v = state
        net.load_state(*(net.pack(s) for s in state), step - 1)
        loss, g = net.grads(x, t)
        o, G, DG, loss_ref, loss_bound = check_pass(net, p, x, t, g)
        assert abs(loss - loss_ref) <= loss_bound, (loss, loss_ref, loss_bound)
        net.train_step(x, t, lr)
        st = net.state()
        assert st["step"] == step
        got = [net.unpack(st[k]) for k in ("params", "adam_m", "adam_v")]
        new = ({}, {}, {})
        for k in p:
            ref_k, bound_k = adam_reference(p[k], m[k], v[k], G[k], DG[k], step, lr)
            for i, what in enumerate(("param", "m", "v")):
                within(got[i][k], ref_k[i], bound_k[i], f"{what} {k} step {step}")
                new[i][k] = ref_k[i].astype(np.float32).astype(np.float64)
        state = new
