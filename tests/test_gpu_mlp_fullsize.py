"""Element-by-element parity of the surrogate network at the size the benchmark trains it:
3840 -> 512 -> 512 -> 101 at batch 256 (the tcgen05 GEMMs' deep-ring tiles, the fused GELU and
bfloat16 epilogues, the transposed operands of the weight and input gradients).

Every tensor the kernels write is compared with the FP64 reference (oracle/mlp.py) one element at a
time, each step fed the GPU's own inputs to that step, so that a rounding decision taken on one
side near a bfloat16 midpoint does not spread into the next layer:
  - GEMM outputs: |got - exact| <= 1e-6 * (|A| |B|^T + |bias|), the product of the same bfloat16
    operands accumulated in FP64 (FP32 accumulation over K <= 3840 products);
  - bfloat16 roundings (activations, dY, dZ): equal to the reference's rounding of the FP64 value
    wherever that rounding is decided by the value give or take the FP32 error of the kernel's
    value (GELU from erff, expf: a few units of 2^-24); elsewhere one of the two neighbours;
  - element-wise FP32 steps (dY, GELU'): the FP64 value within their FP32 error;
  - bias gradients (FP32 column sums over the batch): within batch * 2^-24 * sum |terms|;
  - two Adam steps: m, v and the masters within a few FP32 roundings of the FP64 update.
The end-to-end forward of the reference (its own roundings throughout) is compared as well, with a
bound that propagates the undecided roundings of each layer through the next.
"""
import numpy as np
import pytest
import torch

from oracle import mlp as ref
from paper_1306_2258_gb300 import _lib
from paper_1306_2258_gb300.surrogate import SurrogateMLP

pytestmark = pytest.mark.gpu

N_IN, H, N_OUT, B = 3840, 512, 101, 256
U = 2.0 ** -24
LR = 1e-3
# the optimizer's constants as the kernel holds them (float32)
B1, B2, EPS = float(np.float32(0.9)), float(np.float32(0.999)), float(np.float32(1e-8))


@pytest.fixture(scope="module")
def net():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    _lib.load()
    n = SurrogateMLP(N_IN, H, N_OUT, max_batch=B, seed=31)
    yield n
    n.close()


def _inputs(seed):
    """Standardized-feature-like inputs: unit normal, a fifth of the columns constant (zero after
    standardization), a few heavy columns; unit-normal targets."""
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((B, N_IN))
    x[:, rng.random(N_IN) < 0.2] = 0.0
    x[:, rng.random(N_IN) < 0.05] *= 6.0
    t = rng.standard_normal((B, N_OUT))
    return x.astype(np.float32), t.astype(np.float32)


def _gemm(got, exact, mag, what):
    bound = 1e-6 * mag + 1e-30
    bad = np.abs(got - exact) > bound
    assert not bad.any(), (what, int(bad.sum()), float(np.max(np.abs(got - exact) / bound)))


def _within(got, exact, bound, what):
    bad = np.abs(got - exact) > bound
    assert not bad.any(), (what, int(bad.sum()), float(np.max(np.abs(got - exact) - bound)))


def _rounded(got_b, value, slack, what):
    """got_b = bfloat16(v) for the kernel's FP32 v within `slack` of the FP64 `value`: it lies between
    the reference's roundings of value - slack and value + slack (equal to both where they agree)."""
    lo, hi = ref.bf16(value - slack), ref.bf16(value + slack)
    bad = (got_b < lo) | (got_b > hi)
    assert not bad.any(), (what, int(bad.sum()))
    assert np.mean(lo != hi) < 3e-2, what      # the decision is open for only a few elements
    return lo, hi


def _gelu_slack(z):
    # 0.5 z (1 + erff(z / sqrt 2)) in FP32: erff within 2 units of its last place (2^-23 absolute
    # near -1, where 1 + erff is then exact), so 0.5 |z| 2^-23 absolute, plus a few roundings of the
    # result; taken four times over.  Strongly negative z (tiny GELU) leaves the rounding open.
    return np.abs(z) * 2.0 ** -22 + np.abs(ref.gelu(z)) * 2.0 ** -20 + 1e-38


def _gelu_grad_slack(z):
    # 0.5 (1 + erff(z/sqrt 2)) + z expf(-z^2/2) / sqrt(2 pi): the first term within ~2^-23, the
    # second within a few roundings plus exp's argument error z^2/2 * 2^-24 (relative)
    phi = np.abs(z) * np.exp(-0.5 * z * z) / np.sqrt(2 * np.pi)
    return 2.0 ** -21 + phi * (2.0 ** -20 + 0.5 * z * z * 2.0 ** -22)


def _check_forward_and_backward(net, params, x, t):
    P = {k: v.astype(np.float64) for k, v in net.unpack(params).items()}
    rd = lambda which: net.read_buffer(which, B).astype(np.float64)
    xb, z1, a1b, z2, a2b, y = (rd(w) for w in (_lib.SAS_MLP_BUF_XB, _lib.SAS_MLP_BUF_Z1, _lib.SAS_MLP_BUF_A1B,
                                                _lib.SAS_MLP_BUF_Z2, _lib.SAS_MLP_BUF_A2B, _lib.SAS_MLP_BUF_Y))
    assert np.array_equal(xb, ref.bf16(x))
    W1b, W2b, W3b = ref.bf16(P["W1"]), ref.bf16(P["W2"]), ref.bf16(P["W3"])
    # forward, each layer from the GPU's own operands
    for got, a, Wb, name in ((z1, xb, W1b, "1"), (z2, a1b, W2b, "2"), (y, a2b, W3b, "3")):
        _gemm(got, ref.linear(a, P["W" + name], P["b" + name]), np.abs(a) @ np.abs(Wb).T + np.abs(P["b" + name]),
              "Z" + name if name != "3" else "Y")
    for got_b, z, name in ((a1b, z1, "A1B"), (a2b, z2, "A2B")):
        _rounded(got_b, ref.gelu(z), _gelu_slack(z), name)
    # backward
    dy, dyb, da2, dz2, dz2b, da1, dz1, dz1b = (rd(w) for w in (
        _lib.SAS_MLP_BUF_DY, _lib.SAS_MLP_BUF_DYB, _lib.SAS_MLP_BUF_DA2, _lib.SAS_MLP_BUF_DZ2,
        _lib.SAS_MLP_BUF_DZ2B, _lib.SAS_MLP_BUF_DA1, _lib.SAS_MLP_BUF_DZ1, _lib.SAS_MLP_BUF_DZ1B))
    dy_ref = ref.mse_grad(y, t.astype(np.float64))
    _within(dy, dy_ref, np.abs(dy_ref) * 2 * U + 1e-45, "DY")
    assert np.array_equal(dyb, ref.bf16(dy))
    for dz, dzb, da, z, name in ((dz2, dz2b, da2, z2, "DZ2"), (dz1, dz1b, da1, z1, "DZ1")):
        exact = ref.activation_backward(da, z)
        _within(dz, exact, np.abs(da) * _gelu_grad_slack(z) + np.abs(exact) * 2 * U + 1e-45, name)
        assert np.array_equal(dzb, ref.bf16(dz)), name + "B"
    return dict(xb=xb, a1b=a1b, a2b=a2b, y=y, dy=dy, dyb=dyb, da2=da2, dz2=dz2, dz2b=dz2b, da1=da1, dz1=dz1,
                dz1b=dz1b, P=P, W2b=W2b, W3b=W3b)


def _check_gradients(net, g, c):
    G = {k: v.astype(np.float64) for k, v in net.unpack(g).items()}
    for dz, dzb, a_b, name, da_next in ((c["dy"], c["dyb"], c["a2b"], "3", c["da2"]),
                                        (c["dz2"], c["dz2b"], c["a1b"], "2", c["da1"]),
                                        (c["dz1"], c["dz1b"], c["xb"], "1", None)):
        dW, db, da = ref.linear_backward(dz, dzb, a_b, c["P"]["W" + name])
        _gemm(G["W" + name], dW, np.abs(dzb).T @ np.abs(a_b), "G_W" + name)
        _within(G["b" + name], db, B * U * np.abs(dz).sum(0) + 1e-45, "G_b" + name)
        if da_next is not None:
            _gemm(da_next, da, np.abs(dzb) @ np.abs(ref.bf16(c["P"]["W" + name])), "DA" + str(int(name) - 1))
    return G


def _end_to_end_bound(c, x):
    """|y_gpu - y_ref| bound: the reference's forward from scratch differs from the GPU's only through
    roundings to bfloat16 that neither side decides (value within the FP32 error of a midpoint) and
    FP32 accumulation; propagate both through each layer with magnitudes."""
    P = c["P"]
    xb = ref.bf16(x)
    W1b, W2b, W3b = ref.bf16(P["W1"]), c["W2b"], c["W3b"]
    z1 = ref.linear(xb, P["W1"], P["b1"])
    dz1 = 1e-6 * (np.abs(xb) @ np.abs(W1b).T + np.abs(P["b1"]))
    g1 = ref.gelu(z1)
    s1 = _gelu_slack(z1) + 1.13 * dz1                   # |GELU'| <= 1.13
    d1 = np.abs(ref.bf16(g1 + s1) - ref.bf16(g1 - s1))
    a1 = ref.bf16(g1)
    z2 = ref.linear(a1, P["W2"], P["b2"])
    dz2 = d1 @ np.abs(W2b).T + 1e-6 * ((np.abs(a1) + d1) @ np.abs(W2b).T + np.abs(P["b2"]))
    g2 = ref.gelu(z2)
    s2 = _gelu_slack(z2) + 1.13 * dz2
    d2 = np.abs(ref.bf16(g2 + s2) - ref.bf16(g2 - s2))
    a2 = ref.bf16(g2)
    y = ref.linear(a2, P["W3"], P["b3"])
    dy = d2 @ np.abs(W3b).T + 1e-6 * ((np.abs(a2) + d2) @ np.abs(W3b).T + np.abs(P["b3"]))
    return y, dy


def _check_adam(before, after, G, step):
    """Moments from the GPU's previous moments and gradient; the parameter from the GPU's previous
    parameter and new moments (each FP32 step within a few roundings of its FP64 value)."""
    p, m, v = ({k: vv.astype(np.float64) for k, vv in d.items()} for d in before)
    pa, ma, va = ({k: vv.astype(np.float64) for k, vv in d.items()} for d in after)
    for k in p:
        m_ref, v_ref = ref.adam_moments(m[k], v[k], G[k], B1, B2)
        _within(ma[k], m_ref, 3 * U * (B1 * np.abs(m[k]) + (1 - B1) * np.abs(G[k])) + 1e-45, f"m {k} step {step}")
        _within(va[k], v_ref, np.abs(v_ref) * 6 * U + 1e-45, f"v {k} step {step}")
        p_ref = ref.adam_update(p[k], ma[k], va[k], step, LR, B1, B2, EPS)
        _within(pa[k], p_ref, np.abs(p_ref) * 2 * U + 12 * U * np.abs(p_ref - p[k]) + 1e-45,
                f"param {k} step {step}")


def test_full_size_forward_backward_and_two_adam_steps_element_by_element(net):
    x, t = _inputs(41)
    for step in (1, 2):
        st = net.state()
        before = tuple(net.unpack(st[k]) for k in ("params", "adam_m", "adam_v"))
        loss, g = net.grads(x, t)
        c = _check_forward_and_backward(net, st["params"], x, t)
        G = _check_gradients(net, g, c)
        y_ref, bound = _end_to_end_bound(c, x)
        _within(c["y"], y_ref, bound + 1e-30, f"Y end to end, step {step}")
        d = c["y"] - t
        assert loss == pytest.approx(float(np.sum(d * d)) / (B * N_OUT), rel=1e-6)
        net.train_step(x, t, LR)
        st2 = net.state()
        assert st2["step"] == st["step"] + 1
        after = tuple(net.unpack(st2[k]) for k in ("params", "adam_m", "adam_v"))
        _check_adam(before, after, G, step)
        x, t = _inputs(42)           # the second step on another batch


def test_forward_alone_writes_the_same_activations(net):
    """sas_mlp_forward (inference) takes the forward kernels of a training step: same bits."""
    x, _ = _inputs(43)
    y_pred = net.predict(torch.as_tensor(x).cuda()).cpu().numpy()
    a2_inf = net.read_buffer(_lib.SAS_MLP_BUF_A2B, B)
    net.grads(x, np.zeros((B, N_OUT), np.float32))
    assert np.array_equal(net.read_buffer(_lib.SAS_MLP_BUF_Y, B), y_pred)
    assert np.array_equal(net.read_buffer(_lib.SAS_MLP_BUF_A2B, B), a2_inf)


def test_read_buffer_rejects_bad_arguments(net):
    out = np.empty((B, H), np.float32)
    with pytest.raises(_lib.SasError) as e:
        _lib.sas_mlp_read_buffer(net._h, _lib.SAS_MLP_BUF_COUNT, B, out)
    assert e.value.status == _lib.SAS_ERR_INVALID_ARG
    with pytest.raises(_lib.SasError) as e:
        _lib.sas_mlp_read_buffer(net._h, _lib.SAS_MLP_BUF_Z1, B + 1, out)
    assert e.value.status == _lib.SAS_ERR_INVALID_ARG
