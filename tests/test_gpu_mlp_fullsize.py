"""Element-by-element parity of the surrogate network at the size the benchmark trains it:
3840 -> 512 -> 512 -> 101 at batch 256 (the tcgen05 GEMMs' deep-ring tiles, the fused GELU and
bfloat16 epilogues, the transposed operands of the weight and input gradients), over two Adam steps.

The FP64 reference (oracle/mlp.py) runs from scratch on the test's own inputs: seeded parameters and
batches; before the second step the reference's own state after the first (float32) is loaded into
the network.  Every tensor the kernels write is compared with the reference's one element at a time,
within the bounds of tests/mlp_bounds.py.
"""
import numpy as np
import pytest
import torch

from paper_1306_2258_gb300 import _lib
from paper_1306_2258_gb300.surrogate import SurrogateMLP
from tests import mlp_bounds

pytestmark = pytest.mark.gpu

N_IN, H, N_OUT, B = 3840, 512, 101, 256


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


def test_full_size_forward_backward_and_two_adam_steps_element_by_element(net):
    mlp_bounds.adam_steps(net, [_inputs(41), _inputs(42)], 1e-3, 31)


@pytest.mark.parametrize("batch", [200, 600])
def test_ragged_batches_element_by_element(batch):
    """A batch of 200 rows takes the first layer's split-K path with a partial row tile (200 -> 208
    padded rows); 600 rows take the one-pass GEMMs whose epilogues write the transposed operands with
    their zero padding (600 -> 608).  One Adam step each, checked as above."""
    n = SurrogateMLP(N_IN, H, N_OUT, max_batch=batch, seed=37)
    try:
        rng = np.random.default_rng(batch)
        x = rng.standard_normal((batch, N_IN))
        x[:, rng.random(N_IN) < 0.2] = 0.0
        t = rng.standard_normal((batch, N_OUT))
        mlp_bounds.adam_steps(n, [(x.astype(np.float32), t.astype(np.float32))], 1e-3, 37)
    finally:
        n.close()


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
