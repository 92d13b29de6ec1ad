"""GPU surrogate MLP: the bfloat16 tensor-core GEMM, the network's forward pass and gradients, and
the Adam step against the FP64 reference (oracle/mlp.py, same bfloat16 rounding points); exact
checkpoint/resume; and the ensemble screen end to end."""
import numpy as np
import pytest
import torch

import oracle
from oracle import mlp as ref
from paper_1306_2258_gb300 import _lib, workloads as wl
from paper_1306_2258_gb300.profile import Profile
from paper_1306_2258_gb300.surrogate import SurrogateMLP, run_screen
from tests import mlp_bounds

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    _lib.load()


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


@pytest.mark.parametrize("M,N,K", [(200, 130, 96), (64, 64, 3840), (1, 7, 16), (257, 512, 512), (256, 512, 3840),
                                   (300, 1000, 208), (128, 64, 64)])
def test_gemm_bf16_matches_fp64(M, N, K):
    rng = np.random.default_rng(M + N + K)
    A = torch.from_numpy(rng.standard_normal((M, K)).astype(np.float32)).to(torch.bfloat16).cuda()
    B = torch.from_numpy(rng.standard_normal((N, K)).astype(np.float32)).to(torch.bfloat16).cuda()
    bias = torch.from_numpy(rng.standard_normal(N).astype(np.float32)).cuda()
    C = torch.empty((M, N), dtype=torch.float32, device="cuda")
    _lib.sas_gemm_bf16(M, N, K, A, K, B, K, bias, C, N)
    Ad, Bd = A.double().cpu().numpy(), B.double().cpu().numpy()
    expect = Ad @ Bd.T + bias.double().cpu().numpy()
    bound = np.abs(Ad) @ np.abs(Bd).T + 1.0
    assert np.all(np.abs(C.double().cpu().numpy() - expect) <= 1e-6 * bound)


@pytest.mark.parametrize("M,N,K", [(8192, 2048, 320), (8000, 2000, 208)])
def test_gemm_bf16_large_persistent_path(M, N, K):
    """Problems with several 128 x 256 tiles per SM take the persistent kernel (two tensor-memory
    accumulators, epilogue overlapped with the next tile); K = 208 ends in a partial 64-wide slice and
    8000 x 2000 leaves partial tiles in both M and N.
    Checked on row blocks from every part of C against FP64 products of the same inputs."""
    rng = np.random.default_rng(M + N + K)
    A = torch.from_numpy(rng.standard_normal((M, K)).astype(np.float32)).to(torch.bfloat16).cuda()
    B = torch.from_numpy(rng.standard_normal((N, K)).astype(np.float32)).to(torch.bfloat16).cuda()
    bias = torch.from_numpy(rng.standard_normal(N).astype(np.float32)).cuda()
    C = torch.full((M, N), float("nan"), dtype=torch.float32, device="cuda")
    _lib.sas_gemm_bf16(M, N, K, A, K, B, K, bias, C, N)
    Bd = B.double().cpu().numpy()
    rows = np.concatenate([np.arange(0, 130), np.arange(M // 2 - 70, M // 2 + 70), np.arange(M - 130, M),
                           rng.integers(0, M, 64)])
    Ad = A[torch.as_tensor(rows).cuda()].double().cpu().numpy()
    expect = Ad @ Bd.T + bias.double().cpu().numpy()
    got = C[torch.as_tensor(rows).cuda()].double().cpu().numpy()
    bound = np.abs(Ad) @ np.abs(Bd).T + 1.0
    assert not np.isnan(got).any()
    assert np.all(np.abs(got - expect) <= 1e-6 * bound)


def _net_and_data(n_in=64, h=48, n_out=13, B=40, seed=7):
    net = SurrogateMLP(n_in, h, n_out, max_batch=64, seed=seed)
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((B, n_in)).astype(np.float32)
    t = rng.standard_normal((B, n_out)).astype(np.float32)
    return net, x, t


def test_forward_and_gradients_match_reference():
    net, x, t = _net_and_data()
    p = net.unpack(net.init_params(7))
    y = net.predict(torch.as_tensor(x).cuda()).cpu().numpy()
    y_ref, _ = ref.forward(p, x)
    assert _rel(y, y_ref) <= 1e-3
    loss, g = net.grads(x, t)
    loss_ref, g_ref, _ = ref.loss_and_grads(p, x, t)
    assert loss == pytest.approx(loss_ref, rel=1e-3)
    gd = net.unpack(g)
    for k in g_ref:
        assert _rel(gd[k], g_ref[k]) <= 1e-3, k
    net.close()


def test_adam_steps_match_reference():
    """Three steps on ragged sizes (batch 40, 13 outputs: partial tiles everywhere), each from the
    reference's own state, element by element."""
    net, x, t = _net_and_data(seed=8)
    rng = np.random.default_rng(80)
    batches = [(x, t)] + [(rng.standard_normal(x.shape).astype(np.float32),
                           rng.standard_normal(t.shape).astype(np.float32)) for _ in range(2)]
    mlp_bounds.adam_steps(net, batches, 1e-3, 8)
    net.close()


def test_checkpoint_resume_is_bit_exact(tmp_path):
    rng = np.random.default_rng(9)
    batches = [(rng.standard_normal((32, 64)).astype(np.float32), rng.standard_normal((32, 13)).astype(np.float32))
               for _ in range(6)]
    a = SurrogateMLP(64, 48, 13, max_batch=32, seed=11)
    for x, t in batches:
        a.train_step(x, t, 2e-3)
    b = SurrogateMLP(64, 48, 13, max_batch=32, seed=11)
    for x, t in batches[:3]:
        b.train_step(x, t, 2e-3)
    b.save(str(tmp_path / "ck.npz"))
    b.close()
    c, _ = SurrogateMLP.load(str(tmp_path / "ck.npz"))
    for x, t in batches[3:]:
        c.train_step(x, t, 2e-3)
    sa, sc = a.state(), c.state()
    assert sa["step"] == sc["step"] == 6
    for k in ("params", "adam_m", "adam_v"):
        assert np.array_equal(sa[k], sc[k]), k
    a.close()
    c.close()


def test_screen_finds_good_conformers_with_5_percent_of_exact_evaluations():
    """What the screen buys: ranking the ensemble by the network's correction of the binned profiles
    and re-scoring only its best 5% with the exact kernel still lands on a conformer from the exact top
    5%, for 1/20 of the exact evaluations; its ranking correlates with the exact one."""
    r = run_screen(n_conf=768, n_atoms=600, epochs=40, hidden=128, batch=64, seed=3)
    s = r["screen"]["network"]
    assert r["final_train_loss"] < 0.5 * r["first_train_loss"]
    assert s["exact_rank_of_found"] < 0.05 * r["conformers"]
    assert s["spearman_rank_corr"] > 0.5
    assert r["exact_evaluations"] * 20 <= r["exact_evaluations_without_screen"] + 20


def test_network_gains_over_the_binned_debye_sum_at_the_same_exact_budget():
    """What the trained network gains over the method without it.  The method without the network is
    the Debye sum over the same exact histograms with every pair at its bin centre
    (sas_binned_profile).  The network is trained on the residual log I - log I_binned, so it can
    only correct the baseline.  On held-out conformers its profiles are closer to the exact ones
    than the baseline's, and at the same budget of exact re-scores (the best 5% by each ranking)
    its screen recalls at least as much of the exact top 5% and ranks closer to the exact order."""
    r = run_screen(n_conf=768, n_atoms=600, epochs=40, hidden=128, batch=64, seed=3)
    net, base = r["screen"]["network"], r["screen"]["binned_baseline"]
    assert r["surrogate_rel_err"]["median"] <= 0.75 * r["binned_sinc_rel_err"]["median"]
    assert r["surrogate_rel_err"]["p95"] <= r["binned_sinc_rel_err"]["p95"]
    assert net["recall_of_exact_top_k"] >= base["recall_of_exact_top_k"]
    assert net["spearman_rank_corr"] >= base["spearman_rank_corr"]
    assert net["exact_rank_of_found"] <= base["exact_rank_of_found"]


def test_the_exact_profiles_the_screens_are_scored_by_match_the_oracle():
    """The screen tests score both rankings by the exact kernel's profiles of the 768-conformer,
    600-atom ensemble; conformers from its start, middle and end, and the target, agree with the
    oracle's FP64 sum."""
    w = wl.c5_ensemble(n_conf=768, n=600)
    types = w["base"].types
    p = Profile(w["coef"], w["q"])
    tt = torch.as_tensor(types).cuda()
    idx = [0, 383, 767]
    I = p(torch.as_tensor(w["conformers"][idx]).cuda(), tt).cpu().numpy()
    It = p(torch.as_tensor(w["target"].coords).cuda(), tt).cpu().numpy()
    p.close()
    for row, c in zip(I, idx):
        ref_I = oracle.profile(w["conformers"][c].astype(np.float64), types, w["coef"], w["q"])
        assert np.max(np.abs(row - ref_I) / ref_I) <= 1e-5, c
    ref_t = oracle.profile(w["target"].coords.astype(np.float64), types, w["coef"], w["q"])
    assert np.max(np.abs(It - ref_t) / ref_t) <= 1e-5
