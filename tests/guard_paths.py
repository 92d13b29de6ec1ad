"""Runs every path of the library once on small seeded inputs and saves the outputs (argv[1], .npz);
with SAS_GUARD_BANDS=1 in the environment every buffer the library allocates has guard bands, and
the script then checks them, writes into one band on purpose and checks again.  Prints one JSON line.
Used by tests/test_gpu_guards.py, which runs it with the bands off and on and compares the outputs.
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

from paper_1306_2258_gb300 import _lib, workloads as wl  # noqa: E402
from paper_1306_2258_gb300.profile import Profile  # noqa: E402
from paper_1306_2258_gb300.surrogate import SurrogateMLP  # noqa: E402


class _Band:
    """A device address range as a CUDA array (for torch.as_tensor)."""

    def __init__(self, addr, n):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": "|u1", "data": (addr, False), "version": 3}


def run(out_path):
    dev = torch.device("cuda", 0)
    out = {}
    coef = wl.form_factor_coefficients(5, 901)
    q = wl.q_grid(0.0, 1.0, 201)
    q101 = wl.q_grid(0.01, 0.5, 101)
    small = wl.random_walk_globule(1537, 5, 902).as_f32()
    big = wl.random_walk_globule(9001, 5, 903).as_f32()
    xs, ts = torch.as_tensor(small.coords, device=dev), torch.as_tensor(small.types, device=dev)
    xb, tb = torch.as_tensor(big.coords, device=dev), torch.as_tensor(big.types, device=dev)
    # typed profiles: mixed (64- and 128-atom tiles), FP64, a batch, a deterministic context with its
    # exact sums, a shard, the quadrature and the hybrid
    for name, prec, det in (("mixed", "mixed", False), ("fp64", "fp64", False), ("det", "mixed", True)):
        p = Profile(coef, q, prec, deterministic=det)
        out["I_small_" + name] = p(xs, ts).cpu().numpy()
        out["I_big_" + name] = p(xb, tb).cpu().numpy()
        if det:
            out["exact_big"] = p.exact_sums()
        p.close()
    conf = np.stack([wl.perturbed(small, 0.5, 904 + k).coords for k in range(3)]).astype(np.float32)
    p = Profile(coef, q101, "mixed")
    out["I_batch"] = p(torch.as_tensor(conf, device=dev), ts).cpu().numpy()
    p.set_option(_lib.SAS_OPT_SHARD, 3 * 65536 + 1)   # shard 1 of 3
    out["I_shard"] = p(xb, tb).cpu().numpy()
    p.set_option(_lib.SAS_OPT_SHARD, 1 * 65536 + 0)
    for method in (1, 2):
        p.set_option(_lib.SAS_OPT_METHOD, method)
        out[f"I_method{method}"] = p(xb, tb).cpu().numpy()
    p.close()
    # per-atom form factors and their gradient; chi^2 and its gradient
    ff = torch.as_tensor(wl.atomic_form_factor_table(small.n, q, 905), device=dev)
    for prec in ("mixed", "fp64"):
        p = Profile(coef, q, prec)
        out["Ia_" + prec] = p.atomic(xs, ff).cpu().numpy()
        p.close()
    p = Profile(coef, q101, "mixed")
    ffa = torch.as_tensor(wl.atomic_form_factor_table(small.n, q101, 906), device=dev)
    gI = torch.as_tensor(np.random.default_rng(907).standard_normal(q101.size), device=dev)
    out["grad_vjp_atomic"] = p.vjp_atomic(xs, ffa, gI).cpu().numpy()
    T = p(torch.as_tensor(wl.perturbed(small, 1.0, 908).coords, device=dev), ts)
    chi2, g, _ = p.chi2_grad(xs, ts, T, 1.0 / T ** 2)
    out["chi2"] = np.atleast_1d(np.asarray(chi2.cpu() if hasattr(chi2, "cpu") else chi2, dtype=np.float64))
    out["grad_chi2"] = g.cpu().numpy()
    h, d = p.pair_histogram(xs, ts)
    out["hist"] = h.cpu().numpy()
    out["dropped"] = np.atleast_1d(np.asarray(d.cpu() if hasattr(d, "cpu") else d))
    counts = np.bincount(small.types, minlength=5)
    out["binned"] = p.binned(h, counts).cpu().numpy()
    p.close()
    # the surrogate network: two training steps and a prediction (batch 40, 64-48-13)
    rng = np.random.default_rng(909)
    net = SurrogateMLP(64, 48, 13, max_batch=40, seed=910)
    x = torch.as_tensor(rng.standard_normal((40, 64)).astype(np.float32), device=dev)
    t = torch.as_tensor(rng.standard_normal((40, 13)).astype(np.float32), device=dev)
    out["loss"] = np.array([net.train_step(x, t, 1e-3) for _ in range(2)])
    out["pred"] = net.predict(x).cpu().numpy()
    out["params"] = net.state()["params"]
    net.close()
    np.savez(out_path, **out)
    rep = {"n_outputs": len(out)}
    if os.environ.get("SAS_GUARD_BANDS") == "1":
        # the bands of every buffer still alive (contexts closed above freed theirs)
        keep = Profile(coef, q, "mixed")
        keep(xb, tb)
        torch.cuda.synchronize()
        rep["checked"] = _lib.sas_guard_check()
        live = _lib.sas_guard_list()
        rep["live"] = len(live)
        addr, nbytes = max(live, key=lambda e: e[1])
        torch.as_tensor(_Band(addr + nbytes, 4), device=dev).fill_(0)   # 4 bytes past the buffer's end
        torch.cuda.synchronize()
        try:
            _lib.sas_guard_check()
            rep["detected"] = False
        except _lib.SasError as e:
            rep["detected"] = e.status == _lib.SAS_ERR_CORRUPT
            rep["message"] = e.message
        torch.as_tensor(_Band(addr + nbytes, 4), device=dev).fill_(0xA5)   # put the band back
        torch.cuda.synchronize()
        rep["restored"] = _lib.sas_guard_check()
        keep.close()
        rep["after_close"] = _lib.sas_guard_check()
    print(json.dumps(rep))


if __name__ == "__main__":
    run(sys.argv[1])
