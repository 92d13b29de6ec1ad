"""Learned surrogate and ensemble screen over the C ABI.

A 3-layer MLP maps per-type-pair distance histograms (exact integer counts from the GPU binning
kernel) to a standardized log I(q).  It is trained on exact profiles of perturbed conformers,
ranks an ensemble by its predicted chi^2 against a target profile, and the exact Debye kernel
re-scores the best fraction.  The network's forward, backward and Adam steps run in libsas.so's
kernels (bfloat16 tensor-core GEMMs, FP32 accumulation); this module only prepares inputs,
drives the loop and keeps checkpoints.

    python -m paper_1306_2258_gb300.surrogate [--conformers 4096] [--atoms 2000] [--epochs 60]

prints one JSON report (surrogate error against exact profiles, the binned Debye baseline computed
from the same histograms, both screens' recall and timings).  By default the network learns the
residual log I - log I_binned, a correction of the baseline.
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np
import torch

from . import _lib
from . import workloads as wl
from .profile import Profile

N_BINS = 256
R_MAX = 120.0


class SurrogateMLP:
    """n_in -> h -> h -> n_out MLP on the GPU (sas_mlp_* entry points)."""

    def __init__(self, n_in: int, n_hidden: int, n_out: int, max_batch: int, seed: int = 0):
        self.n_in, self.h, self.n_out, self.max_batch = n_in, n_hidden, n_out, max_batch
        self._h = _lib.sas_mlp_create(n_in, n_hidden, n_out, max_batch)
        self.n_params = _lib.sas_mlp_param_count(self._h)
        self.load_state(self.init_params(seed), None, None, 0)

    def close(self):
        if getattr(self, "_h", None) is not None:
            _lib.sas_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- parameters (packed order W1, b1, W2, b2, W3, b3)
    def shapes(self):
        return [("W1", (self.h, self.n_in)), ("b1", (self.h,)), ("W2", (self.h, self.h)), ("b2", (self.h,)),
                ("W3", (self.n_out, self.h)), ("b3", (self.n_out,))]

    def unpack(self, flat) -> dict:
        out, o = {}, 0
        for name, shp in self.shapes():
            n = int(np.prod(shp))
            out[name] = np.asarray(flat[o:o + n]).reshape(shp)
            o += n
        return out

    def pack(self, d) -> np.ndarray:
        return np.concatenate([np.asarray(d[name], np.float32).reshape(-1) for name, _ in self.shapes()])

    def init_params(self, seed: int) -> np.ndarray:
        """Uniform weights with variance 1/fan_in (bound sqrt(3/fan_in)), zero biases; seeded."""
        rng = np.random.default_rng(seed)
        d = {}
        for name, shp in self.shapes():
            if name.startswith("W"):
                bound = math.sqrt(3.0 / shp[1])
                d[name] = rng.uniform(-bound, bound, size=shp).astype(np.float32)
            else:
                d[name] = np.zeros(shp, np.float32)
        return self.pack(d)

    def state(self):
        p = np.empty(self.n_params, np.float32)
        m = np.empty(self.n_params, np.float32)
        v = np.empty(self.n_params, np.float32)
        step = _lib.sas_mlp_get_state(self._h, p, m, v)
        return {"params": p, "adam_m": m, "adam_v": v, "step": step}

    def load_state(self, params, adam_m, adam_v, step):
        _lib.sas_mlp_set_state(self._h, np.ascontiguousarray(params, np.float32),
                               None if adam_m is None else np.ascontiguousarray(adam_m, np.float32),
                               None if adam_v is None else np.ascontiguousarray(adam_v, np.float32), step)

    def save(self, path: str, extra: dict | None = None):
        st = self.state()
        np.savez(path, params=st["params"], adam_m=st["adam_m"], adam_v=st["adam_v"], step=st["step"],
                 dims=np.array([self.n_in, self.h, self.n_out, self.max_batch]), **(extra or {}))

    @classmethod
    def load(cls, path: str):
        z = np.load(path)
        n_in, h, n_out, mb = (int(v) for v in z["dims"])
        net = cls(n_in, h, n_out, mb)
        net.load_state(z["params"], z["adam_m"], z["adam_v"], int(z["step"]))
        return net, z

    # -- compute
    def train_step(self, x, t, lr: float) -> float:
        loss = np.zeros(1, np.float32)
        _lib.sas_mlp_train_step(self._h, x, t, int(x.shape[0]), lr, loss)
        return float(loss[0])

    def grads(self, x, t):
        g = np.empty(self.n_params, np.float32)
        loss = np.zeros(1, np.float32)
        _lib.sas_mlp_grads(self._h, x, t, int(x.shape[0]), g, loss)
        return float(loss[0]), g

    def read_buffer(self, which: int, batch: int) -> np.ndarray:
        """Rows [0, batch) of an intermediate tensor of the last passes (_lib.SAS_MLP_BUF_*), float32."""
        width = {_lib.SAS_MLP_BUF_XB: self.n_in, _lib.SAS_MLP_BUF_Y: self.n_out, _lib.SAS_MLP_BUF_DY: self.n_out,
                 _lib.SAS_MLP_BUF_DYB: self.n_out}.get(which, self.h)
        out = np.empty((batch, width), np.float32)
        _lib.sas_mlp_read_buffer(self._h, which, batch, out)
        return out

    def predict(self, x) -> torch.Tensor:
        xt = torch.as_tensor(x).float().contiguous()
        out = torch.empty((xt.shape[0], self.n_out), dtype=torch.float32, device=xt.device)
        for s in range(0, xt.shape[0], self.max_batch):
            e = min(xt.shape[0], s + self.max_batch)
            _lib.sas_mlp_forward(self._h, xt[s:e], e - s, out[s:e])
        return out


# ----------------------------------------------------------------------------------------------
# features and targets
# ----------------------------------------------------------------------------------------------

def pair_totals(types: np.ndarray, n_types: int) -> np.ndarray:
    """Number of unordered pairs of each type pair (row-major over a <= b)."""
    nt = np.bincount(types, minlength=n_types).astype(np.float64)
    out = []
    for a in range(n_types):
        for b in range(a, n_types):
            out.append(nt[a] * (nt[a] - 1) / 2 if a == b else nt[a] * nt[b])
    return np.array(out)


class Standardizer:
    def __init__(self, x: np.ndarray, floor: float = 1e-6):
        self.mean = x.mean(0)
        self.std = np.maximum(x.std(0), floor)

    def __call__(self, x):
        return (x - self.mean) / self.std

    def inverse(self, z):
        return z * self.std + self.mean


def histogram_features(hist: np.ndarray, totals: np.ndarray) -> np.ndarray:
    """Counts normalised by the number of pairs of their type pair, flattened to [C, P*n_bins]."""
    h = hist.astype(np.float64) / np.maximum(totals, 1.0)[None, :, None]
    return h.reshape(h.shape[0], -1)


# ----------------------------------------------------------------------------------------------
# the pipeline
# ----------------------------------------------------------------------------------------------

def train(net: SurrogateMLP, X: np.ndarray, Y: np.ndarray, epochs: int, batch: int, lr: float, seed: int,
          log_every: int = 0):
    """Seeded minibatch training (device tensors); returns per-epoch mean losses."""
    dev = torch.device("cuda")
    Xd = torch.as_tensor(X, dtype=torch.float32, device=dev)
    Yd = torch.as_tensor(Y, dtype=torch.float32, device=dev)
    rng = np.random.default_rng(seed)
    losses = []
    for ep in range(epochs):
        order = torch.as_tensor(rng.permutation(X.shape[0]), device=dev)
        tot, nb = 0.0, 0
        for s in range(0, X.shape[0] - batch + 1, batch):
            idx = order[s:s + batch]
            tot += net.train_step(Xd[idx].contiguous(), Yd[idx].contiguous(), lr)
            nb += 1
        losses.append(tot / max(nb, 1))
        if log_every and (ep + 1) % log_every == 0:
            print(f"epoch {ep + 1}: loss {losses[-1]:.4e}", flush=True)
    return losses


def screen_select(net: "SurrogateMLP | None", feats: torch.Tensor | None, ys: "Standardizer | None", target,
                  weights, k: int, base: torch.Tensor | None = None):
    """Rank conformers by the chi^2 of a predicted profile against `target` (weights w_q) and return
    (indices of the k best in increasing chi^2, chi^2 of all), both device tensors.  The prediction is
    base * exp(network) when both are given (a network trained on the residual log I - log base),
    exp(network) without a base, and the base alone without a network.  The chi^2, ranking and
    selection run in the library (sas_screen_select)."""
    pred = net.predict(feats) if net is not None else None
    ref = pred if pred is not None else base
    dev = ref.device
    n_conf, n_q = int(ref.shape[0]), int(ref.shape[1])
    d = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device=dev)
    chi2 = torch.empty(n_conf, dtype=torch.float64, device=dev)
    top = torch.empty(k, dtype=torch.int32, device=dev)
    mean, std = (d(ys.mean), d(ys.std)) if pred is not None else (None, None)
    _lib.sas_screen_select(n_conf, n_q, pred, pred.stride(0) if pred is not None else 0, mean, std,
                           base, base.stride(0) if base is not None else 0, d(target), d(weights), k, top, None, chi2)
    return top, chi2


def gather_conformers(X: torch.Tensor, idx: torch.Tensor) -> torch.Tensor:
    """X[idx] for conformers X [C][n][3] float32 on the device (sas_gather_rows)."""
    out = torch.empty((int(idx.numel()),) + tuple(X.shape[1:]), dtype=X.dtype, device=X.device)
    _lib.sas_gather_rows(X, X[0].numel() * X.element_size(), idx, int(idx.numel()), out)
    return out


def _rel_err_stats(I, I_exact):
    e = np.abs(I - I_exact) / I_exact
    return {"median": float(np.median(e)), "p95": float(np.percentile(e, 95)), "max": float(e.max())}


def _screen_report(top, chi, chi_exact, I_top, target, wq):
    """What a screen found: the selected conformers re-scored exactly, against the exact ranking."""
    rank_exact = np.argsort(chi_exact)
    chi_top = np.sum(wq * (I_top - target) ** 2, axis=1)
    found = int(top[np.argmin(chi_top)])
    k = top.size
    return {"top_k": int(k), "found": found, "exact_rank_of_found": int(np.where(rank_exact == found)[0][0]),
            "recall_of_exact_top10_in_top_k": float(np.mean(np.isin(rank_exact[:10], top))),
            "recall_of_exact_top_k": float(np.mean(np.isin(rank_exact[:k], top))),
            "spearman_rank_corr": float(np.corrcoef(np.argsort(np.argsort(chi)),
                                                    np.argsort(np.argsort(chi_exact)))[0, 1])}


def run_screen(n_conf: int = 4096, n_atoms: int = 2000, n_train: int | None = None, epochs: int = 60,
               batch: int = 256, lr: float = 1e-3, hidden: int = 512, top_frac: float = 0.05, seed: int = 0,
               residual: bool = True):
    """Configuration 5 end to end; returns a report dict.

    The method without the network is the binned Debye sum over the same histograms
    (sas_binned_profile).  With `residual` the network learns log I - log I_binned, so its profile is
    I_binned exp(prediction): a correction of the baseline.  Both screens (network and baseline)
    rank all conformers against one target and re-score the same number k of them exactly."""
    t0 = time.perf_counter()
    w = wl.c5_ensemble(n_conf=n_conf, n=n_atoms)
    n_train = n_train if n_train is not None else n_conf - n_conf // 8
    types = w["base"].types
    coef, q = w["coef"], w["q"]
    T = coef.shape[0]
    nt = np.bincount(types, minlength=T)
    X = torch.as_tensor(w["conformers"], device="cuda")
    t_gen = time.perf_counter() - t0
    prof = Profile(coef, q)
    tt = torch.as_tensor(types, device="cuda")
    # exact profiles, histograms and binned profiles of every conformer (slices bound device memory)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    I_exact = torch.cat([prof(X[s:s + 1024], tt) for s in range(0, n_conf, 1024)]).cpu().numpy()
    torch.cuda.synchronize()
    t_exact_all = time.perf_counter() - t1
    hist_d = torch.cat([prof.pair_histogram(X[s:s + 1024], tt, N_BINS, R_MAX)[0] for s in range(0, n_conf, 1024)])
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    I_bin_d = prof.binned(hist_d, nt, N_BINS, R_MAX)
    torch.cuda.synchronize()
    t_binned = time.perf_counter() - t2
    I_bin = I_bin_d.cpu().numpy()
    hist = hist_d.cpu().numpy()
    feats = histogram_features(hist, pair_totals(types, T))
    logY = np.log(I_exact) - (np.log(I_bin) if residual else 0.0)
    xs = Standardizer(feats[:n_train])
    ys = Standardizer(logY[:n_train])
    Xn = xs(feats).astype(np.float32)
    Yn = ys(logY).astype(np.float32)
    net = SurrogateMLP(Xn.shape[1], hidden, q.size, max_batch=max(batch, 1024), seed=seed)
    t3 = time.perf_counter()
    losses = train(net, Xn[:n_train], Yn[:n_train], epochs, batch, lr, seed)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t3
    # held-out error of the network's profile and of the baseline alone
    test = slice(n_train, n_conf)
    corr = np.exp(ys.inverse(net.predict(torch.as_tensor(Xn[test], device="cuda")).double().cpu().numpy()))
    I_sur = corr * (I_bin[test] if residual else 1.0)
    # screens against a target profile: the network's and the baseline's, the same exact budget k
    target = prof(torch.as_tensor(w["target"].coords, device="cuda"), tt).cpu().numpy()
    wq = 1.0 / target ** 2
    chi_exact = np.sum(wq * (I_exact - target) ** 2, axis=1)
    k = max(1, int(round(top_frac * n_conf)))
    feats_d = torch.as_tensor(Xn, device="cuda")
    screens, seconds = {}, {}
    for name, use_net in (("network", True), ("binned_baseline", False)):
        torch.cuda.synchronize()
        t4 = time.perf_counter()
        top_t, chi_t = screen_select(net if use_net else None, feats_d if use_net else None, ys if use_net else None,
                                     target, wq, k, base=I_bin_d if (residual or not use_net) else None)
        I_top = prof(gather_conformers(X, top_t), tt).cpu().numpy()
        torch.cuda.synchronize()
        seconds[name] = time.perf_counter() - t4   # histograms (and binned profiles) assumed available
        screens[name] = _screen_report(top_t.cpu().numpy(), chi_t.cpu().numpy(), chi_exact, I_top, target, wq)
    net.close()
    prof.close()
    return {
        "conformers": n_conf, "atoms": n_atoms, "q": int(q.size), "train": n_train, "test": n_conf - n_train,
        "epochs": epochs, "batch": batch, "lr": lr, "hidden": hidden, "residual": residual,
        "final_train_loss": losses[-1], "first_train_loss": losses[0],
        "surrogate_rel_err": _rel_err_stats(I_sur, I_exact[test]),
        "binned_sinc_rel_err": _rel_err_stats(I_bin[test], I_exact[test]),
        "true_best": int(np.argmin(chi_exact)), "exact_evaluations": k, "exact_evaluations_without_screen": n_conf,
        "screen": screens,
        "seconds": {"generate": t_gen, "exact_all": t_exact_all, "binned_all": t_binned, "train": t_train,
                    "screen_network": seconds["network"], "screen_binned": seconds["binned_baseline"]},
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--conformers", type=int, default=4096)
    ap.add_argument("--atoms", type=int, default=2000)
    ap.add_argument("--epochs", type=int, default=60)
    ap.add_argument("--hidden", type=int, default=512)
    ap.add_argument("--absolute", action="store_true", help="train on log I itself instead of log I - log I_binned")
    args = ap.parse_args()
    print(json.dumps(run_screen(args.conformers, args.atoms, epochs=args.epochs, hidden=args.hidden,
                                residual=not args.absolute)))


if __name__ == "__main__":
    main()
