"""Learned surrogate and ensemble screen over the C ABI.

A 3-layer MLP maps per-type-pair distance histograms (exact integer counts from the GPU binning
kernel) to a standardized log I(q).  It is trained on exact profiles of perturbed conformers,
ranks an ensemble by its predicted chi^2 against a target profile, and the exact Debye kernel
re-scores the best fraction.  The network's forward, backward and Adam steps run in libsas.so's
kernels (bfloat16 tensor-core GEMMs, FP32 accumulation); this module only prepares inputs,
drives the loop and keeps checkpoints.

    python -m paper_1306_2258_gb300.surrogate [--conformers 4096] [--atoms 2000] [--epochs 60]

prints one JSON report (surrogate error against exact profiles, the binned-sinc baseline
computed from the same histograms, screen recall and timings).
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


def binned_sinc_profiles(hist: np.ndarray, types: np.ndarray, coef: np.ndarray, q: np.ndarray,
                         n_bins: int = N_BINS, r_max: float = R_MAX) -> np.ndarray:
    """The method without the network: the Debye sum over the histogram with every pair at its bin
    centre, I(q) ~ sum_t n_t f_t^2 + sum_p 2 f_a f_b sum_k c_pk sinc(q r_k).  Float64, host."""
    T = coef.shape[0]
    s = q / (4 * math.pi)
    F = coef[:, 8][:, None] + np.sum(coef[:, 0:4][:, :, None] * np.exp(-coef[:, 4:8][:, :, None] * s ** 2), axis=1)
    nt = np.bincount(types, minlength=T).astype(np.float64)
    diag = np.sum(nt[:, None] * F ** 2, axis=0)
    rk = (np.arange(n_bins) + 0.5) * (r_max / n_bins)
    x = q[:, None] * rk[None, :]
    sinc = np.where(x == 0, 1.0, np.sin(x) / np.where(x == 0, 1.0, x))   # [Q, n_bins]
    out = np.tile(diag, (hist.shape[0], 1))
    p = 0
    for a in range(T):
        for b in range(a, T):
            out += 2 * (F[a] * F[b])[None, :] * (hist[:, p, :].astype(np.float64) @ sinc.T)
            p += 1
    return out


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


def screen_select(net: "SurrogateMLP", feats: torch.Tensor, ys: "Standardizer", target, weights, k: int):
    """Rank conformers by the surrogate's chi^2 against `target` (weights w_q) and return (indices of the
    k best in increasing chi^2, chi^2 of all), both device tensors; the chi^2, ranking and selection run
    in the library (sas_screen_select)."""
    dev = feats.device
    pred = net.predict(feats)
    n_conf, n_q = int(pred.shape[0]), int(pred.shape[1])
    d = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device=dev)
    chi2 = torch.empty(n_conf, dtype=torch.float64, device=dev)
    top = torch.empty(k, dtype=torch.int32, device=dev)
    _lib.sas_screen_select(n_conf, n_q, pred, pred.stride(0), d(ys.mean), d(ys.std), d(target), d(weights), k, top,
                           None, chi2)
    return top, chi2


def gather_conformers(X: torch.Tensor, idx: torch.Tensor) -> torch.Tensor:
    """X[idx] for conformers X [C][n][3] float32 on the device (sas_gather_rows)."""
    out = torch.empty((int(idx.numel()),) + tuple(X.shape[1:]), dtype=X.dtype, device=X.device)
    _lib.sas_gather_rows(X, X[0].numel() * X.element_size(), idx, int(idx.numel()), out)
    return out


def run_screen(n_conf: int = 4096, n_atoms: int = 2000, n_train: int | None = None, epochs: int = 60,
               batch: int = 256, lr: float = 1e-3, hidden: int = 512, top_frac: float = 0.05, seed: int = 0):
    """Configuration 5 end to end; returns a report dict."""
    t0 = time.perf_counter()
    w = wl.c5_ensemble(n_conf=n_conf, n=n_atoms)
    n_train = n_train if n_train is not None else n_conf - n_conf // 8
    types = w["base"].types
    coef, q = w["coef"], w["q"]
    T = coef.shape[0]
    X = torch.as_tensor(w["conformers"], device="cuda")
    t_gen = time.perf_counter() - t0
    prof = Profile(coef, q)
    tt = torch.as_tensor(types, device="cuda")
    # exact profiles and histograms of every conformer (in slices to bound device memory)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    I_exact = torch.cat([prof(X[s:s + 1024], tt) for s in range(0, n_conf, 1024)]).cpu().numpy()
    torch.cuda.synchronize()
    t_exact_all = time.perf_counter() - t1
    hist = torch.cat([prof.pair_histogram(X[s:s + 1024], tt, N_BINS, R_MAX)[0]
                      for s in range(0, n_conf, 1024)]).cpu().numpy()
    feats = histogram_features(hist, pair_totals(types, T))
    logI = np.log(I_exact)
    xs = Standardizer(feats[:n_train])
    ys = Standardizer(logI[:n_train])
    Xn = xs(feats).astype(np.float32)
    Yn = ys(logI).astype(np.float32)
    net = SurrogateMLP(Xn.shape[1], hidden, q.size, max_batch=max(batch, 1024), seed=seed)
    t2 = time.perf_counter()
    losses = train(net, Xn[:n_train], Yn[:n_train], epochs, batch, lr, seed)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t2
    # held-out error of the surrogate and of the binned-sinc baseline (same histograms)
    test = slice(n_train, n_conf)
    I_sur = np.exp(ys.inverse(net.predict(torch.as_tensor(Xn[test], device="cuda")).double().cpu().numpy()))
    I_bin = binned_sinc_profiles(hist[test], types, coef, q)
    err_sur = np.abs(I_sur - I_exact[test]) / I_exact[test]
    err_bin = np.abs(I_bin - I_exact[test]) / I_exact[test]
    # screen: rank all conformers by surrogate chi^2 against a target, re-score the best exactly
    target = prof(torch.as_tensor(w["target"].coords, device="cuda"), tt).cpu().numpy()
    wq = 1.0 / target ** 2
    torch.cuda.synchronize()
    t3 = time.perf_counter()
    k = max(1, int(round(top_frac * n_conf)))
    top_t, chi_sur_t = screen_select(net, torch.as_tensor(Xn, device="cuda"), ys, target, wq, k)
    Xtop = gather_conformers(X, top_t)
    I_top = prof(Xtop, tt).cpu().numpy()
    top = top_t.cpu().numpy()
    chi_sur = chi_sur_t.cpu().numpy()
    chi_top = np.sum(wq * (I_top - target) ** 2, axis=1)
    best_screen = int(top[np.argmin(chi_top)])
    torch.cuda.synchronize()
    t_screen = time.perf_counter() - t3   # histograms assumed available, as for any candidate pool
    chi_exact = np.sum(wq * (I_exact - target) ** 2, axis=1)
    rank_exact = np.argsort(chi_exact)
    true_best = int(rank_exact[0])
    rank_of_found = int(np.where(rank_exact == best_screen)[0][0])
    recall10 = float(np.mean(np.isin(rank_exact[:10], top)))
    sp = np.corrcoef(np.argsort(np.argsort(chi_sur)), np.argsort(np.argsort(chi_exact)))[0, 1]
    net.close()
    prof.close()
    return {
        "conformers": n_conf, "atoms": n_atoms, "q": int(q.size), "train": n_train, "test": n_conf - n_train,
        "epochs": epochs, "batch": batch, "lr": lr, "hidden": hidden,
        "final_train_loss": losses[-1], "first_train_loss": losses[0],
        "surrogate_rel_err": {"median": float(np.median(err_sur)), "p95": float(np.percentile(err_sur, 95)),
                              "max": float(err_sur.max())},
        "binned_sinc_rel_err": {"median": float(np.median(err_bin)), "p95": float(np.percentile(err_bin, 95)),
                                "max": float(err_bin.max())},
        "screen": {"top_k": k, "true_best": true_best, "found": best_screen, "exact_rank_of_found": rank_of_found,
                   "recall_of_exact_top10_in_top_k": recall10, "spearman_rank_corr": float(sp),
                   "exact_evaluations": k, "exact_evaluations_without_surrogate": n_conf},
        "seconds": {"generate": t_gen, "exact_all": t_exact_all, "train": t_train, "screen": t_screen},
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--conformers", type=int, default=4096)
    ap.add_argument("--atoms", type=int, default=2000)
    ap.add_argument("--epochs", type=int, default=60)
    ap.add_argument("--hidden", type=int, default=512)
    args = ap.parse_args()
    print(json.dumps(run_screen(args.conformers, args.atoms, epochs=args.epochs, hidden=args.hidden)))


if __name__ == "__main__":
    main()
