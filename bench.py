"""Benchmark: Debye pair*q/s of the mixed-precision path at 50,000 atoms x 201 q
(globular random-walk chain, 5 atom types, q = 0..1 A^-1), next to the all-FP64
plain kernel on the same GB300 and the CPU oracle on the host cores.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--scaling weak|strong] [--profile-case NAME]

One step = one full profile call through the C ABI with device-resident inputs:
count/validate, scan, schedule read-back, pack, pair kernel, item reduction and
assembly.  Under torchrun every rank computes its own molecule (independent
problems, weak scaling, no data-path collective); rank 0 prints one JSON line.
`--scaling strong` splits one molecule over the ranks instead (NCCL all-gather of
the Q-vector shares).  `--impl reference` times the CPU oracle (the paper ships no
program to run, so the FP64 oracle is the reference arm) on a bounded subsample
of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_ATOMS = 50_000
METRIC = "Debye pair·q/s at 50k atoms×201 q: mixed vs FP64 plain at rel err≤1e-5"
SM_COUNT_NOMINAL = 152
FP32_LANES_PER_SM = 128
SM_MAX_MHZ_NOMINAL = 2070.0
OPS_PER_PAIR_Q = 2   # FP32 lane operations per pair*q: one FMA (recurrence) + one add (accumulate)
PAIR_KERNEL = "k_debye_mixed_pairs2<52,101,128,2,false,false>"
# DRAM bytes (read + write) of one pair-kernel launch on this workload, from the one-launch ncu
# capture summarised under profiles/ (same kernel source); None while the kernel has changed since
# that capture.
MIXED_KERNEL_DRAM_BYTES = 988_928


# The paper's own timings (Table 1: 50-point profiles on 0 < q <= 1, single-precision OpenCL; pair·q
# counted as N(N+1)/2 pairs x 50 q, the j <= k form of Section II) with their hardware: context for
# the line, not its target.
def _table1(n, seconds):
    return {"atoms": n, "s": seconds, "pair_q_per_s": n * (n + 1) / 2 * 50 / seconds}


# Table 1 in full: atoms -> (GT 330M s, GTX 295 s), single-precision OpenCL, 50-point profiles.
PAPER_TABLE1 = {1000: (0.03, 0.02), 2000: (0.07, 0.03), 4000: (0.25, 0.08), 10000: (1.34, 0.34),
                20000: (5.02, 1.14), 40000: (20.4, 3.94), 100000: (121.0, 22.5)}

PAPER_CONTEXT = {
    "source": "Table 1 (50-point profiles, 0 < q <= 1 A^-1, FP32 OpenCL GPU, parallel Java CPU)",
    "gtx295_gpu_40k": _table1(40000, 3.94),
    "gtx295_gpu_100k": _table1(100000, 22.5),
    "gt330m_gpu_100k": _table1(100000, 121.0),
    "xeon_2x4core_java_100k": _table1(100000, 806.0),
    "note": "other hardware, precision and q grid; not comparable as a ratio",
}


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clock and throttle samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def _cpu_oracle_sample(w, seconds_hint=20.0):
    """Time the CPU oracle (as it stands) on a seeded subsample of the workload."""
    import oracle
    from paper_1306_2258_gb300 import workloads as wl
    cores = oracle.max_threads()
    n = 1000
    sub = wl.subsample(w.mol, n, wl.seed_for(2, 77))
    t0 = time.perf_counter()
    oracle.profile(sub.coords, sub.types, w.coef, w.q)
    dt = time.perf_counter() - t0
    # scale the subsample so the timed oracle run takes about `seconds_hint`
    n2 = int(min(N_ATOMS, n * max(1.0, (seconds_hint / max(dt, 1e-3))) ** 0.5))
    sub = wl.subsample(w.mol, n2, wl.seed_for(2, 78))
    t0 = time.perf_counter()
    oracle.profile(sub.coords, sub.types, w.coef, w.q)
    dt = time.perf_counter() - t0
    pq = n2 * (n2 - 1) / 2 * w.q.size
    return {"value": pq / dt, "unit": "pair·q/s", "cores": cores, "kind": "oracle",
            "sample": f"{n2}-atom seeded subsample of the 50,000-atom globule x 201 q, "
                      f"{dt:.1f} s, FP64 double loop with libm sin"}, dt


def _cpu_oracle_cases():
    """Two more oracle timings for scale: the 1,000-atom FP64 configuration in full on every core,
    and one core on a 2,000-atom subsample of the 50k globule x 201 q."""
    import oracle
    from paper_1306_2258_gb300 import workloads as wl
    out = {}
    c1 = wl.c1_plain_fp64()
    t0 = time.perf_counter()
    oracle.profile(c1.mol.coords, c1.mol.types, c1.coef, c1.q)
    dt = time.perf_counter() - t0
    n = c1.mol.n
    out["c1_1000_atoms_x51q_all_cores"] = {"s": dt, "value": n * (n - 1) / 2 * c1.q.size / dt, "unit": "pair·q/s",
                                            "cores": oracle.max_threads()}
    w = wl.c2_globule(N_ATOMS)
    sub = wl.subsample(w.mol, 2000, wl.seed_for(2, 79))
    t0 = time.perf_counter()
    oracle.profile(sub.coords, sub.types, w.coef, w.q, n_threads=1)
    dt = time.perf_counter() - t0
    out["globule_2000_atoms_x201q_one_core"] = {"s": dt, "value": 2000 * 1999 / 2 * w.q.size / dt,
                                                 "unit": "pair·q/s", "cores": 1}
    return out


def run_reference(args):
    rank, world, _ = _dist()
    if rank != 0:
        return 0
    from paper_1306_2258_gb300 import workloads as wl
    w = wl.c2_globule(N_ATOMS)
    per_step = max(0.5, args.ref_seconds / max(args.steps + args.warmup, 1))
    vals, times = [], []
    base = None
    for s in range(args.warmup + args.steps):
        cb, dt = _cpu_oracle_sample(w, seconds_hint=per_step)
        if s >= args.warmup:
            vals.append(cb["value"])
            times.append(dt)
            base = cb
    value = float(np.mean(vals))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "pair·q/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * float(np.mean(times)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "globule 50,000 atoms x 201 q (bounded CPU subsample per step)",
                       "n_atoms": N_ATOMS, "n_q": 201, "l2": "n/a (CPU)"},
            "cpu_baseline": dict(base, value=value),
            "e2e": {"value": value, "unit": "pair·q/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def rank_molecule(w, rank: int, n: int = N_ATOMS):
    """Rank r's independent problem: rank 0 the canonical globule of the workload, every other rank
    its own seeded globule of the same size and shape (weak scaling, no data-path collective)."""
    from paper_1306_2258_gb300 import workloads as wl
    if rank == 0 and w is not None:
        return w.mol
    return wl.random_walk_globule(n, 5, wl.seed_for(2, 90_000 + rank)).as_f32()


def aggregate(tot_ms: float, units_per_step: float, steps: int, world: int, device=None):
    """(max over ranks of the timed-region duration in ms, whole-job throughput = all ranks' units
    over that duration).  Collective only when world > 1."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([tot_ms], dtype=torch.float64, device=device)
    u = torch.tensor([units_per_step * steps], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(u, op=dist.ReduceOp.SUM)
    max_ms = float(t.item())
    return max_ms, float(u.item()) / (max_ms / 1e3)


def _measured_peak(key):
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)[key])
    except (OSError, KeyError, ValueError):
        return None


def _timed(fn, stream, reps=3):
    """Median CUDA-event time (ms) of fn() on `stream` after one untimed call."""
    import torch
    fn()
    torch.cuda.synchronize()
    ms = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    return float(statistics.median(ms))


def run_rows(dev, stream):
    """Every other step of the path on its own workload (device-resident inputs, CUDA events)."""
    import torch

    from paper_1306_2258_gb300 import _lib, workloads as wl
    from paper_1306_2258_gb300.profile import Profile
    from paper_1306_2258_gb300.surrogate import (N_BINS, R_MAX, Standardizer, SurrogateMLP, gather_conformers,
                                                 histogram_features, pair_totals, screen_select)

    rows = {}

    def pairs(n):
        return n * (n - 1) // 2

    # elongated rod and sparse chain (configuration 3), mixed profile
    for name, w in (("profile_rod_c3", wl.c3_rod()), ("profile_sparse_chain_c3", wl.c3_sparse())):
        p = Profile(w.coef, w.q, "mixed")
        x = torch.as_tensor(w.mol.coords, device=dev)
        t = torch.as_tensor(w.mol.types, device=dev)
        ms = _timed(lambda: p(x, t, stream), stream)
        pq = pairs(w.mol.n) * w.q.size
        rows[name] = {"workload": f"{w.mol.n} atoms x {w.q.size} q", "ms": ms, "value": pq / (ms / 1e3),
                      "unit": "pair·q/s"}
        p.close()

    # per-atom form factors (no types, a hydration-shell-like table) on the 50,000-atom globule
    w = wl.c2_globule(50000)
    p = Profile(w.coef, w.q, "mixed")
    x = torch.as_tensor(w.mol.coords, device=dev)
    ffa = torch.as_tensor(wl.atomic_form_factor_table(w.mol.n, w.q, 770), device=dev)
    ms = _timed(lambda: p.atomic(x, ffa, stream), stream)
    pq = pairs(w.mol.n) * w.q.size
    rows["profile_atomic_ff_globule50k"] = {"workload": f"{w.mol.n} atoms x {w.q.size} q, per-atom form factors",
                                            "ms": ms, "value": pq / (ms / 1e3), "unit": "pair·q/s",
                                            "pair_kernel_ms": int(p.stats()[4]) / 1e6}
    p.close()
    del ffa

    # the paper's own timing workload (Table 1: globules of 1,000-100,000 atoms, 50 q on 0 < q <= 1),
    # whole mixed calls beside the paper's GPU times, each checked against the FP64 kernel per q
    entries = []
    for n_t1, (s330, s295) in PAPER_TABLE1.items():
        w1 = wl.table1_globule(n_t1)
        x1 = torch.as_tensor(w1.mol.coords, device=dev)
        t1 = torch.as_tensor(w1.mol.types, device=dev)
        p = Profile(w1.coef, w1.q, "mixed")
        ms = _timed(lambda: p(x1, t1, stream), stream)
        I_mixed = p(x1, t1, stream).cpu().numpy()
        p.close()
        p = Profile(w1.coef, w1.q, "fp64")
        I_64 = p(x1, t1, stream).cpu().numpy()
        p.close()
        entries.append({"atoms": n_t1, "ms": ms, "value": pairs(n_t1) * w1.q.size / (ms / 1e3),
                        "rel_err_vs_fp64": float(np.max(np.abs(I_mixed - I_64) / I_64)),
                        "paper_gtx295_s": s295, "paper_gt330m_s": s330,
                        "paper_gtx295_over_this": s295 / (ms / 1e3)})
    rows["table1_paper_workload"] = {
        "workload": "Table 1's workload: random-walk globules of 1,000-100,000 atoms (5 types) x 50 q, "
                    "q = 0.02..1.0 A^-1, mixed, whole calls",
        "unit": "pair·q/s", "entries": entries,
        "note": "the paper's times are single-precision OpenCL on a 2009 GTX 295 and a GT 330M: context, "
                "not a measured ratio of two implementations on this GPU"}

    # large compact molecule at small-angle q: direct sum against the hybrid (orientation average of
    # Eq. 1 by quadrature where cheaper, the direct sum elsewhere)
    mol = wl.random_walk_globule(200000, 5, wl.seed_for(2, 200000))
    q2 = wl.q_grid(0.0, 0.5, 201)
    x = torch.as_tensor(mol.coords, device=dev)
    t = torch.as_tensor(mol.types, device=dev)
    res = {}
    for method in (0, 1):
        p = Profile(w.coef, q2, "mixed")
        p.set_option(_lib.SAS_OPT_METHOD, method)
        res[method] = p(x, t, stream).cpu().numpy()
        ms = _timed(lambda: p(x, t, stream), stream)
        st = p.stats()
        pq = pairs(mol.n) * q2.size
        name = "profile_globule200k_saxs_direct" if method == 0 else "profile_globule200k_saxs_hybrid"
        rows[name] = {"workload": f"{mol.n} atoms (R = {wl.globule_radius(mol.n):.0f} A) x {q2.size} q (0..0.5 A^-1)",
                      "ms": ms, "value": pq / (ms / 1e3),
                      "unit": "pair·q/s" if method == 0 else "pair·q/s equivalent (same profile)",
                      "q_by_quadrature": int(st[6]), "directions": int(st[7])}
        p.close()
    rows["profile_globule200k_saxs_hybrid"]["max_rel_diff_vs_direct"] = float(
        np.max(np.abs(res[1] - res[0]) / np.abs(res[0])))
    del x, t

    # refinement (configuration 4): chi^2 and its gradient for 64 conformers of 5,000 atoms
    c4 = wl.c4_refinement()
    p = Profile(c4["coef"], c4["q"], "mixed")
    tt = torch.as_tensor(c4["base"].types, device=dev)
    target = p(torch.as_tensor(c4["target"].coords.astype(np.float32), device=dev), tt)
    wq = 1.0 / target ** 2
    X4 = torch.as_tensor(c4["conformers"], device=dev)
    B4, n4 = X4.shape[0], X4.shape[1]
    ms = _timed(lambda: p.chi2_grad(X4, tt, target, wq, stream), stream)
    pq = B4 * pairs(n4) * c4["q"].size
    rows["chi2_gradient_c4"] = {"workload": f"{B4} conformers x {n4} atoms x {c4['q'].size} q, forward + adjoint",
                                "ms": ms, "value": pq / (ms / 1e3), "unit": "pair·q/s (forward and adjoint each)",
                                "gradients_per_s": B4 / (ms / 1e3)}
    p.close()
    # the same on a SAS_DETERMINISTIC context (fixed-order per-atom gradient sums)
    p = Profile(c4["coef"], c4["q"], "mixed", deterministic=True)
    rows["chi2_gradient_c4"]["ms_deterministic"] = _timed(lambda: p.chi2_grad(X4, tt, target, wq, stream), stream)
    p.close()

    # the same refinement batch with per-atom form factors (a water-layer table per conformer): the
    # vector-Jacobian product of the per-atom profile
    ffa4 = torch.as_tensor(np.stack([wl.atomic_form_factor_table(n4, c4["q"], 780 + b) for b in range(B4)]),
                           device=dev)
    gI4 = torch.as_tensor(np.random.default_rng(781).standard_normal((B4, c4["q"].size)), device=dev) / target
    p = Profile(c4["coef"], c4["q"], "mixed")
    ms = _timed(lambda: p.vjp_atomic(X4, ffa4, gI4, stream), stream)
    rows["vjp_atomic_c4"] = {"workload": f"{B4} conformers x {n4} atoms x {c4['q'].size} q, per-atom form factors, "
                                         "vector-Jacobian product", "ms": ms, "value": pq / (ms / 1e3),
                             "unit": "pair·q/s", "gradients_per_s": B4 / (ms / 1e3)}
    p.close()
    del ffa4

    # ensemble (configuration 5): exact profiles, pair histograms, surrogate epoch and screen
    c5 = wl.c5_ensemble()
    X5 = torch.as_tensor(c5["conformers"], device=dev)
    B5, n5 = X5.shape[0], X5.shape[1]
    types5 = c5["base"].types
    t5 = torch.as_tensor(types5, device=dev)
    p = Profile(c5["coef"], c5["q"], "mixed")
    ms = _timed(lambda: p(X5, t5, stream), stream)
    pq = B5 * pairs(n5) * c5["q"].size
    rows["profiles_c5"] = {"workload": f"{B5} conformers x {n5} atoms x {c5['q'].size} q", "ms": ms,
                           "value": pq / (ms / 1e3), "unit": "pair·q/s"}
    ms = _timed(lambda: p.pair_histogram(X5, t5, N_BINS, R_MAX, stream), stream)
    rows["histogram_c5"] = {"workload": f"{B5} conformers x {n5} atoms, {N_BINS} bins", "ms": ms,
                            "value": B5 * pairs(n5) / (ms / 1e3), "unit": "pairs/s"}
    hist_d = p.pair_histogram(X5, t5, N_BINS, R_MAX, stream)[0]
    hist = hist_d.cpu().numpy()
    nt5 = np.bincount(types5, minlength=c5["coef"].shape[0])
    # the method without the network: the Debye sum over the histograms at bin centres
    ms = _timed(lambda: p.binned(hist_d, nt5, N_BINS, R_MAX, stream), stream)
    fma = B5 * hist.shape[1] * N_BINS * c5["q"].size
    peak_ops = SM_COUNT_NOMINAL * FP32_LANES_PER_SM * SM_MAX_MHZ_NOMINAL * 1e6
    rows["binned_profiles_c5"] = {"workload": f"{B5} conformers x {hist.shape[1]} type pairs x {N_BINS} bins x "
                                              f"{c5['q'].size} q (Debye sum at bin centres)",
                                  "ms": ms, "value": B5 / (ms / 1e3), "unit": "conformers/s",
                                  "frac_of_fp32_peak": fma / (ms / 1e3) / peak_ops,
                                  "basis": "one FP32 FMA per count and q over 152 x 128 lanes x 2070 MHz"}
    I_bin_d = p.binned(hist_d, nt5, N_BINS, R_MAX, stream)
    feats = torch.as_tensor(histogram_features(hist, pair_totals(types5, c5["coef"].shape[0])).astype(np.float32),
                            device=dev)
    n_in, n_out, hidden, batch = feats.shape[1], c5["q"].size, 512, 256
    n_train = B5 - B5 // 8
    net = SurrogateMLP(n_in, hidden, n_out, max_batch=B5, seed=0)
    tgt = torch.zeros((batch, n_out), dtype=torch.float32, device=dev)

    def epoch():
        for s0 in range(0, n_train - batch + 1, batch):
            net.train_step(feats[s0:s0 + batch], tgt, 1e-3)

    ms = _timed(epoch, stream)
    steps = n_train // batch
    flop = steps * 3 * 2 * batch * (n_in * hidden + hidden * hidden + hidden * n_out)
    rows["surrogate_epoch_c5"] = {"workload": f"{steps} Adam steps of batch {batch}, {n_in}-{hidden}-{hidden}-{n_out} MLP",
                                  "ms": ms, "value": flop / (ms / 1e3) / 1e12, "unit": "TFLOP/s (GEMM flop)"}
    k = int(round(0.05 * B5))

    target5 = p(torch.as_tensor(c5["target"].coords, device=dev), t5).cpu().numpy()
    ys = Standardizer(np.zeros((1, n_out)))   # a stand-in: the timing does not depend on it

    def screen(use_net):
        top, _ = screen_select(net if use_net else None, feats if use_net else None, ys if use_net else None,
                               target5, 1.0 / target5 ** 2, k, base=I_bin_d)
        p(gather_conformers(X5, top), t5, stream)

    for name, use_net in (("screen_c5", True), ("screen_binned_c5", False)):
        ms = _timed(lambda: screen(use_net), stream)
        rows[name] = {"workload": (f"network correction of the binned profiles over {B5} conformers" if use_net else
                                   f"binned profiles alone over {B5} conformers") + f", top {k} re-scored exactly",
                      "ms": ms, "value": B5 / (ms / 1e3), "unit": "conformers screened/s"}
    net.close()
    p.close()

    # the surrogate's GEMM (tcgen05, TMA-fed) on a large square problem, against the measured peak
    G = 8192
    gA = torch.randn((G, G), device=dev).to(torch.bfloat16)
    gB = torch.randn((G, G), device=dev).to(torch.bfloat16)
    gC = torch.empty((G, G), dtype=torch.float32, device=dev)
    ms = _timed(lambda: _lib.sas_gemm_bf16(G, G, G, gA, G, gB, G, None, gC, G, stream), stream)
    tflops = 2.0 * G ** 3 / (ms / 1e3) / 1e12
    peak = _measured_peak("bf16_tflops")
    rows["gemm_bf16_tcgen05"] = {"workload": f"{G}^3 bf16 -> fp32 (C = A B^T)", "ms": ms, "value": tflops,
                                 "unit": "TFLOP/s", "peak": peak, "frac": (tflops / peak) if peak else None,
                                 "peak_basis": "cuBLAS bf16 burst, MEASURED_PEAKS.json"}
    del gA, gB, gC
    # the FP32-recurrence profile rows against the nominal FP32 lane rate, at the headline's count
    # of two lane operations per pair·q (whole call: packing, reductions and assembly included)
    peak_ops = SM_COUNT_NOMINAL * FP32_LANES_PER_SM * SM_MAX_MHZ_NOMINAL * 1e6
    for k in ("profile_rod_c3", "profile_sparse_chain_c3", "profile_atomic_ff_globule50k",
              "profile_globule200k_saxs_direct", "profiles_c5"):
        if k in rows and rows[k].get("unit") == "pair·q/s":
            rows[k]["fp32_frac_whole_call"] = rows[k]["value"] * OPS_PER_PAIR_Q / peak_ops
    return rows


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_1306_2258_gb300 import _lib, workloads as wl
    from paper_1306_2258_gb300.profile import Profile

    rank, world, local = _dist()
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = wl.c2_globule(N_ATOMS)
    mol = rank_molecule(w, rank)
    n, Q = mol.n, w.q.size
    pairs = n * (n - 1) // 2
    pq = pairs * Q

    prof = Profile(w.coef, w.q, "mixed")
    x = torch.as_tensor(mol.coords, device=dev)
    t = torch.as_tensor(mol.types, device=dev)
    out = torch.empty((1, Q), dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # 256 MB > L2
    stream = torch.cuda.current_stream(dev)

    def step():
        _lib.sas_profile_batch(prof._ctx, x, _lib.SAS_COORDS_F32, t, n, 1, out, stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    launches_per_step = int(prof.stats()[5])

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    kern_ns = []
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            flush.fill_(float(k))               # L2 flush between timed steps (not timed)
            ev[k][0].record(stream)
            step()
            ev[k][1].record(stream)
            kern_ns.append(int(prof.stats()[4]))
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    tot_ms, value = aggregate(float(sum(step_ms)), pq, args.steps, world, dev)
    I_mixed = out[0].cpu().numpy().copy()

    if args.skip_extras:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": "pair·q/s", "n_gpus": world,
                              "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot_ms / args.steps,
                              "note": "mixed path only (--skip-extras)"}))
        return 0

    # ---- end to end through the public API with host buffers (copies inside the timed region)
    xh = torch.as_tensor(mol.coords).pin_memory()
    th = torch.as_tensor(mol.types).pin_memory()
    oh = torch.empty((1, Q), dtype=torch.float64).pin_memory()
    _lib.sas_profile_batch(prof._ctx, xh, _lib.SAS_COORDS_F32, th, n, 1, oh, stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_steps = max(3, args.steps // 2)
    for _ in range(e2e_steps):
        _lib.sas_profile_batch(prof._ctx, xh, _lib.SAS_COORDS_F32, th, n, 1, oh, stream)
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    e2e = {"value": pq / e2e_s, "unit": "pair·q/s",
           "h2d_bytes_per_step": int(xh.numel() * 4 + th.numel() * 4), "d2h_bytes_per_step": int(Q * 8)}

    # ---- the FP64 plain kernel on the same molecule (1 timed step after 1 warm-up)
    p64 = Profile(w.coef, w.q, "fp64")
    out64 = torch.empty((1, Q), dtype=torch.float64, device=dev)
    _lib.sas_profile_batch(p64._ctx, x, _lib.SAS_COORDS_F32, t, n, 1, out64, stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    _lib.sas_profile_batch(p64._ctx, x, _lib.SAS_COORDS_F32, t, n, 1, out64, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms64 = e0.elapsed_time(e1)
    I64 = out64[0].cpu().numpy()
    rel = float(np.max(np.abs(I_mixed - I64) / np.abs(I64)))

    if rank != 0:
        return 0
    kern_s = float(np.median(kern_ns)) / 1e9
    clocks = clk.summary()
    peak_ops = SM_COUNT_NOMINAL * FP32_LANES_PER_SM * SM_MAX_MHZ_NOMINAL * 1e6 / 1e12
    achieved_ops = pq * OPS_PER_PAIR_Q / kern_s / 1e12
    # measured denominators (after the timed region): FP32 FMA scalar/packed, MUFU, FP64 FMA
    meas = _lib.sas_measure_peaks(stream)
    fp32_meas = max(meas["ffma"], meas["ffma2"]) / 1e12
    fp64_ops = pq * 2 / (ms64 / 1e3) / 1e12   # the FP64 kernel: one DFMA and one DADD per pair·q
    line = {
        "metric": METRIC, "value": value, "unit": "pair·q/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "globule 50,000 atoms (seeded 3.8 A random walk, R = 110.5 A, 5 types) x 201 q "
                               "(0..1 A^-1), float32 coordinates, mixed FP32/FP64",
                   "n_atoms": n, "n_q": Q, "pairs": pairs, "l2": "flushed between steps (256 MB write)",
                   "work_items": int(prof.stats()[0]),
                   # the metric's comparison: the same molecule by the all-FP64 kernel, and the
                   # largest relative difference per q against the 1e-5 bound
                   "vs_fp64_plain": {"fp64_pair_q_per_s": pq / (ms64 / 1e3), "fp64_ms": ms64,
                                     "mixed_over_fp64": (tot_ms / args.steps) and ms64 / (tot_ms / args.steps),
                                     "rel_err_max": rel, "rel_err_bound": 1e-5}},
        "rel_err_vs_fp64": rel,
        "fp64_plain": {"value": pq / (ms64 / 1e3), "unit": "pair·q/s", "ms_per_step": ms64, "dtype": "f64",
                       "achieved_fp64_tops": fp64_ops, "dfma_peak_tops": meas["dfma"] / 1e12,
                       "frac_of_dfma_peak": fp64_ops / (meas["dfma"] / 1e12)},
        "speedup_vs_fp64": (pq / (tot_ms / args.steps / 1e3)) / (pq / (ms64 / 1e3)),
        "roofline": {"bound": "alu", "achieved": achieved_ops, "peak": peak_ops, "unit": "Tops/s (FP32 lane ops)",
                     "frac": achieved_ops / peak_ops, "traffic": MIXED_KERNEL_DRAM_BYTES,
                     "kernel": PAIR_KERNEL, "kernel_ms": kern_s * 1e3,
                     "peak_basis": "152 SMs x 128 FP32 lanes x 2070 MHz (nominal max clock)",
                     "measured_peak": fp32_meas, "frac_of_measured": achieved_ops / fp32_meas,
                     "measured": {"ffma_tops": meas["ffma"] / 1e12, "ffma2_tops": meas["ffma2"] / 1e12,
                                  "mufu_sin_tops": meas["mufu_sin"] / 1e12, "dfma_tops": meas["dfma"] / 1e12,
                                  "ffma2_3op_tops": meas["ffma2_3op"] / 1e12, "sm_mhz": meas["sm_mhz"],
                                  "basis": "sas_measure_peaks microbenchmarks, same process, after the timed region"}},
        "e2e": e2e,
        "paper_context": PAPER_CONTEXT,
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clocks,
    }
    if not args.skip_rows:
        line["rows"] = run_rows(dev, stream)
        a = line["rows"].get("profile_atomic_ff_globule50k")
        if a and a.get("pair_kernel_ms") and meas.get("ffma2_3op"):
            # the per-atom kernel's core is made of packed FMAs that each read three register pairs of
            # their own: its rate against that instruction form's measured rate
            ops = a["value"] * a["ms"] / a["pair_kernel_ms"] * OPS_PER_PAIR_Q
            a["fp32_frac_pair_kernel"] = ops / (peak_ops * 1e12)
            a["frac_of_3op_ffma2"] = ops / meas["ffma2_3op"]
        h = line["rows"].get("histogram_c5")
        if h and meas.get("atoms_shared"):
            # one shared-memory atomic add per pair: the conflict-free atomic rate bounds the kernel
            h["roofline"] = {"bound": "shared atomics", "achieved": h["value"], "peak": meas["atoms_shared"],
                             "unit": "pairs/s (one shared atomic add each)",
                             "frac": h["value"] / meas["atoms_shared"],
                             "peak_basis": "sas_measure_peaks: conflict-free shared-memory integer atomic adds/s",
                             "note": "the kernel is bound by instruction issue (about 25 warp-instructions per "
                                     "32 pairs), not by the atomic rate"}
    if not args.skip_cpu and world == 1:
        line["cpu_baseline"], _ = _cpu_oracle_sample(w, seconds_hint=15.0)
        line["cpu_baseline"]["cases"] = _cpu_oracle_cases()
    # the headline figures once more, last, where a reader of the line's tail finds them
    line["summary"] = {"value": value, "e2e": e2e["value"], "roofline_frac": achieved_ops / peak_ops,
                       "kernel_ms": kern_s * 1e3, "rel_err_vs_fp64": rel, "rel_err_bound": 1e-5,
                       "fp64_pair_q_per_s": pq / (ms64 / 1e3), "speedup_vs_fp64": line["speedup_vs_fp64"]}
    print(json.dumps(line))
    prof.close()
    p64.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def run_strong(args):
    """One molecule split over the ranks (strong scaling): each rank computes its shard of the work
    list (SAS_OPT_SHARD) and the Q-vector shares are all-gathered over NCCL and summed in rank
    order; a step is the whole profile on every rank.  Timed like the default mode (barriers,
    CUDA events, the maximum over ranks)."""
    import torch
    import torch.distributed as dist

    from paper_1306_2258_gb300 import _lib, workloads as wl
    from paper_1306_2258_gb300.profile import Profile
    from paper_1306_2258_gb300.shard import allreduce_exact, allreduce_shares, set_shard

    rank, world, local = _dist()
    if "MASTER_ADDR" not in os.environ:   # a plain single-process run: a group of one
        os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": "29561", "RANK": "0", "WORLD_SIZE": "1"})
    torch.cuda.set_device(local)
    dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    w = wl.c2_globule(N_ATOMS)
    n, Q = w.mol.n, w.q.size
    pq = n * (n - 1) // 2 * Q
    prof = Profile(w.coef, w.q, "mixed", deterministic=args.exact)
    set_shard(prof, rank, world)
    x = torch.as_tensor(w.mol.coords, device=dev)
    t = torch.as_tensor(w.mol.types, device=dev)
    share = torch.empty((1, Q), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    result = {}
    T = w.coef.shape[0]
    Ush = np.empty((1, T * (T + 1) // 2, Q, 2), dtype=np.int64)   # this shard's exact sums (host)
    whole_I = torch.empty((1, Q), dtype=torch.float64, device=dev)

    def step():
        _lib.sas_profile_batch(prof._ctx, x, _lib.SAS_COORDS_F32, t, n, 1, share, stream)
        if args.exact:   # exact 128-bit sums all-reduced as 32-bit limbs: the unsplit profile's bits
            _lib.sas_exact_sums(prof._ctx, Ush, Ush.size)
            U = allreduce_exact(torch.as_tensor(Ush, device=dev)).cpu().numpy()
            _lib.sas_assemble_exact(prof._ctx, U, 1, whole_I)
            result["I"] = whole_I[0]
        else:
            result["I"] = allreduce_shares(share[0])

    for _ in range(args.warmup):
        step()
    dist.barrier()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(args.steps):
        step()
    b.record(stream)
    torch.cuda.synchronize()
    dist.barrier()
    ms = torch.tensor([a.elapsed_time(b) / args.steps], dtype=torch.float64, device=dev)
    dist.all_reduce(ms, op=dist.ReduceOp.MAX)
    whole = Profile(w.coef, w.q, "mixed", deterministic=args.exact)   # unsharded, untimed: the shares sum to it
    ref = whole(x, t).cpu().numpy()
    whole.close()
    I = result["I"].cpu().numpy()
    if rank == 0:
        t_s = float(ms.item()) / 1e3
        print(json.dumps({
            "metric": METRIC, "value": pq / t_s, "unit": "pair·q/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_s * 1e3, "higher_is_better": True, "scaling": "strong",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "globule 50,000 atoms x 201 q, one molecule split over the ranks "
                                   + ("(shards of equal pair work on deterministic contexts, NCCL all-reduce of their "
                                      "exact 128-bit sums as 32-bit limbs)" if args.exact else
                                      "(shards of equal pair work, NCCL all-gather of the Q-vector shares)"),
                       "n_atoms": n, "n_q": Q, "parallelism": f"shards{world}", "exact": bool(args.exact)},
            "rel_diff_vs_unsharded": float(np.max(np.abs(I - ref) / np.abs(ref))),
            "identical_to_unsharded": bool(np.array_equal(I, ref)),
        }))
    prof.close()
    dist.destroy_process_group()
    return 0


PROFILE_CASES = ("histogram", "gradient", "gradient_recurrence", "gemm", "atomic", "quadrature", "binned", "rod", "pairs2",
                 "train", "table1")


def run_profile_case(args):
    """Reduced launches of the secondary kernels for profiler captures, two launches of each so that
    a capture can skip the first (no timing, no JSON line):

      histogram    512 conformers x 2,000 atoms of the ensemble workload, 256 bins
      gradient     16 conformers x 5,000 atoms x 101 q of the refinement workload (chi^2 + adjoint,
                   the tabulated pair weight)
      gradient_recurrence  the same with the sums over q by the recurrence (SAS_OPT_ADJOINT 1)
      binned       the Debye sum at bin centres over the histograms of 4,096 ensemble conformers
      rod          the 30,000-atom double-helix rod x 101 q (the benchmark row's profile)
      train        four Adam steps of the 3840-512-512-101 surrogate at batch 256 (the epoch row's step)
      gemm         4096 x 4096 x 4096 bfloat16 -> float32 on the tcgen05 GEMM
      atomic       20,000-atom globule x 201 q with a per-atom form-factor table
      quadrature   20,000-atom globule x 65 q (0..0.32 A^-1), orientation average of Eq. 1 on every q
      pairs2       20,000-atom globule x 201 q (0..1 A^-1): the headline's pair kernel on a smaller molecule
      table1       20,000-atom globule of Table 1's workload x 50 q (0.02..1.0 A^-1): the 52-q two-pair form
                   with the coefficient formed both ways and the start phase taken from the step phase
    """
    import torch

    from paper_1306_2258_gb300 import _lib, workloads as wl
    from paper_1306_2258_gb300.profile import Profile
    from paper_1306_2258_gb300.surrogate import N_BINS, R_MAX

    cases = PROFILE_CASES if args.profile_case == "all" else (args.profile_case,)
    dev = torch.device("cuda", 0)
    report = {}
    if "histogram" in cases:
        c5 = wl.c5_ensemble(n_conf=512)
        X5 = torch.as_tensor(c5["conformers"], device=dev)
        t5 = torch.as_tensor(c5["base"].types, device=dev)
        p = Profile(c5["coef"], c5["q"])
        for _ in range(2):
            h, d = p.pair_histogram(X5, t5, N_BINS, R_MAX)
        report["histogram_pairs"] = int(h.sum())
        p.close()
    for case, form in (("gradient", 0), ("gradient_recurrence", 1)):
        if case not in cases:
            continue
        c4 = wl.c4_refinement(batch=16)
        p4 = Profile(c4["coef"], c4["q"])
        p4.set_option(_lib.SAS_OPT_ADJOINT, form)
        tt = torch.as_tensor(c4["base"].types, device=dev)
        T = p4(torch.as_tensor(c4["target"].coords.astype(np.float32), device=dev), tt)
        X4 = torch.as_tensor(c4["conformers"], device=dev)
        for _ in range(2):
            chi2, _, _ = p4.chi2_grad(X4, tt, T, 1.0 / T ** 2)
        report["chi2_sum_" + case] = float(chi2.sum())
        p4.close()
    if "train" in cases:
        from paper_1306_2258_gb300.surrogate import SurrogateMLP
        rng = np.random.default_rng(5)
        net = SurrogateMLP(3840, 512, 101, max_batch=256, seed=0)
        xs = torch.as_tensor(rng.standard_normal((256, 3840)).astype(np.float32), device=dev)
        ts = torch.zeros((256, 101), dtype=torch.float32, device=dev)
        for _ in range(4):
            net.train_step(xs, ts, 1e-3)
        report["train_steps"] = 4
        net.close()
    if "table1" in cases:
        w6 = wl.table1_globule(20000)
        p = Profile(w6.coef, w6.q)
        x6 = torch.as_tensor(w6.mol.coords, device=dev)
        t6 = torch.as_tensor(w6.mol.types, device=dev)
        for _ in range(2):
            I6 = p(x6, t6)
        report["table1_I0"] = float(I6[0])
        p.close()
    if "rod" in cases:
        w3 = wl.c3_rod()
        p = Profile(w3.coef, w3.q)
        x3 = torch.as_tensor(w3.mol.coords, device=dev)
        t3 = torch.as_tensor(w3.mol.types, device=dev)
        for _ in range(2):
            I3 = p(x3, t3)
        report["rod_I0"] = float(I3[0])
        p.close()
    if "binned" in cases:
        c5 = wl.c5_ensemble()
        X5 = torch.as_tensor(c5["conformers"], device=dev)
        t5 = torch.as_tensor(c5["base"].types, device=dev)
        p = Profile(c5["coef"], c5["q"])
        h, _ = p.pair_histogram(X5, t5, N_BINS, R_MAX)
        nt = np.bincount(c5["base"].types, minlength=c5["coef"].shape[0])
        for _ in range(2):
            Ib = p.binned(h, nt, N_BINS, R_MAX)
        report["binned_I0"] = float(Ib[0, 0])
        p.close()
    if "gemm" in cases:
        G = 4096
        gA = torch.randn((G, G), device=dev).to(torch.bfloat16)
        gB = torch.randn((G, G), device=dev).to(torch.bfloat16)
        gC = torch.empty((G, G), dtype=torch.float32, device=dev)
        for _ in range(2):
            _lib.sas_gemm_bf16(G, G, G, gA, G, gB, G, None, gC, G)
        report["gemm"] = G
    w = wl.c2_globule(20000)
    xa = torch.as_tensor(w.mol.coords, device=dev)
    if "atomic" in cases:
        pa = Profile(w.coef, w.q)
        ffa = torch.as_tensor(wl.atomic_form_factor_table(w.mol.n, w.q, 770), device=dev)
        for _ in range(2):
            Ia = pa.atomic(xa, ffa)
        report["atomic_I0"] = float(Ia[0])
        pa.close()
    if "pairs2" in cases:
        pp = Profile(w.coef, w.q)
        for _ in range(2):
            Ip = pp(xa, torch.as_tensor(w.mol.types, device=dev))
        report["pairs2_I0"] = float(Ip[0])
        pp.close()
    if "quadrature" in cases:
        pq = Profile(w.coef, wl.q_grid(0.0, 0.32, 65))
        pq.set_option(_lib.SAS_OPT_METHOD, 2)
        for _ in range(2):
            Iq = pq(xa, torch.as_tensor(w.mol.types, device=dev))
        report["quadrature_I0"] = float(Iq[0])
        pq.close()
    torch.cuda.synchronize()
    print("profile cases:", json.dumps(report))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--skip-cpu", action="store_true", help="leave out the CPU-oracle baseline")
    ap.add_argument("--skip-rows", action="store_true",
                    help="leave out the timings of the other path steps (rod, sparse chain, gradient, ensemble)")
    ap.add_argument("--skip-extras", action="store_true",
                    help="time the mixed path only (no e2e, FP64 or CPU legs; for profiler runs)")
    ap.add_argument("--ref-seconds", type=float, default=120.0,
                    help="CPU time of the whole --impl reference run (each step a subsample sized to its share)")
    ap.add_argument("--scaling", default="weak", choices=["weak", "strong"],
                    help="weak (default): one molecule per rank; strong: one molecule split over the ranks")
    ap.add_argument("--exact", action="store_true",
                    help="with --scaling strong: deterministic contexts whose exact shard sums are all-reduced, "
                         "so that every rank holds the unsplit profile bit for bit")
    ap.add_argument("--profile-case", default=None, choices=("all",) + PROFILE_CASES,
                    help="run reduced launches of the secondary kernels for a profiler capture, then exit")
    args = ap.parse_args()
    if args.profile_case:
        return run_profile_case(args)
    if args.impl == "reference":
        return run_reference(args)
    if args.scaling == "strong":
        return run_strong(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
