"""The benchmark's contract where it needs no GPU: the reference arm (the CPU oracle, timed on the
host's cores) prints one JSON line with the keys the contract names; without a GPU the GPU arm and
the library fail loudly instead of falling back to the CPU."""
import json
import os
import subprocess
import sys

import pytest
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench(args, timeout):
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT, capture_output=True,
                          text=True, timeout=timeout)


def test_reference_arm_prints_one_contract_line():
    r = _bench(["--impl", "reference", "--steps", "2", "--warmup", "1", "--ref-seconds", "3"], timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "pair·q/s"
    assert d["steps"] == 2 and d["warmup"] == 1 and d["n_gpus"] == 1 and d["higher_is_better"] is True
    assert d["data"] == "synthetic" and d["config"]["workload"] and d["dtype"] == "f64"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


@pytest.mark.skipif(torch.cuda.is_available(), reason="behaviour without a GPU")
def test_gpu_arm_fails_without_a_gpu():
    r = _bench(["--steps", "1", "--warmup", "0"], timeout=300)
    assert r.returncode != 0 and not r.stdout.strip()


@pytest.mark.skipif(torch.cuda.is_available(), reason="behaviour without a GPU")
def test_library_calls_fail_without_a_gpu():
    from paper_1306_2258_gb300 import _lib, workloads as wl
    from paper_1306_2258_gb300.profile import Profile
    w = wl.c1_plain_fp64()
    with pytest.raises(_lib.SasError) as e:
        Profile(w.coef, w.q)(w.mol.coords, w.mol.types)
    assert e.value.status == _lib.SAS_ERR_CUDA
