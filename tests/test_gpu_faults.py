"""Failure handling without a GPU fault: an injected device-allocation failure and a host-side wait
that runs out of time both come back as status codes, leave the context usable, and later calls
give the same result as a clean run.  Each case runs in a fresh subprocess (the allocation hook is
read once per process)."""
import json
import os
import subprocess
import sys

import pytest
import torch

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_CHILD = r"""
import json, sys
sys.path.insert(0, {root!r})
import numpy as np, torch
from paper_1306_2258_gb300 import _lib, workloads as wl
mode = {mode!r}
mol = wl.random_walk_globule(3000, 5, 31).as_f32()
coef = wl.form_factor_coefficients(5, 32)
q = wl.q_grid(0, 1, 201)
res = {{}}
ctx = _lib.sas_create(5, coef, q)
out = np.zeros((1, q.size))
def call():
    _lib.sas_profile_batch(ctx, mol.coords, 0, mol.types, mol.n, 1, out)
if mode == "timeout":
    big = wl.c3_sparse(100_000)
    ctx2 = _lib.sas_create(3, big.coef, big.q)
    _lib.sas_set_option(ctx2, _lib.SAS_OPT_TIMEOUT_MS, 1)
    o2 = np.zeros((1, big.q.size))
    try:
        _lib.sas_profile_batch(ctx2, big.mol.coords, 0, big.mol.types, big.mol.n, 1, o2)
        res["first"] = 0
    except _lib.SasError as e:
        res["first"] = e.status
    _lib.sas_destroy(ctx2)
statuses = []
for attempt in range(6):
    try:
        call()
        statuses.append(0)
        break
    except _lib.SasError as e:
        statuses.append(e.status)
res["statuses"] = statuses
res["I"] = out[0].tolist()
_lib.sas_destroy(ctx)
print(json.dumps(res))
"""


def _run(mode, env_extra=None):
    env = dict(os.environ)
    env.pop("SAS_TEST_FAIL_ALLOC", None)
    env.update(env_extra or {})
    r = subprocess.run([sys.executable, "-c", _CHILD.format(root=ROOT, mode=mode)], capture_output=True, text=True,
                       env=env, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_injected_allocation_failure_then_recovery():
    assert torch.cuda.is_available()
    clean = _run("clean")
    assert clean["statuses"] == [0]
    for k in (3, 5, 8):
        r = _run("alloc", {"SAS_TEST_FAIL_ALLOC": str(k)})
        assert r["statuses"][-1] == 0
        assert all(s == 3 for s in r["statuses"][:-1])      # SAS_ERR_ALLOC, then success
        assert r["I"] == clean["I"]


def test_wait_limit_returns_timeout_and_context_survives():
    r = _run("timeout")
    assert r["first"] == 5                                     # SAS_ERR_TIMEOUT
    assert r["statuses"] == [0]
    clean = _run("clean")
    assert r["I"] == clean["I"]
