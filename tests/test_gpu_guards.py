"""Guard bands around the library's device buffers (sas_guard_bands, sas_guard_check): the checker
that stands in for a device memory checker on this hardware.

tests/guard_paths.py runs every path of the library (typed profiles mixed, FP64, deterministic with
exact sums, batched, sharded, by quadrature and by the hybrid; per-atom profiles and their gradient;
chi^2 and its gradient; pair histograms and the binned sum; two training steps and a prediction of the
surrogate network) in a fresh process, once without guard bands and once with SAS_GUARD_BANDS=1, so
that every buffer the library allocates lies between two bands.  The outputs must be the same (bit for
bit; the float32 gradients, whose per-atom sums use FP64 atomics in completion order, to a unit or
two of their last place), every
band must be intact after the calls, and four bytes written just past a buffer's end must be reported
as SAS_ERR_CORRUPT, naming that side of the buffer, and pass again once the band is restored.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_1306_2258_gb300 import _lib

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SCRIPT = os.path.join(ROOT, "tests", "guard_paths.py")


def _run(tmp_path, guards):
    out = tmp_path / f"out_{guards}.npz"
    env = dict(os.environ, SAS_GUARD_BANDS="1" if guards else "0")
    r = subprocess.run([sys.executable, SCRIPT, str(out)], capture_output=True, text=True, env=env, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    return np.load(out), json.loads(r.stdout.strip().splitlines()[-1])


def test_guard_bands_change_nothing_and_catch_an_overrun(tmp_path):
    _lib.load()   # built before the subprocesses start
    plain, _ = _run(tmp_path, False)
    guarded, rep = _run(tmp_path, True)
    assert sorted(plain.files) == sorted(guarded.files) and len(plain.files) >= 20
    for k in plain.files:
        a, b = plain[k], guarded[k]
        assert a.shape == b.shape, k
        if k.startswith("grad_"):
            # float32 outputs of FP64 sums taken in completion order: a unit or two of the last place
            assert np.allclose(a, b, rtol=2.0 ** -21, atol=2.0 ** -21 * float(np.max(np.abs(a)))), k
        else:
            assert np.array_equal(a, b), k
    assert rep["checked"] > 0 and rep["live"] == rep["checked"], rep
    assert rep["detected"], rep
    assert "after" in rep["message"], rep
    assert rep["restored"] == rep["checked"], rep
    assert rep["after_close"] < rep["checked"], rep   # the context's buffers went with it

