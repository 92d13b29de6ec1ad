"""The pins catch plausible mistakes: each mutant of the oracle's C source (a
dropped factor, a dropped diagonal, a transposed operand, a wrong scaling, a
sign flip, an off-by-one bin rule) is compiled on the CPU and must fail at
least one pin of tests/test_oracle_pins.py or tests/test_oracle_grad_hist.py."""
import ctypes
import os
import shutil
import subprocess

import pytest

import oracle
from tests import test_oracle_grad_hist as tg
from tests import test_oracle_pins as tp

SRC = os.path.join(os.path.dirname(oracle.__file__), "debye_oracle.c")

MUTANTS = {
    "no_factor_two": ("nadd(&tot, 2.0 * row[i * n_q + k]);", "nadd(&tot, 1.0 * row[i * n_q + k]);"),
    "no_diagonal": ("nadd(&tot, d);", "(void)d;"),
    "ff_scaling": ("double s = q / (4.0 * ORACLE_PI);", "double s = q / (2.0 * ORACLE_PI);"),
    "transposed_ff": ("double term = fi[k] * fj[k] * sinc(q[k] * r);",
                      "double term = fi[k] * fi[k] * sinc(q[k] * r);"),
    "diag_in_pairs": ("for (int64_t j = i + 1; j < n; ++j) {\n                const double *fj",
                      "for (int64_t j = i; j < n; ++j) {\n                const double *fj"),
    "grad_sign": ("nadd(&g[c], wij * (xyz[3 * i + c] - xyz[3 * j + c]));",
                  "nadd(&g[c], wij * (xyz[3 * j + c] - xyz[3 * i + c]));"),
    "grad_bracket": ("double br = (cos(x) - sin(x) / x) / (r * r);",
                     "double br = (cos(x) + sin(x) / x) / (r * r);"),
    "bin_rule": ("if (e2[mid] <= r2)", "if (e2[mid] < r2)"),
    "atomic_layout": ("f[i * n_q + k] = ff[(int64_t)k * n + i];", "f[i * n_q + k] = ff[i * n_q + k];"),
    "atomic_vjp_layout": ("f[i * n_q + k] = ff[i + (int64_t)k * n];", "f[i * n_q + k] = ff[i * n_q + k];"),
    "pair_index": ("return a * T - a * (a - 1) / 2 + (b - a);",
                   "return (a * T - a * (a - 1) / 2 + (b - a) + 1) % (T * (T + 1) / 2);"),
}

PINS = [getattr(tp, n) for n in dir(tp) if n.startswith("test_")] + \
       [getattr(tg, n) for n in dir(tg) if n.startswith("test_")]


def _run_pins():
    failed = []
    for fn in PINS:
        argnames = getattr(fn, "pytestmark", [])
        params = [m for m in argnames if m.name == "parametrize"]
        cases = [dict(zip([params[0].args[0]], [v])) for v in params[0].args[1]] if params else [{}]
        for kw in cases:
            try:
                fn(**kw)
            except (AssertionError, ValueError, MemoryError):
                failed.append(fn.__name__)
                break
    return failed


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    text = open(SRC).read()
    assert text.count(old) >= 1, f"mutation anchor missing: {name}"
    mut = tmp_path / "mut.c"
    mut.write_text(text.replace(old, new, 1))
    so = tmp_path / "libmut.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-fopenmp", "-ffp-contract=off", "-shared",
                    "-o", str(so), str(mut), "-lm"], check=True)
    lib = oracle._configure(ctypes.CDLL(str(so)))
    saved = oracle._load()
    oracle._lib = lib
    try:
        failed = _run_pins()
    finally:
        oracle._lib = saved
    assert failed, f"mutant {name} passed every pin"
