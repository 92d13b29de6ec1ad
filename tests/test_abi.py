"""The C-ABI library builds, loads and exports every symbol include/sas.h declares;
argument checks that need no GPU return the documented status codes."""
import os
import re
import subprocess

import numpy as np
import pytest

from paper_1306_2258_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sas.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sas_[a-z_0-9]+)\s*\(", text)))


def test_header_declarations_match_binding():
    assert _declared() == sorted(_lib.EXPORTS)


def test_library_exports_every_declared_symbol():
    path = _lib.load()._name
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (sas_[a-z_0-9]+)\b", out))
    missing = set(_declared()) - exported
    assert not missing, missing


def test_version_and_last_error_are_strings():
    assert "sm_103a" in _lib.sas_version()
    assert isinstance(_lib.sas_last_error(), str)


@pytest.mark.parametrize("n_types,nq,code", [(0, 11, _lib.SAS_ERR_INVALID_ARG),
                                            (17, 11, _lib.SAS_ERR_INVALID_ARG),
                                            (3, 0, _lib.SAS_ERR_INVALID_ARG),
                                            (3, 1665, _lib.SAS_ERR_INVALID_ARG)])
def test_create_rejects_bad_sizes(n_types, nq, code):
    import ctypes
    coef = np.ones((max(n_types, 1), 9))
    q = np.linspace(0, 1, max(nq, 1))
    h = ctypes.c_void_p()
    st = _lib.load().sas_create(n_types, coef.ctypes.data, q.ctypes.data, nq, 0, ctypes.byref(h))
    assert st == code and not h.value


def test_create_rejects_grids_beyond_64_uniform_runs_and_bad_grids():
    coef = np.ones((2, 9))
    q = np.cumsum(np.random.default_rng(3).uniform(0.001, 0.01, 300))   # no three points in line: 150 runs
    with pytest.raises(_lib.SasError) as e:
        _lib.sas_create(2, coef, q)
    assert e.value.status == _lib.SAS_ERR_UNSUPPORTED
    with pytest.raises(_lib.SasError) as e:
        _lib.sas_create(2, coef, np.linspace(-0.1, 1, 51))
    assert e.value.status == _lib.SAS_ERR_INVALID_ARG
    bad = coef.copy()
    bad[1, 3] = np.nan
    with pytest.raises(_lib.SasError) as e:
        _lib.sas_create(2, bad, np.linspace(0, 1, 51))
    assert e.value.status == _lib.SAS_ERR_INVALID_ARG
    with pytest.raises(_lib.SasError) as e:
        _lib.sas_create(2, coef, np.linspace(1, 0, 51))
    assert e.value.status == _lib.SAS_ERR_UNSUPPORTED


def test_null_context_is_rejected():
    with pytest.raises(_lib.SasError) as e:
        _lib.sas_profile(None, None, 0, None, 0, None, 0)
    assert e.value.status == _lib.SAS_ERR_INVALID_ARG
    with pytest.raises(_lib.SasError):
        _lib.sas_set_option(None, _lib.SAS_OPT_JMAX, 0)
    _lib.sas_destroy(None)


def test_create_flags_constant_and_unknown_bits():
    text = open(HEADER).read()
    assert int(re.search(r"#define SAS_DETERMINISTIC (\d+)", text).group(1)) == _lib.SAS_DETERMINISTIC
    import ctypes
    coef = np.ones((2, 9))
    q = np.linspace(0, 1, 11)
    for bad in (2, 1 << 5, _lib.SAS_DETERMINISTIC | 8):
        h = ctypes.c_void_p()
        st = _lib.load().sas_create(2, coef.ctypes.data, q.ctypes.data, 11, bad, ctypes.byref(h))
        assert st == _lib.SAS_ERR_INVALID_ARG and not h.value, bad


def test_header_constants_match_binding():
    """Every SAS_* enumerator and #define of the header has the binding's value."""
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    consts = {k: int(v) for k, v in re.findall(r"#define (SAS_[A-Z0-9_]+) (\d+)\b", text)}
    for body in re.findall(r"enum\s*\{(.*?)\}", text, flags=re.S) + re.findall(r"typedef enum\s*\{(.*?)\}", text,
                                                                                 flags=re.S):
        for k, v in re.findall(r"(SAS_[A-Z0-9_]+)\s*=\s*(\d+)", body):
            consts[k] = int(v)
    expected = [k for k in consts if not k.startswith("SAS_STATIC_") and k != "SAS_H"]
    assert len(expected) >= 20
    for k in expected:
        assert getattr(_lib, k) == consts[k], k


@pytest.mark.parametrize("lang,std", [("c", "-std=c99"), ("c++", "-std=c++17")])
def test_header_compiles_as_plain_c_and_cpp(tmp_path, lang, std):
    """include/sas.h is a C header: it compiles on its own as C99 and C++17 with warnings as errors,
    and every declared entry point can be referenced."""
    import shutil
    cc = shutil.which("gcc" if lang == "c" else "g++")
    if cc is None:
        pytest.skip("no host compiler")
    names = _declared()
    src = tmp_path / ("probe.c" if lang == "c" else "probe.cpp")
    src.write_text('#include "sas.h"\nvoid *sas_probe_table[] = {\n' +
                   "".join(f"    (void *)&{n},\n" for n in names) + "};\n")
    r = subprocess.run([cc, std, "-Wall", "-Wextra", "-Werror",
                        "-I", os.path.join(ROOT, "include"), "-c", str(src), "-o", str(tmp_path / "probe.o")],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


_C_CLIENT = r"""
#include <stdio.h>
#include <string.h>
#include "sas.h"

int main(void)
{
    const double coef[9] = {1, 1, 1, 1, 1, 1, 1, 1, 0};
    const double q[3] = {0.0, 0.1, 0.2};
    sas_ctx *ctx = NULL;
    if (strstr(sas_version(), "sm_103a") == NULL) return 1;
    if (sas_create(0, coef, q, 3, SAS_MIXED, &ctx) != SAS_ERR_INVALID_ARG || ctx) return 2;
    if (strlen(sas_last_error()) == 0) return 3;
    if (sas_create(1, coef, q, 3, 1u << 5, &ctx) != SAS_ERR_INVALID_ARG || ctx) return 4;
    if (sas_destroy(NULL) != SAS_OK) return 5;
    if (sas_profile(NULL, NULL, SAS_COORDS_F32, NULL, 0, NULL, NULL) != SAS_ERR_INVALID_ARG) return 6;
    if (sas_exact_sums(NULL, NULL, 0, NULL) != SAS_ERR_INVALID_ARG) return 7;
    printf("ok\n");
    return 0;
}
"""


def test_plain_c_client_links_and_gets_status_codes(tmp_path):
    """A C program linked against libsas.so (no Python) gets the documented status codes from the
    argument checks, which need no GPU."""
    import shutil
    cc = shutil.which("gcc")
    if cc is None:
        pytest.skip("no host compiler")
    lib = _lib.load()._name
    src = tmp_path / "client.c"
    src.write_text(_C_CLIENT)
    exe = tmp_path / "client"
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src), lib,
                        "-Wl,-rpath," + os.path.dirname(lib), "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0 and r.stdout.strip() == "ok", (r.returncode, r.stdout, r.stderr)


def test_guard_band_calls_need_no_gpu_when_nothing_is_guarded():
    """sas_guard_bands validates its switch; with no guarded buffer alive, sas_guard_check and
    sas_guard_list make no CUDA call and report nothing."""
    lib = _lib.load()
    assert lib.sas_guard_bands(2) == _lib.SAS_ERR_INVALID_ARG
    assert lib.sas_guard_bands(0) == _lib.SAS_OK
    assert _lib.sas_guard_check() == 0
    assert _lib.sas_guard_list() == []
    assert lib.sas_guard_list(-1, None, None, None) == _lib.SAS_ERR_INVALID_ARG
