"""FP64 CPU oracle for the Debye summation (Section I-A, Eq. 2) — TEST INFRASTRUCTURE.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library never does, and this
package imports nothing from it: the two share no code.

The numerical work is in ``debye_oracle.c`` (plain double loops, libm, Neumaier
sums; built by ``make`` into ``_build/liboracle.so``).  The MLP reference is
``mlp.py`` (NumPy float64).  This module only marshals NumPy arrays.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

_i64 = ctypes.c_int64
_i32 = ctypes.c_int
_dp = ctypes.POINTER(ctypes.c_double)
_fp = ctypes.POINTER(ctypes.c_float)
_ip = ctypes.POINTER(ctypes.c_int32)
_lp = ctypes.POINTER(ctypes.c_int64)


def build() -> str:
    """Compile the oracle with ``make`` (idempotent) and return the library path."""
    subprocess.run(["make", "-s", "-C", _HERE], check=True)
    return _LIB_PATH


def _configure(lib):
    """Declare the C signatures on a loaded oracle library."""
    lib.oracle_max_threads.restype = _i32
    lib.oracle_form_factors.argtypes = [_i64, _ip, _i32, _dp, _i32, _dp, _dp]
    lib.oracle_profile.argtypes = [_i64, _dp, _ip, _i32, _dp, _i32, _dp, _i32, _dp, _dp]
    lib.oracle_profile_full.argtypes = [_i64, _dp, _ip, _i32, _dp, _i32, _dp, _dp]
    lib.oracle_profile_atomic.argtypes = [_i64, _dp, _dp, _i32, _dp, _i32, _dp, _dp]
    lib.oracle_pair_sums.argtypes = [_i64, _dp, _ip, _i32, _i32, _dp, _i32, _dp]
    lib.oracle_vjp.argtypes = [_i64, _dp, _ip, _i32, _dp, _i32, _dp, _dp, _i32, _dp]
    lib.oracle_vjp_atomic.argtypes = [_i64, _dp, _dp, _i32, _dp, _dp, _i32, _dp]
    lib.oracle_chi2_grad.argtypes = [_i64, _dp, _ip, _i32, _dp, _i32, _dp, _dp, _dp, _i32,
                                     _dp, _dp, _dp]
    lib.oracle_pair_histogram.argtypes = [_i64, _fp, _ip, _i32, _i32, ctypes.c_float, _ip, _lp]
    for f in ("oracle_form_factors", "oracle_profile", "oracle_profile_full", "oracle_profile_atomic",
              "oracle_pair_sums", "oracle_vjp", "oracle_vjp_atomic", "oracle_chi2_grad", "oracle_pair_histogram"):
        getattr(lib, f).restype = _i32
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = _configure(ctypes.CDLL(_LIB_PATH))
    return _lib


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_dp)


def _t(types):
    t = np.ascontiguousarray(types, dtype=np.int32)
    return t, t.ctypes.data_as(_ip)


def _check(rc: int, what: str):
    if rc == -1:
        raise ValueError(f"{what}: atom type out of range or bad argument")
    if rc != 0:
        raise MemoryError(f"{what}: allocation failed ({rc})")


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def form_factors(types, coef, q) -> np.ndarray:
    """f[i, k] = f_{type(i)}(q_k), per atom."""
    lib = _load()
    t, tp = _t(types)
    c, cp = _d(coef)
    qq, qp = _d(q)
    out = np.empty((t.size, qq.size))
    _check(lib.oracle_form_factors(t.size, tp, c.shape[0], cp, qq.size, qp,
                                   out.ctypes.data_as(_dp)), "form_factors")
    return out


def profile(coords, types, coef, q, n_threads: int = 0, with_kappa: bool = False):
    """I(q) by Eq. 2 over i<j plus the diagonal, float64.  Coordinates are
    promoted to float64 exactly (a float32 input is used as its exact value)."""
    lib = _load()
    x, xp = _d(np.asarray(coords).reshape(-1, 3))
    t, tp = _t(types)
    c, cp = _d(coef)
    qq, qp = _d(q)
    I = np.empty(qq.size)
    kap = np.empty(qq.size)
    _check(lib.oracle_profile(x.shape[0], xp, tp, c.shape[0], cp, qq.size, qp, n_threads,
                              I.ctypes.data_as(_dp), kap.ctypes.data_as(_dp)), "profile")
    return (I, kap) if with_kappa else I


def profile_atomic(coords, ff, q, n_threads: int = 0, with_kappa: bool = False):
    """I(q) by Eq. 2 with per-atom form factors ff[k, i] = f_i(q_k) (shape [n_q, n]), float64."""
    lib = _load()
    x, xp = _d(np.asarray(coords).reshape(-1, 3))
    qq, qp = _d(q)
    f, fp = _d(np.asarray(ff).reshape(qq.size, x.shape[0]))
    I = np.empty(qq.size)
    kap = np.empty(qq.size)
    _check(lib.oracle_profile_atomic(x.shape[0], xp, fp, qq.size, qp, n_threads,
                                     I.ctypes.data_as(_dp), kap.ctypes.data_as(_dp)), "profile_atomic")
    return (I, kap) if with_kappa else I


def profile_full(coords, types, coef, q) -> np.ndarray:
    """Eq. 2 literally: all N x N ordered pairs including the diagonal (small N)."""
    lib = _load()
    x, xp = _d(np.asarray(coords).reshape(-1, 3))
    t, tp = _t(types)
    c, cp = _d(coef)
    qq, qp = _d(q)
    I = np.empty(qq.size)
    _check(lib.oracle_profile_full(x.shape[0], xp, tp, c.shape[0], cp, qq.size, qp,
                                   I.ctypes.data_as(_dp)), "profile_full")
    return I


def pair_sums(coords, types, n_types: int, q, n_threads: int = 0) -> np.ndarray:
    """S[p, k] = sum over unordered pairs of type pair p of sinc(q_k r), p row-major over a<=b."""
    lib = _load()
    x, xp = _d(np.asarray(coords).reshape(-1, 3))
    t, tp = _t(types)
    qq, qp = _d(q)
    P = n_types * (n_types + 1) // 2
    S = np.empty((P, qq.size))
    _check(lib.oracle_pair_sums(x.shape[0], xp, tp, n_types, qq.size, qp, n_threads,
                                S.ctypes.data_as(_dp)), "pair_sums")
    return S


def vjp(coords, types, coef, q, grad_I, n_threads: int = 0) -> np.ndarray:
    """sum_q grad_I[q] dI(q)/dx, shape [n, 3]."""
    lib = _load()
    x, xp = _d(np.asarray(coords).reshape(-1, 3))
    t, tp = _t(types)
    c, cp = _d(coef)
    qq, qp = _d(q)
    g, gp = _d(grad_I)
    out = np.empty_like(x)
    _check(lib.oracle_vjp(x.shape[0], xp, tp, c.shape[0], cp, qq.size, qp, gp, n_threads,
                          out.ctypes.data_as(_dp)), "vjp")
    return out


def vjp_atomic(coords, ff, q, grad_I, n_threads: int = 0) -> np.ndarray:
    """sum_q grad_I[q] dI(q)/dx [n, 3] with per-atom form factors ff[k, i] = f_i(q_k)."""
    lib = _load()
    x, xp = _d(np.asarray(coords).reshape(-1, 3))
    qq, qp = _d(q)
    f, fp = _d(np.asarray(ff).reshape(qq.size, x.shape[0]))
    g, gp = _d(grad_I)
    out = np.empty_like(x)
    _check(lib.oracle_vjp_atomic(x.shape[0], xp, fp, qq.size, qp, gp, n_threads, out.ctypes.data_as(_dp)),
           "vjp_atomic")
    return out


def chi2_grad(coords, types, coef, q, target, weights, n_threads: int = 0, grad: bool = True):
    """(chi2, d chi2/dx [n,3] or None, I) with chi2 = sum_q w_q (I(q) - T(q))^2."""
    lib = _load()
    x, xp = _d(np.asarray(coords).reshape(-1, 3))
    t, tp = _t(types)
    c, cp = _d(coef)
    qq, qp = _d(q)
    tg, tgp = _d(target)
    w, wp = _d(weights)
    chi2 = ctypes.c_double(0.0)
    g = np.empty_like(x) if grad else None
    I = np.empty(qq.size)
    _check(lib.oracle_chi2_grad(x.shape[0], xp, tp, c.shape[0], cp, qq.size, qp, tgp, wp,
                                n_threads, ctypes.byref(chi2),
                                g.ctypes.data_as(_dp) if grad else None,
                                I.ctypes.data_as(_dp)), "chi2_grad")
    return chi2.value, g, I


def pair_histogram(coords_f32, types, n_types: int, n_bins: int = 256, r_max: float = 120.0):
    """(hist [P, n_bins] int32, dropped) of unordered pairs by type pair and float32 distance bin."""
    lib = _load()
    x = np.ascontiguousarray(np.asarray(coords_f32).reshape(-1, 3), dtype=np.float32)
    t, tp = _t(types)
    P = n_types * (n_types + 1) // 2
    h = np.empty((P, n_bins), dtype=np.int32)
    dropped = ctypes.c_int64(0)
    _check(lib.oracle_pair_histogram(x.shape[0], x.ctypes.data_as(_fp), tp, n_types, n_bins,
                                     ctypes.c_float(r_max), h.ctypes.data_as(_ip),
                                     ctypes.byref(dropped)), "pair_histogram")
    return h, int(dropped.value)


def pair_index(a: int, b: int, n_types: int) -> int:
    a, b = min(a, b), max(a, b)
    return a * n_types - a * (a - 1) // 2 + (b - a)
