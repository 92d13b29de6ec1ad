"""Eq. 2 with every pair distance replaced by the centre of its histogram bin — TEST INFRASTRUCTURE.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may use
this module; the CUDA library never does.  It is the plain definition of the binned Debye sum, the
learned surrogate's baseline (the paper sums every pair exactly, Section I-A, Eq. 2; this replaces
the distances by bin centres and nothing else):

    I(q) = sum_t n_t f_t(q)^2 + sum_{a<=b} 2 f_a(q) f_b(q) sum_k h[p(a,b)][k] sinc(q r_k),
    r_k = (k + 1/2) r_max / n_bins,  sinc(0) = 1,

in float64, with the per-type form factors of the oracle's C code and a matrix product over bins.
"""
from __future__ import annotations

import numpy as np

from . import form_factors


def profile(hist, type_counts, coef, q, n_bins: int = 256, r_max: float = 120.0) -> np.ndarray:
    """Binned Debye profiles [C, n_q] of histograms hist [C, T(T+1)/2, n_bins] (type pairs
    row-major over a <= b) of molecules with type_counts[t] atoms of type t."""
    coef = np.asarray(coef, dtype=np.float64)
    q = np.asarray(q, dtype=np.float64)
    T = coef.shape[0]
    h = np.asarray(hist, dtype=np.float64).reshape(-1, T * (T + 1) // 2, n_bins)
    F = form_factors(np.arange(T, dtype=np.int32), coef, q)            # [T, n_q]
    nt = np.asarray(type_counts, dtype=np.float64)
    r = (np.arange(n_bins) + 0.5) * (r_max / n_bins)
    x = q[:, None] * r[None, :]
    sinc = np.ones_like(x)
    nz = x != 0.0
    sinc[nz] = np.sin(x[nz]) / x[nz]                                   # [n_q, n_bins]
    out = np.tile(np.sum(nt[:, None] * F * F, axis=0), (h.shape[0], 1))
    p = 0
    for a in range(T):
        for b in range(a, T):
            out += 2.0 * (F[a] * F[b])[None, :] * (h[:, p, :] @ sinc.T)
            p += 1
    return out
