"""ctypes binding of libsas.so: the C ABI of include/sas.h under the same names.

Argument marshalling only: every array argument may be a torch tensor (CPU or
CUDA) or a NumPy array; it is passed as a raw pointer.  Streams are torch
streams (or None for the current torch stream).  A non-OK status raises
SasError carrying the status and the library's message.  There is no CPU
fallback: if the library cannot be built or loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import threading

import numpy as np

from . import build as _build

SAS_OK, SAS_ERR_INVALID_ARG, SAS_ERR_CUDA, SAS_ERR_ALLOC, SAS_ERR_UNSUPPORTED, SAS_ERR_TIMEOUT, SAS_ERR_CORRUPT = range(7)
STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "CUDA", 3: "ALLOC", 4: "UNSUPPORTED", 5: "TIMEOUT", 6: "CORRUPT"}
SAS_MIXED, SAS_FP64 = 0, 1
SAS_DETERMINISTIC = 16
SAS_COORDS_F32, SAS_COORDS_F64 = 0, 1
SAS_OPT_JMAX, SAS_OPT_RESEED, SAS_OPT_VALIDATE, SAS_OPT_GRID, SAS_OPT_TIMEOUT_MS, SAS_OPT_STEP, SAS_OPT_VARIANT = 1, 2, 3, 4, 5, 6, 7
SAS_OPT_SHARD, SAS_OPT_METHOD, SAS_OPT_ADJOINT, SAS_OPT_COEF = 8, 9, 10, 11
SAS_MAX_TYPES, SAS_MAX_Q = 16, 1664
(SAS_MLP_BUF_XB, SAS_MLP_BUF_Z1, SAS_MLP_BUF_A1B, SAS_MLP_BUF_Z2, SAS_MLP_BUF_A2B, SAS_MLP_BUF_Y, SAS_MLP_BUF_DY,
 SAS_MLP_BUF_DYB, SAS_MLP_BUF_DA2, SAS_MLP_BUF_DZ2, SAS_MLP_BUF_DZ2B, SAS_MLP_BUF_DA1, SAS_MLP_BUF_DZ1,
 SAS_MLP_BUF_DZ1B, SAS_MLP_BUF_COUNT) = range(15)

# every symbol include/sas.h declares (checked by the test suite)
EXPORTS = (
    "sas_create", "sas_destroy", "sas_profile", "sas_profile_batch", "sas_profile_grad",
    "sas_profile_vjp", "sas_partials", "sas_pair_histogram", "sas_set_option", "sas_last_stats",
    "sas_last_error", "sas_version", "sas_profile_static", "sas_mlp_create", "sas_mlp_destroy",
    "sas_mlp_param_count", "sas_mlp_set_state", "sas_mlp_get_state", "sas_mlp_forward", "sas_mlp_train_step",
    "sas_mlp_grads", "sas_gemm_bf16", "sas_screen_select", "sas_gather_rows", "sas_profile_atomic",
    "sas_measure_peaks", "sas_exact_sums", "sas_assemble_exact", "sas_mlp_read_buffer",
    "sas_binned_profile", "sas_profile_vjp_atomic", "sas_guard_bands", "sas_guard_check", "sas_guard_list",
)


class SasError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status
        self.message = message


_lock = threading.Lock()
_lib = None
_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_int = ctypes.c_int


def load():
    """Build (if stale) and load libsas.so; raises if either fails."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            lib = ctypes.CDLL(path)
            sig = {
                "sas_create": [_int, _vp, _vp, _int, ctypes.c_uint, ctypes.POINTER(_vp)],
                "sas_destroy": [_vp],
                "sas_profile": [_vp, _vp, _int, _vp, _i64, _vp, _vp],
                "sas_profile_batch": [_vp, _vp, _int, _vp, _i64, _i64, _vp, _vp],
                "sas_profile_grad": [_vp, _vp, _vp, _i64, _i64, _vp, _vp, _vp, _vp, _vp, _vp],
                "sas_profile_vjp": [_vp, _vp, _vp, _i64, _i64, _vp, _vp, _vp],
                "sas_partials": [_vp, _vp, _i64, _vp],
                "sas_pair_histogram": [_vp, _vp, _vp, _i64, _i64, _int, ctypes.c_float, _vp, _vp, _vp],
                "sas_set_option": [_vp, _int, _i64],
                "sas_last_stats": [_vp, _vp, _int],
                "sas_profile_static": [_vp, _vp, _i64, _int, _vp, ctypes.c_double, ctypes.c_double, _int,
                                       _vp, _vp],
                "sas_mlp_create": [_int, _int, _int, _int, ctypes.POINTER(_vp)],
                "sas_mlp_destroy": [_vp],
                "sas_mlp_set_state": [_vp, _vp, _vp, _vp, _i64],
                "sas_mlp_get_state": [_vp, _vp, _vp, _vp, _vp],
                "sas_mlp_forward": [_vp, _vp, _int, _vp, _vp],
                "sas_mlp_train_step": [_vp, _vp, _vp, _int, ctypes.c_float, _vp, _vp],
                "sas_mlp_grads": [_vp, _vp, _vp, _int, _vp, _vp, _vp],
                "sas_mlp_read_buffer": [_vp, _int, _int, _vp, _vp],
                "sas_gemm_bf16": [_int, _int, _int, _vp, _int, _vp, _int, _vp, _vp, _int, _vp],
                "sas_screen_select": [_int, _int, _vp, _int, _vp, _vp, _vp, _int, _vp, _vp, _int, _vp, _vp, _vp,
                                      _vp],
                "sas_gather_rows": [_vp, _i64, _vp, _i64, _vp, _vp],
                "sas_profile_atomic": [_vp, _vp, _int, _i64, _i64, _vp, _vp, _vp],
                "sas_measure_peaks": [_vp, _int, _vp],
                "sas_exact_sums": [_vp, _vp, _i64, _vp],
                "sas_assemble_exact": [_vp, _vp, _i64, _vp, _vp],
                "sas_binned_profile": [_vp, _vp, _i64, _int, ctypes.c_float, _vp, _vp, _vp],
                "sas_profile_vjp_atomic": [_vp, _vp, _i64, _i64, _vp, _vp, _vp, _vp],
                "sas_guard_bands": [_int],
                "sas_guard_check": [_vp],
                "sas_guard_list": [_i64, _vp, _vp, _vp],
            }
            for name, args in sig.items():
                f = getattr(lib, name)
                f.argtypes = args
                f.restype = _int
            lib.sas_last_error.restype = ctypes.c_char_p
            lib.sas_last_error.argtypes = []
            lib.sas_version.restype = ctypes.c_char_p
            lib.sas_version.argtypes = []
            lib.sas_mlp_param_count.restype = _i64
            lib.sas_mlp_param_count.argtypes = [_vp]
            _lib = lib
    return _lib


def ptr(x):
    """Raw address of a torch tensor / NumPy array (None -> NULL).  Must be contiguous."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    if isinstance(x, int):
        return x
    raise TypeError(f"cannot pass {type(x).__name__} as a pointer")


def stream_handle(stream=None):
    """cudaStream_t of a torch stream (default: torch's current stream), or 0 without CUDA."""
    import torch
    if stream is None:
        if not torch.cuda.is_available():
            return None
        stream = torch.cuda.current_stream()
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def check(status: int):
    if status != SAS_OK:
        raise SasError(status, load().sas_last_error().decode())


# ---- the C ABI under its own names ---------------------------------------------------------

def sas_create(n_types: int, ff_coef, q, flags: int = SAS_MIXED):
    lib = load()
    c = np.ascontiguousarray(ff_coef, dtype=np.float64)
    qq = np.ascontiguousarray(q, dtype=np.float64)
    h = _vp()
    check(lib.sas_create(int(n_types), c.ctypes.data, qq.ctypes.data, int(qq.size), int(flags),
                         ctypes.byref(h)))
    return h


def sas_destroy(ctx):
    check(load().sas_destroy(ctx))


def sas_profile(ctx, coords, coords_type, types, n_atoms, I_out, stream=None):
    check(load().sas_profile(ctx, ptr(coords), int(coords_type), ptr(types), int(n_atoms), ptr(I_out),
                             stream_handle(stream)))


def sas_profile_batch(ctx, coords, coords_type, types, n_atoms, batch, I_out, stream=None):
    check(load().sas_profile_batch(ctx, ptr(coords), int(coords_type), ptr(types), int(n_atoms),
                                   int(batch), ptr(I_out), stream_handle(stream)))


def sas_profile_grad(ctx, coords, types, n_atoms, batch, target, weights, chi2_out, grad_out,
                     I_out=None, stream=None):
    check(load().sas_profile_grad(ctx, ptr(coords), ptr(types), int(n_atoms), int(batch), ptr(target),
                                  ptr(weights), ptr(chi2_out), ptr(grad_out), ptr(I_out),
                                  stream_handle(stream)))


def sas_profile_vjp(ctx, coords, types, n_atoms, batch, grad_I, grad_out, stream=None):
    check(load().sas_profile_vjp(ctx, ptr(coords), ptr(types), int(n_atoms), int(batch), ptr(grad_I),
                                 ptr(grad_out), stream_handle(stream)))


def sas_profile_atomic(ctx, coords, coords_type, n_atoms, batch, ff, I_out, stream=None):
    check(load().sas_profile_atomic(ctx, ptr(coords), int(coords_type), int(n_atoms), int(batch), ptr(ff),
                                    ptr(I_out), stream_handle(stream)))


def sas_partials(ctx, S_out, capacity, stream=None):
    check(load().sas_partials(ctx, ptr(S_out), int(capacity), stream_handle(stream)))


def sas_exact_sums(ctx, U_out, capacity, stream=None):
    check(load().sas_exact_sums(ctx, ptr(U_out), int(capacity), stream_handle(stream)))


def sas_assemble_exact(ctx, U, batch, I_out, stream=None):
    check(load().sas_assemble_exact(ctx, ptr(U), int(batch), ptr(I_out), stream_handle(stream)))


def sas_pair_histogram(ctx, coords, types, n_atoms, batch, n_bins, r_max, hist_out, dropped_out=None,
                       stream=None):
    check(load().sas_pair_histogram(ctx, ptr(coords), ptr(types), int(n_atoms), int(batch), int(n_bins),
                                    float(r_max), ptr(hist_out), ptr(dropped_out), stream_handle(stream)))


def sas_set_option(ctx, option: int, value: int):
    check(load().sas_set_option(ctx, int(option), int(value)))


def sas_last_stats(ctx):
    out = np.zeros(9, dtype=np.int64)
    check(load().sas_last_stats(ctx, out.ctypes.data, 9))
    return out


def sas_profile_static(coords, types, n_atoms, n_types, ff_coef, q0, dq, n_q, I_out, stream=None):
    """Allocation-free profile (device coords/types/I_out, host coefficients); status codes only."""
    c = np.ascontiguousarray(ff_coef, dtype=np.float64)
    st = load().sas_profile_static(ptr(coords), ptr(types), int(n_atoms), int(n_types), c.ctypes.data,
                                   float(q0), float(dq), int(n_q), ptr(I_out), stream_handle(stream))
    if st != SAS_OK:
        raise SasError(st, "sas_profile_static failed")


def sas_profile_vjp_atomic(ctx, coords, n_atoms, batch, ff, grad_I, grad_out, stream=None):
    check(load().sas_profile_vjp_atomic(ctx, ptr(coords), int(n_atoms), int(batch), ptr(ff), ptr(grad_I),
                                        ptr(grad_out), stream_handle(stream)))


def sas_binned_profile(ctx, hist, batch, n_bins, r_max, type_counts, I_out, stream=None):
    """Debye sum over pair-distance histograms at bin centres (hist [batch][P][n_bins] int32)."""
    tc = np.ascontiguousarray(type_counts, dtype=np.int64)
    check(load().sas_binned_profile(ctx, ptr(hist), int(batch), int(n_bins), float(r_max), tc.ctypes.data, ptr(I_out),
                                    stream_handle(stream)))


def sas_mlp_create(n_in, n_hidden, n_out, max_batch):
    h = _vp()
    check(load().sas_mlp_create(int(n_in), int(n_hidden), int(n_out), int(max_batch), ctypes.byref(h)))
    return h


def sas_mlp_destroy(mlp):
    check(load().sas_mlp_destroy(mlp))


def sas_mlp_param_count(mlp) -> int:
    return int(load().sas_mlp_param_count(mlp))


def sas_mlp_set_state(mlp, params, adam_m=None, adam_v=None, step=0):
    check(load().sas_mlp_set_state(mlp, ptr(params), ptr(adam_m), ptr(adam_v), int(step)))


def sas_mlp_get_state(mlp, params, adam_m=None, adam_v=None):
    st = ctypes.c_int64(0)
    check(load().sas_mlp_get_state(mlp, ptr(params), ptr(adam_m), ptr(adam_v), ctypes.byref(st)))
    return int(st.value)


def sas_mlp_forward(mlp, x, batch, y, stream=None):
    check(load().sas_mlp_forward(mlp, ptr(x), int(batch), ptr(y), stream_handle(stream)))


def sas_mlp_train_step(mlp, x, t, batch, lr, loss_out=None, stream=None):
    check(load().sas_mlp_train_step(mlp, ptr(x), ptr(t), int(batch), float(lr), ptr(loss_out),
                                    stream_handle(stream)))


def sas_mlp_grads(mlp, x, t, batch, grads, loss_out=None, stream=None):
    check(load().sas_mlp_grads(mlp, ptr(x), ptr(t), int(batch), ptr(grads), ptr(loss_out), stream_handle(stream)))


def sas_mlp_read_buffer(mlp, which, batch, out):
    """Rows [0, batch) of intermediate tensor `which` (SAS_MLP_BUF_*) into out (float32); returns its width."""
    w = ctypes.c_int(0)
    check(load().sas_mlp_read_buffer(mlp, int(which), int(batch), ptr(out), ctypes.byref(w)))
    return int(w.value)


def sas_gemm_bf16(M, N, K, A, lda, B, ldb, bias, C, ldc, stream=None):
    check(load().sas_gemm_bf16(int(M), int(N), int(K), ptr(A), int(lda), ptr(B), int(ldb), ptr(bias), ptr(C),
                               int(ldc), stream_handle(stream)))


def sas_screen_select(n_conf, n_q, z, ld, mean, stdv, base, ld_base, target, weights, k, top_idx, top_chi2,
                      chi2_all, stream=None):
    check(load().sas_screen_select(int(n_conf), int(n_q), ptr(z), int(ld), ptr(mean), ptr(stdv), ptr(base),
                                   int(ld_base), ptr(target), ptr(weights), int(k), ptr(top_idx), ptr(top_chi2),
                                   ptr(chi2_all), stream_handle(stream)))


def sas_gather_rows(src, row_bytes, idx, n_idx, dst, stream=None):
    check(load().sas_gather_rows(ptr(src), int(row_bytes), ptr(idx), int(n_idx), ptr(dst), stream_handle(stream)))


def sas_measure_peaks(stream=None) -> dict:
    """Measured peaks of the current device: FP32 FMA and packed-FMA lane-ops/s, MUFU sine ops/s,
    FP64 FMA lane-ops/s, the SM clock (MHz) of the FMA run, conflict-free shared-memory integer
    atomic adds/s, and packed-FMA lane-ops/s with three distinct source register pairs."""
    out = np.zeros(7)
    check(load().sas_measure_peaks(out.ctypes.data, 7, stream_handle(stream)))
    return {"ffma": float(out[0]), "ffma2": float(out[1]), "mufu_sin": float(out[2]), "dfma": float(out[3]),
            "sm_mhz": float(out[4]), "atoms_shared": float(out[5]), "ffma2_3op": float(out[6])}


def sas_last_error() -> str:
    return load().sas_last_error().decode()


def sas_guard_bands(enable: bool):
    """Guard bands around device buffers allocated from now on (on) or not (off)."""
    check(load().sas_guard_bands(1 if enable else 0))


def sas_guard_check() -> int:
    """Compare every band of every live guarded buffer with its pattern; returns the number of
    buffers checked, raises SasError (SAS_ERR_CORRUPT) if a band was overwritten."""
    n = ctypes.c_int64(0)
    check(load().sas_guard_check(ctypes.byref(n)))
    return int(n.value)


def sas_guard_list():
    """[(device address, bytes)] of the live guarded buffers."""
    lib = load()
    n = ctypes.c_int64(0)
    check(lib.sas_guard_list(0, None, None, ctypes.byref(n)))
    cap = int(n.value)
    ptrs = (ctypes.c_void_p * max(cap, 1))()
    sizes = np.zeros(max(cap, 1), dtype=np.int64)
    check(lib.sas_guard_list(cap, ptrs, sizes.ctypes.data, ctypes.byref(n)))
    k = min(cap, int(n.value))
    return [(int(ptrs[i]), int(sizes[i])) for i in range(k)]


def sas_version() -> str:
    return load().sas_version().decode()
