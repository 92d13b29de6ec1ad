"""Python face of the library: a context object and a torch.autograd.Function.

PyTorch provides device memory and streams only; every step of the Debye
computation runs in libsas.so's kernels through the C ABI.
"""
from __future__ import annotations

import numpy as np
import torch

from . import _lib


def _as_tensor_like(x, dtype):
    if isinstance(x, torch.Tensor):
        return x.contiguous() if x.dtype == dtype else x.to(dtype).contiguous()
    return torch.from_numpy(np.ascontiguousarray(x)).to(dtype)


class Profile:
    """I(q) by the Debye sum (Section I-A, Eq. 2) for one set of atom types and q grid.

    ``Profile(coef [T,9], q [Q], precision="mixed"|"fp64", deterministic=False)``.
    Calling it with coordinates [n,3] or [B,n,3] (float32 or float64; CUDA or CPU)
    and types [n] returns float64 I(q) [Q] or [B,Q] on the coordinates' device.
    ``deterministic=True`` makes the gradients bitwise reproducible as well
    (SAS_DETERMINISTIC); every other output is on any context.
    """

    def __init__(self, coef, q, precision: str = "mixed", deterministic: bool = False):
        coef = np.ascontiguousarray(coef, dtype=np.float64)
        self.q = np.ascontiguousarray(q, dtype=np.float64)
        self.n_types = int(coef.shape[0])
        self.coef = coef
        flags = {"mixed": _lib.SAS_MIXED, "fp64": _lib.SAS_FP64}[precision]
        if deterministic:
            flags |= _lib.SAS_DETERMINISTIC
        self.precision = precision
        self._ctx = _lib.sas_create(self.n_types, coef, self.q, flags)
        self._last_batch = 0

    # -- lifetime
    def close(self):
        if getattr(self, "_ctx", None) is not None:
            _lib.sas_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def n_q(self) -> int:
        return int(self.q.size)

    @property
    def n_pairs_types(self) -> int:
        return self.n_types * (self.n_types + 1) // 2

    def set_option(self, option: int, value: int):
        _lib.sas_set_option(self._ctx, option, value)

    def stats(self):
        return _lib.sas_last_stats(self._ctx)

    # -- forward
    def __call__(self, coords, types, stream=None):
        single = coords.ndim == 2
        x = coords.unsqueeze(0) if (single and isinstance(coords, torch.Tensor)) else (
            coords[None] if single else coords)
        if not isinstance(x, torch.Tensor):
            x = torch.from_numpy(np.ascontiguousarray(x))
        x = x.contiguous()
        if x.dtype not in (torch.float32, torch.float64):
            x = x.float()
        B, n = int(x.shape[0]), int(x.shape[1])
        t = _as_tensor_like(types, torch.int32)
        if x.is_cuda and not t.is_cuda:
            t = t.to(x.device)
        ctype = _lib.SAS_COORDS_F64 if x.dtype == torch.float64 else _lib.SAS_COORDS_F32
        out = torch.empty((B, self.n_q), dtype=torch.float64, device=x.device)
        _lib.sas_profile_batch(self._ctx, x, ctype, t, n, B, out, stream)
        self._last_batch = B
        return out[0] if single else out

    def atomic(self, coords, ff, stream=None):
        """I(q) with per-atom form factors ff [n_q, n] (or [B, n_q, n]), f_i(q_k) at ff[..., k, i]:
        Eq. 2 without types (the context's type coefficients are unused).  Returns float64 [Q]
        or [B, Q] on the coordinates' device."""
        single = coords.ndim == 2
        x = coords if isinstance(coords, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(coords))
        if single:
            x = x.unsqueeze(0)
        x = x.contiguous()
        if x.dtype not in (torch.float32, torch.float64):
            x = x.float()
        B, n = int(x.shape[0]), int(x.shape[1])
        f = _as_tensor_like(ff, torch.float64).reshape(B, self.n_q, n)
        if x.is_cuda and not f.is_cuda:
            f = f.to(x.device)
        ctype = _lib.SAS_COORDS_F64 if x.dtype == torch.float64 else _lib.SAS_COORDS_F32
        out = torch.empty((B, self.n_q), dtype=torch.float64, device=x.device)
        _lib.sas_profile_atomic(self._ctx, x, ctype, n, B, f, out, stream)
        self._last_batch = 0
        return out[0] if single else out

    def vjp_atomic(self, coords, ff, grad_I, stream=None):
        """sum_q grad_I[q] dI(q)/dx [n, 3] (or [B, n, 3]) float32 for the per-atom profile of
        ff [n_q, n] (or [B, n_q, n]); the form factors are held fixed (sas_profile_vjp_atomic)."""
        x = coords if isinstance(coords, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(coords))
        single = x.ndim == 2
        if single:
            x = x.unsqueeze(0)
        x = x.to(torch.float32).contiguous()
        B, n = int(x.shape[0]), int(x.shape[1])
        f = _as_tensor_like(ff, torch.float64).reshape(B, self.n_q, n).to(x.device)
        gI = _as_tensor_like(grad_I, torch.float64).reshape(B, self.n_q).to(x.device)
        g = torch.empty((B, n, 3), dtype=torch.float32, device=x.device)
        _lib.sas_profile_vjp_atomic(self._ctx, x, n, B, f, gI, g, stream)
        return g[0] if single else g

    def partials(self):
        """Type-pair sinc sums S[b, p, q] of the last call (float64, host)."""
        S = np.empty((self._last_batch, self.n_pairs_types, self.n_q))
        _lib.sas_partials(self._ctx, S, S.size)
        return S

    def exact_sums(self):
        """The last profile call's exact type-pair sums (SAS_DETERMINISTIC contexts): int64 [B, P, Q, 2],
        (low, high) 64-bit halves of U_p(q) * 2^60 in two's complement (host)."""
        U = np.empty((self._last_batch, self.n_pairs_types, self.n_q, 2), dtype=np.int64)
        _lib.sas_exact_sums(self._ctx, U, U.size)
        return U

    def assemble_exact(self, U, device=None):
        """I(q) [B, Q] (float64) of the whole molecule from exact sums U [B, P, Q, 2] (e.g. summed over
        shards with shard.add_exact), with the type counts of this context's last profile call."""
        U = np.ascontiguousarray(U, dtype=np.int64)
        B = int(U.shape[0])
        out = torch.empty((B, self.n_q), dtype=torch.float64, device=device or "cpu")
        _lib.sas_assemble_exact(self._ctx, U, B, out)
        return out

    # -- adjoint
    def chi2_grad(self, coords, types, target, weights, stream=None):
        """(chi2 [B], d chi2/dx [B,n,3] float32, I [B,Q]) for float32 coordinates [B,n,3]."""
        x = coords if isinstance(coords, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(coords))
        single = x.ndim == 2
        if single:
            x = x.unsqueeze(0)
        x = x.to(torch.float32).contiguous()
        B, n = int(x.shape[0]), int(x.shape[1])
        dev = x.device
        t = _as_tensor_like(types, torch.int32).to(dev)
        tg = _as_tensor_like(target, torch.float64).to(dev)
        w = _as_tensor_like(weights, torch.float64).to(dev)
        chi2 = torch.empty(B, dtype=torch.float64, device=dev)
        g = torch.empty((B, n, 3), dtype=torch.float32, device=dev)
        I = torch.empty((B, self.n_q), dtype=torch.float64, device=dev)
        _lib.sas_profile_grad(self._ctx, x, t, n, B, tg, w, chi2, g, I, stream)
        if single:
            return chi2[0], g[0], I[0]
        return chi2, g, I

    def vjp(self, coords, types, grad_I, stream=None):
        x = coords.to(torch.float32).contiguous()
        single = x.ndim == 2
        if single:
            x = x.unsqueeze(0)
        gI = grad_I.to(torch.float64).contiguous()
        if gI.ndim == 1:
            gI = gI.unsqueeze(0)
        B, n = int(x.shape[0]), int(x.shape[1])
        t = _as_tensor_like(types, torch.int32).to(x.device)
        g = torch.empty((B, n, 3), dtype=torch.float32, device=x.device)
        _lib.sas_profile_vjp(self._ctx, x, t, n, B, gI.to(x.device), g, stream)
        return g[0] if single else g

    # -- histogram
    def pair_histogram(self, coords, types, n_bins: int = 256, r_max: float = 120.0, stream=None):
        """(hist [B, P, n_bins] int32, dropped [B] int64) of unordered pair distances."""
        x = coords if isinstance(coords, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(coords))
        single = x.ndim == 2
        if single:
            x = x.unsqueeze(0)
        x = x.to(torch.float32).contiguous()
        B, n = int(x.shape[0]), int(x.shape[1])
        t = _as_tensor_like(types, torch.int32).to(x.device)
        h = torch.empty((B, self.n_pairs_types, n_bins), dtype=torch.int32, device=x.device)
        d = torch.empty(B, dtype=torch.int64, device=x.device)
        _lib.sas_pair_histogram(self._ctx, x, t, n, B, n_bins, r_max, h, d, stream)
        return (h[0], d[0]) if single else (h, d)


    def binned(self, hist, type_counts, n_bins: int = 256, r_max: float = 120.0, stream=None):
        """Binned Debye profiles [B, n_q] float64 of pair histograms hist [B, P, n_bins] (every pair at
        its bin centre; sas_binned_profile) of molecules with type_counts[t] atoms of type t."""
        h = hist if isinstance(hist, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(hist))
        single = h.ndim == 2
        if single:
            h = h.unsqueeze(0)
        h = h.to(torch.int32).contiguous()
        B = int(h.shape[0])
        out = torch.empty((B, self.n_q), dtype=torch.float64, device=h.device)
        _lib.sas_binned_profile(self._ctx, h, B, n_bins, r_max, np.asarray(type_counts, np.int64), out, stream)
        return out[0] if single else out


class DebyeFunction(torch.autograd.Function):
    """I = DebyeFunction.apply(coords, profile, types): differentiable in coords.

    The backward is the vector-Jacobian product of Eq. 2 computed by the
    adjoint kernel (sas_profile_vjp)."""

    @staticmethod
    def forward(ctx, coords, profile: Profile, types):
        ctx.profile = profile
        ctx.types = types
        ctx.save_for_backward(coords)
        return profile(coords.detach(), types)

    @staticmethod
    def backward(ctx, grad_I):
        (coords,) = ctx.saved_tensors
        g = ctx.profile.vjp(coords.detach(), ctx.types, grad_I.contiguous())
        return g.to(coords.dtype), None, None
