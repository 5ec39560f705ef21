"""Python binding of libpttk (include/pttk.h): argument marshalling only.

Every computation runs in the CUDA library; this module converts torch tensors to
device pointers, checks shapes and dtypes, and turns status codes into exceptions.
It raises if libpttk.so has not been built: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpttk.so")

OK, EINVAL, EDOMAIN, ENOMEM, ECUDA, ETIMEOUT, ENOTSUP = range(7)
STATUS_NAMES = {0: "PTTK_OK", 1: "PTTK_EINVAL", 2: "PTTK_EDOMAIN", 3: "PTTK_ENOMEM",
                4: "PTTK_ECUDA", 5: "PTTK_ETIMEOUT", 6: "PTTK_ENOTSUP"}
GAUSS, MATERN32, MATERN_NU = 0, 1, 2
EXPONENTIAL, MATERN52, MULTIQUADRIC, THIN_PLATE_SPLINE = 3, 4, 5, 6
BIHARMONIC, LAPLACE3D, LAPLACE2D, THIN_PLATE = 7, 8, 9, 10      # no parameter (d_theta = 0)
FP64, FP32, TF32, TF32X3, BF16, BF16X3, FP16, FP16X3 = range(8)
PREC_NAMES = {"fp64": FP64, "fp32": FP32, "tf32": TF32, "tf32x3": TF32X3, "bf16": BF16, "bf16x3": BF16X3,
              "fp16": FP16, "fp16x3": FP16X3}

_c_double_p = ctypes.POINTER(ctypes.c_double)
_c_int_p = ctypes.POINTER(ctypes.c_int)
_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_int = ctypes.c_int

# (name, restype, argtypes) for every entry point of include/pttk.h
SIGNATURES = [
    ("pttk_last_error", ctypes.c_char_p, []),
    ("pttk_version", _int, []),
    ("pttk_grid_coeffs", _int, [_int, _int, _c_double_p, _c_double_p, _int, _c_double_p, _int, _int, _vp, _vp]),
    ("pttk_grid_entries", _int, [_int, _int, _c_double_p, _c_double_p, _int, _c_double_p, _int, _vp, _i64,
                                 _int, _vp, _vp]),
    ("pttk_tt_from_coeffs", _int, [_int, _int, _c_double_p, _c_double_p, _int, _c_double_p, _int,
                                   ctypes.c_double, _vp, _int, _vp, ctypes.POINTER(_vp)]),
    ("pttk_build_offline", _int, [_int, _int, _c_double_p, _c_double_p, _int, _c_double_p, _int,
                                  ctypes.c_double, _int, _vp, ctypes.POINTER(_vp)]),
    ("pttk_tt_dims", _int, [_vp, _c_int_p, _c_int_p, _c_int_p, _c_int_p]),
    ("pttk_tt_ranks", _int, [_vp, _c_int_p]),
    ("pttk_tt_get_core", _int, [_vp, _int, _c_double_p]),
    ("pttk_tt_save", _int, [_vp, ctypes.c_char_p]),
    ("pttk_tt_load", _int, [ctypes.c_char_p, ctypes.POINTER(_vp)]),
    ("pttk_tt_round", _int, [_vp, ctypes.c_double, _vp, ctypes.POINTER(_vp)]),
    ("pttk_tt_from_cores", _int, [_int, _int, _c_double_p, _c_double_p, _int, _c_double_p, _int, _c_int_p,
                                  _c_double_p, ctypes.POINTER(_vp)]),
    ("pttk_tt_free", None, [_vp]),
    ("pttk_theta_core", _int, [_vp, _c_double_p, _int, _vp, _vp]),
    ("pttk_tt_check", _int, [_vp, _vp]),
    ("pttk_instantiate", _int, [_vp, _c_double_p, _vp, _i64, _vp, _i64, _int, _vp, _vp, _vp, _vp]),
    ("pttk_apply", _int, [_vp, _vp, _vp, _i64, _i64, _int, _int, _int, _vp, _vp, _vp]),
    ("pttk_batch_create", _int, [_vp, _int, ctypes.POINTER(_i64), ctypes.POINTER(_i64), _int, _vp,
                                 ctypes.POINTER(_vp)]),
    ("pttk_batch_free", None, [_vp]),
    ("pttk_batch_set_config", _int, [_vp, _int]),
    ("pttk_batch_get_config", _int, [_vp, _c_int_p, _c_int_p]),
    ("pttk_batch_autotune", _int, [_vp, _vp, _vp, _vp, _vp, ctypes.POINTER(ctypes.c_float), _vp]),
    ("pttk_instantiate_batched", _int, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    ("pttk_grad", _int, [_vp, _c_double_p, _vp, _i64, _vp, _i64, _vp, _vp, _int, _c_double_p, _c_double_p,
                         _vp, _vp]),
    ("pttk_apply_noalloc", _int, [_vp, _vp, _vp, _i64, _i64, _int, _int, _int, _vp, _vp, _vp]),
    ("pttk_profile_enable", _int, [_int]),
    ("pttk_profile_reset", _int, []),
    ("pttk_profile_get", _int, [ctypes.c_char_p, _c_double_p, ctypes.POINTER(_i64)]),
    ("pttk_profile_names", _int, [ctypes.c_char_p, _i64]),
    ("pttk_launch_count", _i64, []),
    ("pttk_selftest_wait_timeout", _int, [_vp]),
    ("pttk_global_create", _int, [_vp, _vp, _i64, _vp, ctypes.POINTER(_vp)]),
    ("pttk_global_dims", _int, [_vp, ctypes.POINTER(_i64), _c_int_p, _c_int_p, _c_int_p]),
    ("pttk_global_get_q", _int, [_vp, _vp, _vp]),
    ("pttk_global_get_r", _int, [_vp, _c_double_p]),
    ("pttk_global_instantiate", _int, [_vp, _c_double_p, ctypes.c_double, _int, _int, _vp, _vp, _c_int_p, _vp]),
    ("pttk_global_instantiate_batched", _int, [_vp, _int, _c_double_p, _int, _vp, _vp]),
    ("pttk_global_free", None, [_vp]),
    ("pttk_splitmix64", ctypes.c_uint64, [ctypes.c_uint64, ctypes.c_uint64]),
    ("pttk_peak_probe", _int, [_int, _i64, _vp, _c_double_p, _c_double_p]),
    ("pttk_fixed_create", _int, [_vp, _vp, _i64, _vp, _i64, ctypes.c_double, _vp, ctypes.POINTER(_vp)]),
    ("pttk_fixed_dims", _int, [_vp, ctypes.POINTER(_i64), ctypes.POINTER(_i64), _c_int_p, _c_int_p]),
    ("pttk_fixed_get_factors", _int, [_vp, _vp, _vp, _vp]),
    ("pttk_fixed_get_core", _int, [_vp, _int, _c_double_p]),
    ("pttk_fixed_theta_core", _int, [_vp, _c_double_p, _int, _vp, _vp]),
    ("pttk_fixed_free", None, [_vp]),
    ("pttk_gp_kv", _int, [_int, _int, _vp, _i64, _c_double_p, ctypes.c_double, _vp, _vp, _int, _vp]),
    ("pttk_gp_pcg", _int, [_int, _int, _vp, _i64, _c_double_p, ctypes.c_double, _vp, _vp, _int, _vp, _vp,
                           ctypes.c_double, _int, _int, _c_int_p, _c_double_p, _vp]),
    ("pttk_gp_lml", _int, [_vp, _c_double_p, ctypes.c_double, _vp, _c_double_p, _c_double_p, _vp]),
    ("pttk_cross_build", _int, [_int, _int, _c_double_p, _c_double_p, _int, _c_double_p, _int, ctypes.c_double,
                                ctypes.c_uint64, _int, _int, _int, _vp, ctypes.POINTER(_vp), _c_int_p,
                                ctypes.POINTER(_i64)]),
]

_lib = None


class PttkError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libpttk.so (built by paper_2406_06344_gb300._build); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_2406_06344_gb300._build.build()")
    lib = ctypes.CDLL(path)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(status: int):
    if status != OK:
        raise PttkError(status, load().pttk_last_error().decode())


def _dbl(values: Sequence[float]):
    arr = (ctypes.c_double * max(1, len(values)))(*[float(v) for v in values])
    return arr


def _boxflat(box) -> list:
    return [float(v) for pair in box for v in pair]


def _ptr(t) -> int:
    if t is None:
        return None
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError("expected a torch tensor")
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return t.data_ptr()


def _stream(stream) -> Optional[int]:
    import torch
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _prec(p) -> int:
    return PREC_NAMES[p] if isinstance(p, str) else int(p)


def _dtype(prec: int):
    import torch
    return torch.float64 if prec == FP64 else torch.float32


def grid_coeffs(kernel: int, d: int, src_box, tgt_box, dtheta: int, theta_box, n: int,
                prec="fp64", out=None, stream=None):
    """pttk_grid_coeffs: coefficient tensor C (n^D, column-major) on the current device.
    Returned as a 1-D tensor of n^D entries."""
    import torch
    prec = _prec(prec)
    D = 2 * d + dtheta
    if out is None:
        out = torch.empty(n ** D, dtype=_dtype(prec), device="cuda")
    _check(load().pttk_grid_coeffs(kernel, d, _dbl(_boxflat(src_box)), _dbl(_boxflat(tgt_box)), dtheta,
                                   _dbl(_boxflat(theta_box)), n, prec, _ptr(out), _stream(stream)))
    return out


def grid_entries(kernel: int, d: int, src_box, tgt_box, dtheta: int, theta_box, n: int, idx,
                 prec="fp64", out=None, stream=None):
    """pttk_grid_entries: kernel values at the multi-indices idx (M x D int32 CUDA tensor,
    0-based node indices, variable order (x, theta, y)) of the grid tensor M."""
    import torch
    prec = _prec(prec)
    if idx.dtype != torch.int32 or idx.dim() != 2 or idx.shape[1] != 2 * d + dtheta:
        raise ValueError(f"idx must be (M, {2 * d + dtheta}) int32")
    if out is None:
        out = torch.empty(idx.shape[0], dtype=_dtype(prec), device="cuda")
    _check(load().pttk_grid_entries(kernel, d, _dbl(_boxflat(src_box)), _dbl(_boxflat(tgt_box)), dtheta,
                                    _dbl(_boxflat(theta_box)), n, _ptr(idx), idx.shape[0], prec, _ptr(out),
                                    _stream(stream)))
    return out


class TT:
    """Owns a pttk_tt handle (TT cores on the device)."""

    def __init__(self, handle: int):
        self._h = ctypes.c_void_p(handle)

    @property
    def handle(self):
        if not self._h:
            raise ValueError("TT handle already freed")
        return self._h

    @classmethod
    def build_offline(cls, kernel: int, d: int, src_box, tgt_box, dtheta: int, theta_box, n: int,
                      tol: float, grid_prec="fp64", stream=None) -> "TT":
        h = ctypes.c_void_p()
        _check(load().pttk_build_offline(kernel, d, _dbl(_boxflat(src_box)), _dbl(_boxflat(tgt_box)),
                                         dtheta, _dbl(_boxflat(theta_box)), n, tol, _prec(grid_prec),
                                         _stream(stream), ctypes.byref(h)))
        return cls(h.value)

    @classmethod
    def from_coeffs(cls, kernel: int, d: int, src_box, tgt_box, dtheta: int, theta_box, n: int,
                    tol: float, C, stream=None) -> "TT":
        import torch
        prec = FP64 if C.dtype == torch.float64 else FP32
        h = ctypes.c_void_p()
        _check(load().pttk_tt_from_coeffs(kernel, d, _dbl(_boxflat(src_box)), _dbl(_boxflat(tgt_box)),
                                          dtheta, _dbl(_boxflat(theta_box)), n, tol, _ptr(C), prec,
                                          _stream(stream), ctypes.byref(h)))
        return cls(h.value)

    @classmethod
    def cross(cls, kernel: int, d: int, src_box, tgt_box, dtheta: int, theta_box, n: int, eps: float, key: int,
              max_sweeps: int = 60, n_check: int = 1000, init_it: int = 10, stream=None):
        """pttk_cross_build (TT greedy-cross, Algorithms 5-7): (TT, sweeps, kernel evaluations)."""
        h = _vp()
        sw, ev = _int(), _i64()
        _check(load().pttk_cross_build(kernel, d, _dbl(_boxflat(src_box)), _dbl(_boxflat(tgt_box)), dtheta,
                                       _dbl(_boxflat(theta_box)), n, float(eps), int(key) & ((1 << 64) - 1),
                                       int(max_sweeps), int(n_check), int(init_it), _stream(stream), ctypes.byref(h),
                                       ctypes.byref(sw), ctypes.byref(ev)))
        return cls(h.value), sw.value, ev.value

    @classmethod
    def from_cores(cls, kernel: int, d: int, src_box, tgt_box, dtheta: int, theta_box, n: int, cores) -> "TT":
        """pttk_tt_from_cores: a handle from host cores (core k: r_{k-1} x n x r_k, Chebyshev
        coefficient form)."""
        ranks = [int(cores[0].shape[0])] + [int(G.shape[2]) for G in cores]
        packed = np.ascontiguousarray(np.concatenate(
            [np.asarray(G, dtype=np.float64).reshape(-1, order="F") for G in cores]))
        r = (_int * len(ranks))(*ranks)
        h = _vp()
        _check(load().pttk_tt_from_cores(kernel, d, _dbl(_boxflat(src_box)), _dbl(_boxflat(tgt_box)), dtheta,
                                         _dbl(_boxflat(theta_box)), n, r, packed.ctypes.data_as(_c_double_p),
                                         ctypes.byref(h)))
        return cls(h.value)

    def round(self, tol: float, stream=None) -> "TT":
        """pttk_tt_round: a new TT of the same tensor with ranks reduced to relative
        Frobenius accuracy tol (Algorithm 1, TT-Round)."""
        h = _vp()
        _check(load().pttk_tt_round(self.handle, tol, _stream(stream), ctypes.byref(h)))
        return TT(h.value)

    @classmethod
    def load(cls, path: str) -> "TT":
        h = ctypes.c_void_p()
        _check(load().pttk_tt_load(path.encode(), ctypes.byref(h)))
        return cls(h.value)

    def save(self, path: str):
        _check(load().pttk_tt_save(self.handle, path.encode()))

    @property
    def dims(self):
        d, dth, n, k = _int(), _int(), _int(), _int()
        _check(load().pttk_tt_dims(self.handle, ctypes.byref(d), ctypes.byref(dth), ctypes.byref(n),
                                   ctypes.byref(k)))
        return d.value, dth.value, n.value, k.value

    @property
    def ranks(self) -> list:
        d, dth, _, _ = self.dims
        arr = (_int * (2 * d + dth + 1))()
        _check(load().pttk_tt_ranks(self.handle, arr))
        return list(arr)

    def core(self, k: int) -> np.ndarray:
        """Core k as a (r_{k-1}, n, r_k) FP64 numpy array (copied from the device)."""
        r = self.ranks
        n = self.dims[2]
        buf = np.empty(r[k] * n * r[k + 1], dtype=np.float64)
        _check(load().pttk_tt_get_core(self.handle, k, buf.ctypes.data_as(_c_double_p)))
        return buf.reshape(r[k], n, r[k + 1], order="F")

    def cores(self) -> list:
        d, dth, _, _ = self.dims
        return [self.core(k) for k in range(2 * d + dth)]

    def check(self, stream=None):
        """pttk_tt_check: synchronise and raise if a bounded device wait ran out."""
        _check(load().pttk_tt_check(self.handle, _stream(stream)))

    def free(self):
        if self._h:
            load().pttk_tt_free(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def theta_core(tt: TT, theta, prec="fp64", M=None, stream=None):
    import torch
    prec = _prec(prec)
    r = tt.ranks
    d, dth, _, _ = tt.dims
    if M is None:
        M = torch.empty(r[d], r[d + dth], dtype=_dtype(prec), device="cuda")
    _check(load().pttk_theta_core(tt.handle, _dbl(theta), prec, _ptr(M), _stream(stream)))
    return M


def instantiate(tt: TT, theta, X, Y, prec="fp64", U=None, M=None, V=None, stream=None):
    """pttk_instantiate: returns (U, M, V) with K(X, Y; theta) ~= U M V^T."""
    import torch
    prec = _prec(prec)
    dt = _dtype(prec)
    r = tt.ranks
    d, dth, _, _ = tt.dims
    for P in (X, Y):
        if P.dtype != dt or P.dim() != 2 or P.shape[1] != d:
            raise ValueError(f"points must be (N, {d}) {dt}")
    if U is None:
        U = torch.empty(X.shape[0], r[d], dtype=dt, device="cuda")
    if M is None:
        M = torch.empty(r[d], r[d + dth], dtype=dt, device="cuda")
    if V is None:
        V = torch.empty(Y.shape[0], r[d + dth], dtype=dt, device="cuda")
    _check(load().pttk_instantiate(tt.handle, _dbl(theta), _ptr(X), X.shape[0], _ptr(Y), Y.shape[0],
                                   prec, _ptr(U), _ptr(M), _ptr(V), _stream(stream)))
    return U, M, V


def _check_apply_args(U, M, V, w, out):
    """Shapes and dtypes of an apply call: the library reads and writes these buffers by raw
    pointer, so a mismatch would run past the end of one of them."""
    import torch
    if U.dtype not in (torch.float64, torch.float32):
        raise ValueError("U must be float64 or float32")
    if U.dim() != 2 or M.dim() != 2 or V.dim() != 2:
        raise ValueError("U, M and V must be matrices")
    for name, t in (("M", M), ("V", V), ("w", w), ("out", out)):
        if t is not None and t.dtype != U.dtype:
            raise ValueError(f"{name} must have U's dtype {U.dtype}")
    if tuple(M.shape) != (U.shape[1], V.shape[1]):
        raise ValueError(f"M must be {U.shape[1]} x {V.shape[1]}, got {tuple(M.shape)}")
    if w.numel() != V.shape[0]:
        raise ValueError(f"w must have {V.shape[0]} entries, got {w.numel()}")
    if out is not None and out.numel() != U.shape[0]:
        raise ValueError(f"out must have {U.shape[0]} entries, got {out.numel()}")


def apply(U, M, V, w, out=None, stream=None):
    """pttk_apply: out = U (M (V^T w))."""
    import torch
    _check_apply_args(U, M, V, w, out)
    prec = FP64 if U.dtype == torch.float64 else FP32
    if out is None:
        out = torch.empty(U.shape[0], dtype=U.dtype, device="cuda")
    _check(load().pttk_apply(_ptr(U), _ptr(M), _ptr(V), U.shape[0], V.shape[0], U.shape[1], V.shape[1],
                             prec, _ptr(w), _ptr(out), _stream(stream)))
    return out


def grad(tt: TT, theta, X, Y, w, z, prec="fp32", want_dX=True, stream=None):
    """pttk_grad: returns (loss, dL/dtheta as a numpy array, dL/dX as a CUDA tensor or None)."""
    import torch
    prec = _prec(prec)
    d, dth, _, _ = tt.dims
    loss = ctypes.c_double()
    dtheta = (ctypes.c_double * max(1, dth))()
    dX = torch.empty_like(X) if want_dX else None
    _check(load().pttk_grad(tt.handle, _dbl(theta), _ptr(X), X.shape[0], _ptr(Y), Y.shape[0], _ptr(w), _ptr(z),
                            prec, ctypes.byref(loss), dtheta, _ptr(dX) if want_dX else None, _stream(stream)))
    return loss.value, np.array(dtheta[:dth]), dX


def _make_loss_function():
    import torch

    class PTTKLoss(torch.autograd.Function):
        """L = w^T K~(X, Y; theta) z with gradients in theta and X from pttk_grad.

        forward(theta (d_theta tensor), X (N_s x d CUDA tensor), Y, w, z, tt, prec) -> scalar.
        The gradients are computed by the library in the same call as the loss and handed
        back by backward (scaled by the incoming gradient)."""

        @staticmethod
        def forward(ctx, theta, X, Y, w, z, tt, prec):
            th = [float(v) for v in theta.detach().cpu().reshape(-1)]
            loss, dth, dX = grad(tt, th, X.detach().contiguous(), Y.detach().contiguous(),
                                 w.detach().contiguous(), z.detach().contiguous(), prec,
                                 want_dX=X.requires_grad)
            ctx.save_for_backward(torch.tensor(dth, dtype=theta.dtype, device=theta.device),
                                  dX if dX is not None else torch.empty(0))
            ctx.has_dX = dX is not None
            return torch.tensor(loss, dtype=X.dtype, device=X.device)

        @staticmethod
        def backward(ctx, grad_out):
            dth, dX = ctx.saved_tensors
            g = grad_out.to(dth.dtype)
            return (g.to(dth.device) * dth, (grad_out * dX) if ctx.has_dX else None,
                    None, None, None, None, None)

    return PTTKLoss


_loss_fn = None


def pttk_loss(theta, X, Y, w, z, tt: TT, prec="fp32"):
    """Differentiable L = w^T K~ z (theta: tensor of d_theta values; X: CUDA tensor)."""
    global _loss_fn
    if _loss_fn is None:
        _loss_fn = _make_loss_function()
    return _loss_fn.apply(theta, X, Y, w, z, tt, prec)


class Batch:
    """pttk_batch plan: B instances with concatenated point sets (offsets on the host)."""

    def __init__(self, tt: TT, xoff, yoff, prec="fp32", stream=None):
        self.tt = tt
        self.prec = _prec(prec)
        xo = np.ascontiguousarray(xoff, dtype=np.int64)
        yo = np.ascontiguousarray(yoff, dtype=np.int64)
        self.B = len(xo) - 1
        self.Ns, self.Nt = int(xo[-1]), int(yo[-1])
        h = ctypes.c_void_p()
        _check(load().pttk_batch_create(tt.handle, self.B, xo.ctypes.data_as(ctypes.POINTER(_i64)),
                                        yo.ctypes.data_as(ctypes.POINTER(_i64)), self.prec, _stream(stream),
                                        ctypes.byref(h)))
        self._h = h

    @property
    def config(self):
        c, n = _int(), _int()
        _check(load().pttk_batch_get_config(self._h, ctypes.byref(c), ctypes.byref(n)))
        return c.value, n.value

    def set_config(self, cfg: int):
        _check(load().pttk_batch_set_config(self._h, cfg))

    def autotune(self, X, Y, U, V, stream=None):
        """Times every launch configuration (pttk_batch_autotune); returns ms per configuration."""
        n = self.config[1]
        ms = (ctypes.c_float * n)()
        _check(load().pttk_batch_autotune(self._h, _ptr(X), _ptr(Y), _ptr(U), _ptr(V), ms, _stream(stream)))
        return list(ms)

    def instantiate(self, thetas, X, Y, U=None, M=None, V=None, stream=None):
        """pttk_instantiate_batched: thetas is a (B, d_theta) float64 CUDA tensor."""
        import torch
        dt = _dtype(self.prec)
        r = self.tt.ranks
        d, dth, _, _ = self.tt.dims
        if U is None:
            U = torch.empty(self.Ns, r[d], dtype=dt, device="cuda")
        if V is None:
            V = torch.empty(self.Nt, r[d + dth], dtype=dt, device="cuda")
        if M is None:
            M = torch.empty(self.B, r[d], r[d + dth], dtype=dt, device="cuda")
        _check(load().pttk_instantiate_batched(self._h, _ptr(thetas), _ptr(X), _ptr(Y), _ptr(U), _ptr(M),
                                               _ptr(V), _stream(stream)))
        return U, M, V

    def free(self):
        if getattr(self, "_h", None):
            load().pttk_batch_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Global:
    """PTTK-Global (Algorithm 4) on one point set X (source box = target box): owns a
    pttk_global handle holding Q and R of the thin QR of [S T] = [U(X) V(X)]."""

    def __init__(self, tt: TT, X, stream=None):
        import torch
        d = tt.dims[0]
        if X.dtype != torch.float64 or X.dim() != 2 or X.shape[1] != d:
            raise ValueError(f"points must be (N, {d}) float64")
        h = _vp()
        _check(load().pttk_global_create(tt.handle, _ptr(X), X.shape[0], _stream(stream), ctypes.byref(h)))
        self._h = h

    @property
    def handle(self):
        if not self._h:
            raise ValueError("PTTK-Global handle already freed")
        return self._h

    @property
    def dims(self):
        """(N, k, r_s, r_t): points, columns of Q, columns of S and of T."""
        N, k, rs, rt = _i64(), _int(), _int(), _int()
        _check(load().pttk_global_dims(self.handle, ctypes.byref(N), ctypes.byref(k), ctypes.byref(rs),
                                       ctypes.byref(rt)))
        return N.value, k.value, rs.value, rt.value

    def Q(self, stream=None):
        """Q (N x k float64 CUDA tensor, orthonormal columns)."""
        import torch
        N, k, _, _ = self.dims
        Q = torch.empty(N, k, dtype=torch.float64, device="cuda")
        _check(load().pttk_global_get_q(self.handle, _ptr(Q), _stream(stream)))
        return Q

    def R(self) -> np.ndarray:
        """R = Q^T [S T] (k x (r_s + r_t)) as a numpy array."""
        _, k, rs, rt = self.dims
        buf = np.empty(k * (rs + rt), dtype=np.float64)
        _check(load().pttk_global_get_r(self.handle, buf.ctypes.data_as(_c_double_p)))
        return buf.reshape(k, rs + rt, order="F")

    def instantiate(self, theta, eps: float = 0.0, compress: bool = False, definite: bool = True,
                    stream=None):
        """pttk_global_instantiate: returns (Z, W) with K(X, X; theta) ~= Z W Z^T.
        PTTK-Global-1 (compress False): Z = Q (N x k), W = U Lambda U^T (k x k).
        PTTK-Global-2 (compress True): Z = Q U^ (N x rank), W = diag(lambda^) (rank x rank)."""
        import torch
        N, k, _, _ = self.dims
        W = torch.empty(k * k, dtype=torch.float64, device="cuda")
        Z = torch.empty(N * k, dtype=torch.float64, device="cuda") if compress else None
        rank = _int()
        _check(load().pttk_global_instantiate(self.handle, _dbl(theta), float(eps), 1 if compress else 0,
                                              1 if definite else 0, _ptr(Z), _ptr(W), ctypes.byref(rank),
                                              _stream(stream)))
        r = rank.value
        if not compress:
            return self.Q(stream), W.view(k, k)
        return Z[:N * r].view(N, r), W[:r * r].view(r, r)

    def instantiate_batched(self, thetas, definite: bool = True, stream=None):
        """pttk_global_instantiate_batched: W (B x k x k) of PTTK-Global-1 for every row of
        thetas (B x d_theta); K(X, X; theta_b) ~= Q W[b] Q^T."""
        import torch
        th = np.ascontiguousarray(np.atleast_2d(np.asarray(thetas, dtype=np.float64)))
        B = th.shape[0]
        _, k, _, _ = self.dims
        W = torch.empty(B * k * k, dtype=torch.float64, device="cuda")
        _check(load().pttk_global_instantiate_batched(self.handle, B, th.ctypes.data_as(_c_double_p),
                                                      1 if definite else 0, _ptr(W), _stream(stream)))
        return W.view(B, k, k)

    def free(self):
        if self._h:
            load().pttk_global_free(self._h)
            self._h = _vp()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Fixed:
    """Algorithm 2 for fixed point sets X, Y: Phase 3 (S = U(X), T = V(Y) in FP64) and Phase 4
    (TT-Round of the twisted TT at `tol`; 0 skips it). Online: K ~= S' H'(theta) T'^T."""

    def __init__(self, tt: TT, X, Y, tol: float, stream=None):
        import torch
        d = tt.dims[0]
        for P_ in (X, Y):
            if P_.dtype != torch.float64 or P_.dim() != 2 or P_.shape[1] != d:
                raise ValueError(f"points must be (N, {d}) float64")
        h = _vp()
        _check(load().pttk_fixed_create(tt.handle, _ptr(X), X.shape[0], _ptr(Y), Y.shape[0], float(tol),
                                        _stream(stream), ctypes.byref(h)))
        self._h = h
        self._n = tt.dims[2]

    @property
    def handle(self):
        if not self._h:
            raise ValueError("fixed-point handle already freed")
        return self._h

    @property
    def dims(self):
        """(N_s, N_t, d_theta, ranks): ranks = [r_s', inner.., r_t']."""
        Ns, Nt, dth = _i64(), _i64(), _int()
        r = (_int * 9)()
        _check(load().pttk_fixed_dims(self.handle, ctypes.byref(Ns), ctypes.byref(Nt), ctypes.byref(dth), r))
        return Ns.value, Nt.value, dth.value, list(r[:max(dth.value, 0) + 1])

    def factors(self, stream=None):
        """(S', T') as float64 CUDA tensors."""
        import torch
        Ns, Nt, dth, r = self.dims
        S = torch.empty(Ns, r[0], dtype=torch.float64, device="cuda")
        T = torch.empty(Nt, r[dth], dtype=torch.float64, device="cuda")
        _check(load().pttk_fixed_get_factors(self.handle, _ptr(S), _ptr(T), _stream(stream)))
        return S, T

    def cores(self) -> list:
        """The rounded theta cores (r_j x n x r_{j+1} numpy arrays)."""
        Ns, Nt, dth, r = self.dims
        out = []
        n = self._n
        for j in range(dth):
            buf = np.empty(r[j] * n * r[j + 1], dtype=np.float64)
            _check(load().pttk_fixed_get_core(self.handle, j, buf.ctypes.data_as(_c_double_p)))
            out.append(buf.reshape(r[j], n, r[j + 1], order="F"))
        return out

    def theta_core(self, theta, prec="fp64", M=None, stream=None):
        import torch
        prec = _prec(prec)
        Ns, Nt, dth, r = self.dims
        if M is None:
            M = torch.empty(r[0], r[dth], dtype=_dtype(prec), device="cuda")
        _check(load().pttk_fixed_theta_core(self.handle, _dbl(theta), prec, _ptr(M), _stream(stream)))
        return M

    def free(self):
        if self._h:
            load().pttk_fixed_free(self._h)
            self._h = _vp()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def _f64_points(X):
    import torch
    if X.dtype != torch.float64 or X.dim() != 2:
        raise ValueError("points must be an (N, d) float64 CUDA tensor")


def gp_kv(kernel: int, X, theta, s2: float, v, out=None, prec="fp64", stream=None):
    """pttk_gp_kv: (K(X, X; theta) + s2 I) v, kernel entries evaluated on the fly in FP64, or in
    FP32 with FP64 sums of the tiles (prec="fp32")."""
    import torch
    _f64_points(X)
    if v.dtype != torch.float64 or v.numel() != X.shape[0]:
        raise ValueError("v must hold N float64 values")
    if out is None:
        out = torch.empty_like(v)
    _check(load().pttk_gp_kv(int(kernel), X.shape[1], _ptr(X), X.shape[0], _dbl(theta), float(s2), _ptr(v),
                             _ptr(out), _prec(prec), _stream(stream)))
    return out


def gp_pcg(kernel: int, X, theta, s2: float, b, Z=None, lam=None, tol: float = 1e-10, maxit: int = 1000,
           prec="fp64", stream=None):
    """pttk_gp_pcg: (x, iterations, relative residual) for (K + s2 I) x = b, preconditioned by
    (Z diag(lam) Z^T + s2 I)^{-1} when Z and lam are given; K v in the precision `prec`."""
    import torch
    _f64_points(X)
    N = X.shape[0]
    if b.dtype != torch.float64 or b.numel() != N:
        raise ValueError("b must hold N float64 values")
    m = 0
    if Z is not None:
        m = Z.shape[1]
        if Z.dtype != torch.float64 or Z.shape[0] != N or lam is None or lam.numel() != m:
            raise ValueError("Z must be (N, m) float64 with m eigenvalues in lam")
    x = torch.empty_like(b)
    it, res = _int(), ctypes.c_double()
    _check(load().pttk_gp_pcg(int(kernel), X.shape[1], _ptr(X), N, _dbl(theta), float(s2), _ptr(Z) if m else None,
                              _ptr(lam) if m else None, m, _ptr(b), _ptr(x), float(tol), int(maxit), _prec(prec),
                              ctypes.byref(it), ctypes.byref(res), _stream(stream)))
    return x, it.value, res.value


def gp_lml(g: "Global", theta, s2: float, y, stream=None):
    """pttk_gp_lml: (log marginal likelihood, gradient in theta) for the low-rank kernel of g."""
    import torch
    N = g.dims[0]
    if y.dtype != torch.float64 or y.numel() != N:
        raise ValueError("y must hold N float64 values")
    lml = ctypes.c_double()
    grad = (ctypes.c_double * 2)()
    _check(load().pttk_gp_lml(g.handle, _dbl(theta), float(s2), _ptr(y), ctypes.byref(lml), grad, _stream(stream)))
    return lml.value, np.array(grad[:len(theta)])


def apply_noalloc(U, M, V, w, out, stream=None):
    """pttk_apply_noalloc: out = U (M (V^T w)) with no device allocation (fixed library scratch)."""
    import torch
    _check_apply_args(U, M, V, w, out)
    prec = FP64 if U.dtype == torch.float64 else FP32
    _check(load().pttk_apply_noalloc(_ptr(U), _ptr(M), _ptr(V), U.shape[0], V.shape[0], U.shape[1],
                                     V.shape[1], prec, _ptr(w), _ptr(out), _stream(stream)))
    return out


PROBE_DFMA, PROBE_FFMA, PROBE_DMMA, PROBE_TF32, PROBE_F16, PROBE_F16S64, PROBE_F16S128, PROBE_F16S256 = range(8)
PROBE_NAMES = {"dfma": PROBE_DFMA, "ffma": PROBE_FFMA, "dmma": PROBE_DMMA, "tf32": PROBE_TF32, "f16": PROBE_F16,
               "f16s64": PROBE_F16S64, "f16s128": PROBE_F16S128, "f16s256": PROBE_F16S256}


def peak_probe(kind, iters: int, stream=None):
    """pttk_peak_probe: (TFLOP/s, ms) of one loop kernel of the given kind."""
    k = PROBE_NAMES[kind] if isinstance(kind, str) else int(kind)
    tf, ms = ctypes.c_double(), ctypes.c_double()
    _check(load().pttk_peak_probe(k, int(iters), _stream(stream), ctypes.byref(tf), ctypes.byref(ms)))
    return tf.value, ms.value


def splitmix64(key: int, counter: int) -> int:
    """pttk_splitmix64: output `counter` of the SplitMix64 stream seeded with `key`."""
    return int(load().pttk_splitmix64(key & ((1 << 64) - 1), counter & ((1 << 64) - 1)))


def profile_enable(on: bool = True):
    _check(load().pttk_profile_enable(1 if on else 0))


def profile_reset():
    _check(load().pttk_profile_reset())


def profile_get(name: str):
    """(total ms, launches) accumulated for a library kernel since the last reset."""
    ms, n = ctypes.c_double(), _i64()
    _check(load().pttk_profile_get(name.encode(), ctypes.byref(ms), ctypes.byref(n)))
    return ms.value, n.value


def profile_names() -> list:
    buf = ctypes.create_string_buffer(4096)
    _check(load().pttk_profile_names(buf, 4096))
    return [s for s in buf.value.decode().split("\n") if s]


def launch_count() -> int:
    """Kernels launched by the library so far in this process."""
    return int(load().pttk_launch_count())


def selftest_wait_timeout(stream=None) -> int:
    """Runs a kernel whose bounded wait can never complete; returns the library status
    (ETIMEOUT when the wait gave up as designed)."""
    return int(load().pttk_selftest_wait_timeout(_stream(stream)))
