"""Thin Python binding of the C ABI in ``include/sdl.h`` (ctypes).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Tensors are PyTorch CUDA tensors; PyTorch provides device memory
and streams.  There is no CPU fallback: if the library has not been built,
``lib()`` raises.

Layout helpers: signals are (N, p1, p2) tensors whose memory is column-major
per signal (strides (p1*p2, 1, p1)); dictionaries are (p, n) column-major
tensors (strides (1, p)).  ``signals()`` and ``dictionary()`` produce them.
"""
from __future__ import annotations

import ctypes
import os

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libsdl_gb300.so")
_lib = None

SDL_OK = 0
ERRORS = {
    -1: "SDL_ERR_ARG", -2: "SDL_ERR_CUDA", -3: "SDL_ERR_NONFINITE", -4: "SDL_ERR_SINGULAR",
    -5: "SDL_ERR_TIMEOUT", -6: "SDL_ERR_WORKSPACE", -7: "SDL_ERR_UNSUPPORTED",
    -8: "SDL_ERR_CAPACITY",
}

_P = ctypes.c_void_p
_I = ctypes.c_int
_L = ctypes.c_int64
_F = ctypes.c_float

# name -> argtypes (every entry point returns int)
SIGNATURES = {
    "sdl_create": [ctypes.POINTER(_P), _I],
    "sdl_destroy": [_P],
    "sdl_status": [_P, _P],
    "sdl_shape_supported": [_I, _I, _I, _I, _I],
    "sdl_reserve": [_P, _I, _I, _I, _I, _I],
    "sdl_sparse_code": [_P, _P, _I, _I, _L, _P, _I, _P, _I, _I, _F, _P, _P, _P, _P, _P],
    "sdl_update_D1": [_P, _P, _I, _I, _L, _P, _I, _P, _I, _I, _P, _P, _P, _P],
    "sdl_update_D2": [_P, _P, _I, _I, _L, _P, _I, _P, _I, _I, _P, _P, _P, _P],
    "sdl_iterate": [_P, _P, _I, _I, _L, _P, _I, _P, _I, _I, _F, _P, _P, _P, _P, _P],
    "sdl_sparse_code_static": [_P, _I, _I, _L, _P, _I, _P, _I, _I, _F, _P, _P, _P, _P, _P],
    "sdl_static_status": [_P],
    "sdl_fp32_fma_peak": [_I, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), _P],
    "sdl_batch_create": [_P, _P, _I, _I, _P, ctypes.POINTER(_P)],
    "sdl_batch_sparse_code": [_P, _P],
    "sdl_batch_iterate": [_P, _P, _P],
    "sdl_batch_tuning": [_P, _P, _P, _P],
    "sdl_batch_tuning_log": [_P, _P, _P, _P, _P, _I],
    "sdl_batch_destroy": [_P],
    "sdl_extract_patches": [_P, _I, _I, _I, _P, _P, _P],
    "sdl_patch_average": [_P, _P, _P, _P, _I, _P, _I, _P, _I, _I, _I, _I, _P, _P],
    "sdl_psnr": [_P, _P, _L, _F, _P, _P],
    "sdl_gemm_bf16": [_P, _P, _I, _P, _I, _I, _I, _I, _F, _P, _I, _P, _I, _I, _P, _I, _P, _I,
                      _P, _I, _P],
    "sdl_gemm_bf16_terms": [_P, _P, _I, _P, _I, _I, _I, _I, _I, _F, _P, _I, _P, _I, _I, _P, _I,
                            _P, _I, _P, _I, _P],
    "sdl_mlp_create": [_P, _I, _I, _I, _I, _I, _I, ctypes.POINTER(_P)],
    "sdl_mlp_destroy": [_P],
    "sdl_mlp_set_weights": [_P, _P, _P, _P, _P],
    "sdl_mlp_get_weights": [_P, _P, _P, _P, _P],
    "sdl_mlp_train_step": [_P, _P, _P, _I, _I, _F, _P, _P],
    "sdl_mlp_gradients": [_P, _P, _P, _I, _I, _P, _P, _P, _P, _P, _P],
    "sdl_mlp_forward": [_P, _P, _L, _P, _P],
    "sdl_sparse_code_learned": [_P, _P, _P, _I, _I, _L, _P, _I, _P, _I, _I, _I, _P, _P, _P, _P,
                                _P, _P, _P, _P],
    "sdl_learned_shortlists": [_P, _P, _L, _I, _I, _I, _P, _P],
    "sdl_sparse_code_shortlist": [_P, _P, _I, _I, _L, _P, _I, _P, _I, _I, _P, _I, _I, _P, _P, _P, _P,
                                  _P, _P],
    "sdl_ortho_sparse_code": [_P, _P, _I, _I, _L, _P, _P, _I, _F, _P, _P, _P, _P, _P],
    "sdl_ortho_iterate": [_P, _P, _I, _I, _L, _P, _P, _I, _F, _P, _P, _P, _P, _P],
    "sdl_selftest_timeout": [_P, ctypes.c_longlong, _P],
    "sdl_sparse_code3": [_P, _P, _I, _I, _I, _L, _P, _I, _P, _I, _P, _I, _I, _P, _P, _P, _P, _P],
    "sdl_iterate3": [_P, _P, _I, _I, _I, _L, _P, _I, _P, _I, _P, _I, _I, _P, _P, _P, _P, _P],
    "sdl_ssim": [_P, _P, _P, _I, _I, _F, _P, _P],
    "sdl_set_precision": [_P, _I],
    "sdl_tilings": [_I, _I, _I, _I, _I, _P, _I],
    "sdl_set_tiling": [_P, _I, _I, _I, _I, _I, _I, _I],
    "sdl_tune_tiling": [_P, _P, _I, _I, _L, _P, _I, _P, _I, _I, _P, _P],
    "sdl_tune_log": [_P, _P, _P, _P, _I],
    "sdl_precision_stats": [_P, ctypes.POINTER(ctypes.c_uint64)],
    "sdl_profile_enable": [_P, _I],
    "sdl_profile_collect": [_P, _P, _P, _I],
}


class SDLError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {ERRORS.get(code, code)}")


def lib() -> ctypes.CDLL:
    """Load the CUDA library (built by ``__graft_entry__.build()``)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing "
                               "(run __graft_entry__.build())")
        L = ctypes.CDLL(LIB_PATH)
        for name, argtypes in SIGNATURES.items():
            fn = getattr(L, name)
            fn.argtypes = argtypes
            fn.restype = _I
        for name in ("sdl_strerror", "sdl_kernel_name"):
            getattr(L, name).argtypes = [_I]
            getattr(L, name).restype = ctypes.c_char_p
        _lib = L
    return _lib


def _check(rc: int, where: str) -> None:
    if rc != SDL_OK:
        raise SDLError(rc, where)


def signals(Y: torch.Tensor) -> torch.Tensor:
    """(N, p1, p2) tensor -> same values, memory column-major per signal."""
    return Y.transpose(1, 2).contiguous().transpose(1, 2)


def signals3(Y: torch.Tensor) -> torch.Tensor:
    """(N, p1, p2, p3) tensor -> same values, memory column-major per signal
    (element (a, b, c) of signal k at a + p1 b + p1 p2 c + p1 p2 p3 k)."""
    return Y.permute(0, 3, 2, 1).contiguous().permute(0, 3, 2, 1)


def dictionary(D: torch.Tensor) -> torch.Tensor:
    """(p, n) tensor -> same values, column-major memory."""
    return D.t().contiguous().t()


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _need(t: torch.Tensor, dtype, shape, strides, name: str):
    if t.device.type != "cuda":
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    # the stride of a dimension of size 1 never enters an address
    if strides is not None and t.numel() > 1 and any(
            n > 1 and st != want for n, st, want in zip(t.shape, t.stride(), strides)):
        raise ValueError(f"{name} has strides {t.stride()}, expected {strides}")


def tilings(p1, p2, n1, n2, s):
    """Compiled tiling ids of the specialised coder for a shape (empty: none)."""
    L = lib()
    n = L.sdl_tilings(p1, p2, n1, n2, s, None, 0)
    ids = (_I * max(n, 1))()
    L.sdl_tilings(p1, p2, n1, n2, s, ids, n)
    return [ids[k] for k in range(n)]


def _check_Y(Y):
    if Y.dim() != 3:
        raise ValueError("Y must be (N, p1, p2)")
    N, p1, p2 = Y.shape
    _need(Y, torch.float32, (N, p1, p2), (p1 * p2, 1, p1), "Y")
    return N, p1, p2


def _check_Y3(Y):
    if Y.dim() != 4:
        raise ValueError("Y must be (N, p1, p2, p3)")
    N, p1, p2, p3 = Y.shape
    _need(Y, torch.float32, (N, p1, p2, p3), (p1 * p2 * p3, 1, p1, p1 * p2), "Y")
    return N, p1, p2, p3


def _check_D(D, p, name):
    if D.dim() != 2 or D.shape[0] != p:
        raise ValueError(f"{name} must be ({p}, n)")
    _need(D, torch.float32, D.shape, (1, p), name)
    return D.shape[1]


def shape_supported(p1, p2, n1, n2, s) -> bool:
    return bool(lib().sdl_shape_supported(p1, p2, n1, n2, s))


def sparse_code_static(Y, D1, D2, s, eps=0.0, out: "Codes | None" = None, stream=None) -> "Codes":
    """``sdl_sparse_code_static``: the sparse coder without a context and
    without device allocation (scratch in a static device array; see the
    header for its limits)."""
    N, p1, p2 = _check_Y(Y)
    n1, n2 = _check_D(D1, p1, "D1"), _check_D(D2, p2, "D2")
    if out is None:
        out = Codes.empty(N, s, Y.device, with_energy=True)
    _need(out.support, torch.int32, (N, s), None, "support")
    _need(out.coef, torch.float32, (N, s), None, "coef")
    _need(out.nnz, torch.int32, (N,), None, "nnz")
    rc = lib().sdl_sparse_code_static(_ptr(Y), p1, p2, N, _ptr(D1), n1, _ptr(D2), n2, s,
                                      float(eps), _ptr(out.support), _ptr(out.coef),
                                      _ptr(out.nnz), _ptr(out.res_energy), _stream(stream))
    _check(rc, "sdl_sparse_code_static")
    return out


def static_status(stream=None) -> int:
    """``sdl_static_status``: the first device-side error of the
    allocation-free calls on the current device since the last query (0 if
    none), cleared by the query."""
    return lib().sdl_static_status(_stream(stream))


def fp32_fma_peak(packed=True, stream=None):
    """``sdl_fp32_fma_peak``: measured FP32 FMA throughput of the current
    device in TFLOP/s, and the duration (ms) of the timed launch."""
    tf, ms = ctypes.c_double(), ctypes.c_double()
    _check(lib().sdl_fp32_fma_peak(1 if packed else 0, ctypes.byref(tf), ctypes.byref(ms),
                                   _stream(stream)), "sdl_fp32_fma_peak")
    return tf.value, ms.value


class Codes:
    """Sparse codes of N signals: support (N, s) int32 pair indices q = i + n1*j
    (-1 unused), coef (N, s) float32, nnz (N,) int32."""

    def __init__(self, support, coef, nnz, res_energy=None):
        self.support, self.coef, self.nnz, self.res_energy = support, coef, nnz, res_energy

    @staticmethod
    def empty(N, s, device, with_energy=False):
        return Codes(torch.empty((N, s), dtype=torch.int32, device=device),
                     torch.empty((N, s), dtype=torch.float32, device=device),
                     torch.empty((N,), dtype=torch.int32, device=device),
                     torch.empty((N,), dtype=torch.float32, device=device) if with_energy else None)


class Context:
    """One library context (``sdl_create``) on one CUDA device."""

    def __init__(self, device: int = 0):
        self._lib = lib()
        h = ctypes.c_void_p()
        _check(self._lib.sdl_create(ctypes.byref(h), int(device)), "sdl_create")
        self._h = h
        self.device = device

    def close(self):
        if getattr(self, "_h", None):
            self._lib.sdl_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def status(self, stream=None) -> int:
        """Synchronise and return (and clear) the recorded device-side error."""
        return self._lib.sdl_status(self._h, _stream(stream))

    def selftest_timeout(self, max_cycles: int = 1 << 24, stream=None) -> None:
        """``sdl_selftest_timeout``: a bounded wait that runs out on the GPU."""
        _check(self._lib.sdl_selftest_timeout(self._h, int(max_cycles), _stream(stream)),
               "sdl_selftest_timeout")

    def check(self, stream=None) -> None:
        _check(self.status(stream), "device")

    def profile(self, enable: bool = True) -> None:
        """Turn per-kernel event timing on or off (launch counts are always kept)."""
        _check(self._lib.sdl_profile_enable(self._h, int(bool(enable))), "sdl_profile_enable")

    def profile_collect(self) -> dict:
        """{kernel name: (total device ms, launches)} since the last collect."""
        n = NUM_KERNEL_KINDS
        ms = (ctypes.c_double * n)()
        cnt = (ctypes.c_int64 * n)()
        k = self._lib.sdl_profile_collect(self._h, ms, cnt, n)
        if k < 0:
            raise SDLError(k, "sdl_profile_collect")
        return {self._lib.sdl_kernel_name(i).decode(): (ms[i], cnt[i]) for i in range(k)}

    PREC_FP32, PREC_BF16_CORR, PREC_NO_RESCORE, PREC_FP64_SOLVE = 0, 1, 2, 4

    def set_precision(self, flags: int) -> None:
        """SDL_PREC_* flags (see include/sdl.h)."""
        _check(self._lib.sdl_set_precision(self._h, int(flags)), "sdl_set_precision")

    def precision_stats(self) -> int:
        """Correlation entries re-scored in FP32 since the last call."""
        v = ctypes.c_uint64()
        _check(self._lib.sdl_precision_stats(self._h, ctypes.byref(v)), "sdl_precision_stats")
        return v.value

    def reserve(self, p1, p2, n1, n2, s) -> None:
        _check(self._lib.sdl_reserve(self._h, p1, p2, n1, n2, s), "sdl_reserve")

    def sparse_code(self, Y, D1, D2, s, eps=0.0, out: Codes | None = None, stream=None) -> Codes:
        N, p1, p2 = _check_Y(Y)
        n1, n2 = _check_D(D1, p1, "D1"), _check_D(D2, p2, "D2")
        if out is None:
            out = Codes.empty(N, s, Y.device, with_energy=True)
        _need(out.support, torch.int32, (N, s), None, "support")
        _need(out.coef, torch.float32, (N, s), None, "coef")
        _need(out.nnz, torch.int32, (N,), None, "nnz")
        rc = self._lib.sdl_sparse_code(self._h, _ptr(Y), p1, p2, N, _ptr(D1), n1, _ptr(D2), n2,
                                       s, float(eps), _ptr(out.support), _ptr(out.coef),
                                       _ptr(out.nnz), _ptr(out.res_energy), _stream(stream))
        _check(rc, "sdl_sparse_code")
        return out

    def _update(self, fn, Y, D1, D2, codes: Codes, objective_out, stream):
        N, p1, p2 = _check_Y(Y)
        n1, n2 = _check_D(D1, p1, "D1"), _check_D(D2, p2, "D2")
        s = codes.support.shape[1]
        _need(codes.support, torch.int32, (N, s), None, "support")
        _need(codes.coef, torch.float32, (N, s), None, "coef")
        if objective_out is not None:
            _need(objective_out, torch.float64, (2,), None, "objective_out")
        rc = fn(self._h, _ptr(Y), p1, p2, N, _ptr(D1), n1, _ptr(D2), n2, s,
                _ptr(codes.support), _ptr(codes.coef), _ptr(objective_out), _stream(stream))
        return rc

    def update_D1(self, Y, D1, D2, codes: Codes, objective_out=None, stream=None):
        """Corollary 1: D1 and codes.coef updated in place."""
        _check(self._update(self._lib.sdl_update_D1, Y, D1, D2, codes, objective_out, stream),
               "sdl_update_D1")

    def update_D2(self, Y, D1, D2, codes: Codes, objective_out=None, stream=None):
        """Result 1: D2 and codes.coef updated in place."""
        _check(self._update(self._lib.sdl_update_D2, Y, D1, D2, codes, objective_out, stream),
               "sdl_update_D2")

    def iterate(self, Y, D1, D2, s, eps=0.0, out: Codes | None = None, rmse_out=None,
                stream=None) -> Codes:
        """One iteration of Algorithm 1; D1, D2 updated in place."""
        N, p1, p2 = _check_Y(Y)
        n1, n2 = _check_D(D1, p1, "D1"), _check_D(D2, p2, "D2")
        if out is None:
            out = Codes.empty(N, s, Y.device)
        _need(out.support, torch.int32, (N, s), None, "support")
        _need(out.coef, torch.float32, (N, s), None, "coef")
        _need(out.nnz, torch.int32, (N,), None, "nnz")
        if rmse_out is not None:
            _need(rmse_out, torch.float64, (2,), None, "rmse_out")
        rc = self._lib.sdl_iterate(self._h, _ptr(Y), p1, p2, N, _ptr(D1), n1, _ptr(D2), n2, s,
                                   float(eps), _ptr(out.support), _ptr(out.coef), _ptr(out.nnz),
                                   _ptr(rmse_out), _stream(stream))
        _check(rc, "sdl_iterate")
        return out

    # ---- the learned coder's shortlist steps on their own
    def learned_shortlists(self, scores, k1, k2, stream=None):
        """``sdl_learned_shortlists``: (N, k2) int32 candidate lists from
        (N, Q) FP32 scores (the k1-best shortlist, then the check set)."""
        N, Q = scores.shape
        _need(scores, torch.float32, (N, Q), (Q, 1), "scores")
        cand = torch.empty((N, k2), dtype=torch.int32, device=scores.device)
        _check(self._lib.sdl_learned_shortlists(self._h, _ptr(scores), N, Q, int(k1), int(k2),
                                                _ptr(cand), _stream(stream)), "sdl_learned_shortlists")
        return cand

    def sparse_code_shortlist(self, Y, D1, D2, s, cand, k1, stream=None):
        """``sdl_sparse_code_shortlist``: 2D-OMP over the first k1 pairs of
        each candidate list, without fallback; returns (codes, flags)."""
        N, p1, p2 = _check_Y(Y)
        n1, n2 = _check_D(D1, p1, "D1"), _check_D(D2, p2, "D2")
        k2 = cand.shape[1]
        _need(cand, torch.int32, (N, k2), (k2, 1), "cand")
        out = Codes.empty(N, s, Y.device, with_energy=True)
        flag = torch.empty((N,), dtype=torch.int32, device=Y.device)
        _check(self._lib.sdl_sparse_code_shortlist(
            self._h, _ptr(Y), p1, p2, N, _ptr(D1), n1, _ptr(D2), n2, s, _ptr(cand), int(k1), int(k2),
            _ptr(out.support), _ptr(out.coef), _ptr(out.nnz), _ptr(out.res_energy), _ptr(flag),
            _stream(stream)), "sdl_sparse_code_shortlist")
        return out, flag

    # ---- coder tilings
    def set_tiling(self, p1, p2, n1, n2, s, tiling, ctas_per_sm=0) -> None:
        """Pin a compiled tiling (see ``tilings``) for the shape; tiling < 0 unpins."""
        _check(self._lib.sdl_set_tiling(self._h, p1, p2, n1, n2, s, int(tiling), int(ctas_per_sm)),
               "sdl_set_tiling")

    def tune_tiling(self, Y, D1, D2, s, stream=None):
        """Time every tiling of the shape on these signals, pin the fastest;
        returns (tiling id, [dict(tiling, ctas_per_sm, us), ...])."""
        N, p1, p2 = _check_Y(Y)
        n1, n2 = _check_D(D1, p1, "D1"), _check_D(D2, p2, "D2")
        tid = ctypes.c_int(-1)
        _check(self._lib.sdl_tune_tiling(self._h, _ptr(Y), p1, p2, N, _ptr(D1), n1, _ptr(D2), n2, s,
                                         ctypes.byref(tid), _stream(stream)), "sdl_tune_tiling")
        n = self._lib.sdl_tune_log(self._h, None, None, None, 0)
        t, c, u = (_I * n)(), (_I * n)(), (_F * n)()
        self._lib.sdl_tune_log(self._h, t, c, u, n)
        return tid.value, [dict(tiling=t[e], ctas_per_sm=c[e], us=u[e]) for e in range(n)]

    # ---- three modes (Remark 3)
    def sparse_code3(self, Y, D1, D2, D3, s, out: Codes | None = None, stream=None) -> Codes:
        """``sdl_sparse_code3``: Y a (N, p1, p2, p3) CUDA tensor whose signals are
        stored column-major (see ``signals3``), D_m (p_m, n_m) column-major."""
        N, p1, p2, p3 = _check_Y3(Y)
        n1, n2, n3 = _check_D(D1, p1, "D1"), _check_D(D2, p2, "D2"), _check_D(D3, p3, "D3")
        if out is None:
            out = Codes.empty(N, s, Y.device, with_energy=True)
        _check(self._lib.sdl_sparse_code3(
            self._h, _ptr(Y), p1, p2, p3, N, _ptr(D1), n1, _ptr(D2), n2, _ptr(D3), n3, s,
            _ptr(out.support), _ptr(out.coef), _ptr(out.nnz), _ptr(out.res_energy),
            _stream(stream)), "sdl_sparse_code3")
        return out

    def iterate3(self, Y, D1, D2, D3, s, out: Codes | None = None, rmse_out=None,
                 stream=None) -> Codes:
        """``sdl_iterate3``: one three-mode iteration; D1, D2, D3 updated in place."""
        N, p1, p2, p3 = _check_Y3(Y)
        n1, n2, n3 = _check_D(D1, p1, "D1"), _check_D(D2, p2, "D2"), _check_D(D3, p3, "D3")
        if out is None:
            out = Codes.empty(N, s, Y.device)
        if rmse_out is not None:
            _need(rmse_out, torch.float64, (3,), None, "rmse_out")
        _check(self._lib.sdl_iterate3(
            self._h, _ptr(Y), p1, p2, p3, N, _ptr(D1), n1, _ptr(D2), n2, _ptr(D3), n3, s,
            _ptr(out.support), _ptr(out.coef), _ptr(out.nnz), _ptr(rmse_out), _stream(stream)),
            "sdl_iterate3")
        return out

    # ---- orthonormal variant (Remark 1)
    def ortho_sparse_code(self, Y, D1, D2, s, eps=0.0, out: Codes | None = None,
                          stream=None) -> Codes:
        """``sdl_ortho_sparse_code``: X_k = T_s(D1^T Y_k D2) for square orthonormal D
        (error-driven with eps > 0)."""
        N, p1, p2 = _check_Y(Y)
        if _check_D(D1, p1, "D1") != p1 or _check_D(D2, p2, "D2") != p2:
            raise ValueError("the orthonormal variant needs square dictionaries")
        if out is None:
            out = Codes.empty(N, s, Y.device, with_energy=True)
        _check(self._lib.sdl_ortho_sparse_code(
            self._h, _ptr(Y), p1, p2, N, _ptr(D1), _ptr(D2), s, float(eps), _ptr(out.support),
            _ptr(out.coef), _ptr(out.nnz), _ptr(out.res_energy), _stream(stream)),
            "sdl_ortho_sparse_code")
        return out

    def ortho_iterate(self, Y, D1, D2, s, eps=0.0, out: Codes | None = None, rmse_out=None,
                      stream=None) -> Codes:
        """``sdl_ortho_iterate``: one iteration of Algorithm 1 - Orthonormal."""
        N, p1, p2 = _check_Y(Y)
        if _check_D(D1, p1, "D1") != p1 or _check_D(D2, p2, "D2") != p2:
            raise ValueError("the orthonormal variant needs square dictionaries")
        if out is None:
            out = Codes.empty(N, s, Y.device)
        _need(out.support, torch.int32, (N, s), None, "support")
        _need(out.coef, torch.float32, (N, s), None, "coef")
        _need(out.nnz, torch.int32, (N,), None, "nnz")
        if rmse_out is not None:
            _need(rmse_out, torch.float64, (2,), None, "rmse_out")
        _check(self._lib.sdl_ortho_iterate(
            self._h, _ptr(Y), p1, p2, N, _ptr(D1), _ptr(D2), s, float(eps), _ptr(out.support),
            _ptr(out.coef), _ptr(out.nnz), _ptr(rmse_out), _stream(stream)), "sdl_ortho_iterate")
        return out


class _Group(ctypes.Structure):
    """Mirror of ``sdl_group`` in include/sdl.h."""
    _fields_ = [("Y", _P), ("p1", _I), ("p2", _I), ("N", _L), ("D1", _P), ("n1", _I),
                ("D2", _P), ("n2", _I), ("s_max", _I), ("eps", _F), ("support", _P),
                ("coef", _P), ("nnz", _P), ("res_energy", _P)]


NUM_KERNEL_KINDS = 18   # SDL_NUM_KERNEL_KINDS

BATCH_AUTOTUNE = 1
BATCH_GRAPH = 2
BATCH_RETUNE = 4


class Batch:
    """Several dictionary-learning problems run together (``sdl_batch_*``).

    groups: list of dicts with keys Y, D1, D2, s, eps (optional) and codes
    (optional :class:`Codes`; allocated when absent).  The tensors must stay
    alive and in place for the batch's lifetime (the batch keeps references).
    """

    def __init__(self, ctx: Context, groups, autotune: bool = True, graph: bool = True,
                 stream=None, retune: bool = False):
        self.ctx = ctx
        self._lib = ctx._lib
        self.groups = []
        arr = (_Group * len(groups))()
        for g, spec in enumerate(groups):
            Y, D1, D2, s = spec["Y"], spec["D1"], spec["D2"], int(spec["s"])
            N, p1, p2 = _check_Y(Y)
            n1, n2 = _check_D(D1, p1, "D1"), _check_D(D2, p2, "D2")
            codes = spec.get("codes") or Codes.empty(N, s, Y.device, with_energy=True)
            self.groups.append(dict(Y=Y, D1=D1, D2=D2, s=s, eps=float(spec.get("eps", 0.0)),
                                    codes=codes))
            arr[g] = _Group(Y.data_ptr(), p1, p2, N, D1.data_ptr(), n1, D2.data_ptr(), n2, s,
                            float(spec.get("eps", 0.0)), codes.support.data_ptr(),
                            codes.coef.data_ptr(), codes.nnz.data_ptr(),
                            codes.res_energy.data_ptr() if codes.res_energy is not None else None)
        flags = ((BATCH_AUTOTUNE if autotune else 0) | (BATCH_GRAPH if graph else 0) |
                 (BATCH_RETUNE if retune else 0))
        h = ctypes.c_void_p()
        _check(self._lib.sdl_batch_create(ctx._h, arr, len(groups), flags, _stream(stream),
                                          ctypes.byref(h)), "sdl_batch_create")
        self._h = h

    def sparse_code(self, stream=None):
        _check(self._lib.sdl_batch_sparse_code(self._h, _stream(stream)), "sdl_batch_sparse_code")

    def iterate(self, rmse_out=None, stream=None):
        if rmse_out is not None:
            _need(rmse_out, torch.float64, (2 * len(self.groups),), None, "rmse_out")
        _check(self._lib.sdl_batch_iterate(self._h, _ptr(rmse_out), _stream(stream)),
               "sdl_batch_iterate")

    def tuning(self):
        G = len(self.groups)
        sid, ctas, cost = (_I * G)(), (_I * G)(), (_F * G)()
        self._lib.sdl_batch_tuning(self._h, sid, ctas, cost)
        return [dict(shape_id=sid[g], ctas=ctas[g], cost_us=cost[g]) for g in range(G)]

    def tuning_log(self):
        """Every (group, tiling, CTAs per SM, microseconds) the autotuner timed."""
        n = self._lib.sdl_batch_tuning_log(self._h, None, None, None, None, 0)
        if n <= 0:
            return []
        g, sid, cps, cost = (_I * n)(), (_I * n)(), (_I * n)(), (_F * n)()
        self._lib.sdl_batch_tuning_log(self._h, g, sid, cps, cost, n)
        return [dict(group=g[e], shape_id=sid[e], ctas_per_sm=cps[e], cost_us=cost[e])
                for e in range(n)]

    def close(self):
        if getattr(self, "_h", None):
            self._lib.sdl_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def extract_patches(image: torch.Tensor, p: int, stream=None):
    """Every stride-1 p x p patch of a (H, W) FP32 CUDA image, mean removed.
    Returns (patches as an (N, p, p) signals tensor, means (N,))."""
    if image.dim() != 2:
        raise ValueError("image must be (H, W)")
    H, W = image.shape
    _need(image, torch.float32, (H, W), (W, 1), "image")
    N = (H - p + 1) * (W - p + 1)
    buf = torch.empty((N, p, p), dtype=torch.float32, device=image.device)   # (k, b, a)
    means = torch.empty((N,), dtype=torch.float32, device=image.device)
    _check(lib().sdl_extract_patches(_ptr(image), H, W, p, _ptr(buf), _ptr(means),
                                     _stream(stream)), "sdl_extract_patches")
    return buf.transpose(1, 2), means


def psnr(x: torch.Tensor, ref: torch.Tensor, peak: float = 255.0, stream=None) -> torch.Tensor:
    """Device scalar PSNR in dB (``sdl_psnr``)."""
    if x.shape != ref.shape or not x.is_contiguous() or not ref.is_contiguous():
        raise ValueError("x and ref must be contiguous and of one shape")
    out = torch.empty(1, dtype=torch.float32, device=x.device)
    _check(lib().sdl_psnr(_ptr(x), _ptr(ref), x.numel(), float(peak), _ptr(out), _stream(stream)),
           "sdl_psnr")
    return out


def ssim(ctx: Context, x: torch.Tensor, ref: torch.Tensor, peak: float = 255.0,
         stream=None) -> torch.Tensor:
    """Device scalar mean SSIM of x against ref (``sdl_ssim``)."""
    if x.shape != ref.shape or x.dim() != 2 or not x.is_contiguous() or not ref.is_contiguous():
        raise ValueError("x and ref must be contiguous 2-D images of one shape")
    out = torch.empty(1, dtype=torch.float32, device=x.device)
    _check(ctx._lib.sdl_ssim(ctx._h, _ptr(x), _ptr(ref), x.shape[0], x.shape[1], float(peak),
                             _ptr(out), _stream(stream)), "sdl_ssim")
    return out[0]


def patch_average(ctx: Context, codes: Codes, means, D1, D2, p: int, H: int, W: int,
                  stream=None) -> torch.Tensor:
    """Rebuild an (H, W) image from coded patches (``sdl_patch_average``)."""
    n1, n2 = _check_D(D1, p, "D1"), _check_D(D2, p, "D2")
    s = codes.support.shape[1]
    out = torch.empty((H, W), dtype=torch.float32, device=means.device)
    _check(ctx._lib.sdl_patch_average(ctx._h, _ptr(codes.support), _ptr(codes.coef), _ptr(means),
                                      s, _ptr(D1), n1, _ptr(D2), n2, p, H, W, _ptr(out),
                                      _stream(stream)), "sdl_patch_average")
    return out


def gemm_bf16(ctx: Context, A: torch.Tensor, B: torch.Tensor, alpha: float = 1.0, bias=None,
              act: int = 0, C=None, accumulate: bool = False, Cb=None, Ct=None, pre=None,
              stream=None):
    """``sdl_gemm_bf16``: act(alpha A B^T + bias) with A (M, K), B (N, K) BF16
    (row stride = shape[1] padded to a multiple of 8).  Returns C (allocated
    as FP32 (M, N) when not given and no other output is requested)."""
    M, K = A.shape
    N = B.shape[0]
    if B.shape[1] != K:
        raise ValueError("A and B must share K")
    for t, name in ((A, "A"), (B, "B")):
        if t.dtype != torch.bfloat16 or t.stride(1) != 1:
            raise ValueError(f"{name} must be BF16 with contiguous rows")
    if C is None and Cb is None and Ct is None and pre is None:
        C = torch.empty((M, N), dtype=torch.float32, device=A.device)
    rc = ctx._lib.sdl_gemm_bf16(
        ctx._h, _ptr(A), A.stride(0), _ptr(B), B.stride(0), M, N, K, float(alpha), _ptr(bias),
        int(act), _ptr(C), C.stride(0) if C is not None else 0, int(bool(accumulate)), _ptr(Cb),
        Cb.stride(0) if Cb is not None else 0, _ptr(Ct), Ct.stride(0) if Ct is not None else 0,
        _ptr(pre), pre.stride(0) if pre is not None else 0, _stream(stream))
    _check(rc, "sdl_gemm_bf16")
    return C


def gemm_bf16_terms(ctx: Context, A, B, alpha: float = 1.0, bias=None, act: int = 0, C=None,
                    accumulate: bool = False, Cb=None, Ct=None, pre=None, stream=None):
    """``sdl_gemm_bf16_terms``: act(alpha sum_t A[t] B[t]^T + bias) in one
    accumulator, A and B sequences of 1 to 3 BF16 tensors of equal shapes and
    row strides (the rules of :func:`gemm_bf16` for each)."""
    A, B = list(A), list(B)
    if not A or len(A) != len(B):
        raise ValueError("A and B must hold the same number (1 to 3) of operands")
    M, K = A[0].shape
    N = B[0].shape[0]
    for t in A + B:
        if t.dtype != torch.bfloat16 or t.stride(1) != 1:
            raise ValueError("operands must be BF16 with contiguous rows")
    for t in A:
        if tuple(t.shape) != (M, K) or t.stride(0) != A[0].stride(0):
            raise ValueError("every A[t] must share shape and row stride")
    for t in B:
        if tuple(t.shape) != (N, K) or t.stride(0) != B[0].stride(0):
            raise ValueError("every B[t] must share shape and row stride")
    if C is None and Cb is None and Ct is None and pre is None:
        C = torch.empty((M, N), dtype=torch.float32, device=A[0].device)
    pa = (ctypes.c_void_p * len(A))(*[t.data_ptr() for t in A])
    pb = (ctypes.c_void_p * len(B))(*[t.data_ptr() for t in B])
    rc = ctx._lib.sdl_gemm_bf16_terms(
        ctx._h, ctypes.cast(pa, ctypes.c_void_p), A[0].stride(0), ctypes.cast(pb, ctypes.c_void_p),
        B[0].stride(0), len(A), M, N, K, float(alpha), _ptr(bias), int(act), _ptr(C),
        C.stride(0) if C is not None else 0, int(bool(accumulate)), _ptr(Cb),
        Cb.stride(0) if Cb is not None else 0, _ptr(Ct), Ct.stride(0) if Ct is not None else 0,
        _ptr(pre), pre.stride(0) if pre is not None else 0, _stream(stream))
    _check(rc, "sdl_gemm_bf16_terms")
    return C


def _host_f32(a):
    import numpy as np
    a = np.ascontiguousarray(a, dtype=np.float32)
    return a, a.ctypes.data_as(ctypes.c_void_p)


class MLP:
    """The support-proposal network (``sdl_mlp_*``): p1*p2 -> hidden (GELU) ->
    n1*n2 scores, trained on the GPU by the library's own kernels."""

    def __init__(self, ctx: Context, p1, p2, n1, n2, hidden=512, max_batch=4096):
        self.ctx, self._lib = ctx, ctx._lib
        self.shape = (p1, p2, n1, n2, hidden)
        h = ctypes.c_void_p()
        _check(self._lib.sdl_mlp_create(ctx._h, p1, p2, n1, n2, hidden, max_batch,
                                        ctypes.byref(h)), "sdl_mlp_create")
        self._h = h
        self.max_batch = max_batch

    def init(self, seed=0):
        """He-style random initial weights from a seeded generator."""
        import numpy as np
        p1, p2, n1, n2, H = self.shape
        rng = np.random.default_rng(seed)
        P, Q = p1 * p2, n1 * n2
        self.set_weights(rng.standard_normal((H, P)) * np.sqrt(2.0 / P), np.zeros(H),
                         rng.standard_normal((Q, H)) * np.sqrt(1.0 / H), np.full(Q, -3.0))

    def set_weights(self, W1, b1, W2, b2):
        arrs = [_host_f32(a) for a in (W1, b1, W2, b2)]
        _check(self._lib.sdl_mlp_set_weights(self._h, *[p for _, p in arrs]), "sdl_mlp_set_weights")

    def get_weights(self):
        import numpy as np
        p1, p2, n1, n2, H = self.shape
        out = [np.empty((H, p1 * p2), np.float32), np.empty(H, np.float32),
               np.empty((n1 * n2, H), np.float32), np.empty(n1 * n2, np.float32)]
        _check(self._lib.sdl_mlp_get_weights(self._h, *[o.ctypes.data_as(ctypes.c_void_p) for o in out]),
               "sdl_mlp_get_weights")
        return out

    def train_step(self, Y, support, lr, loss_out=None, stream=None):
        N, p1, p2 = _check_Y(Y)
        _check(self._lib.sdl_mlp_train_step(self._h, _ptr(Y), _ptr(support), support.shape[1], N,
                                            float(lr), _ptr(loss_out), _stream(stream)),
               "sdl_mlp_train_step")

    def gradients(self, Y, support, stream=None):
        import numpy as np
        N, p1, p2 = _check_Y(Y)
        _, _, n1, n2, H = self.shape
        g = [np.empty((H, p1 * p2), np.float32), np.empty(H, np.float32),
             np.empty((n1 * n2, H), np.float32), np.empty(n1 * n2, np.float32)]
        loss = torch.zeros(1, dtype=torch.float32, device=Y.device)
        _check(self._lib.sdl_mlp_gradients(self._h, _ptr(Y), _ptr(support), support.shape[1], N,
                                           _ptr(loss), *[a.ctypes.data_as(ctypes.c_void_p) for a in g],
                                           _stream(stream)), "sdl_mlp_gradients")
        return loss.item(), dict(W1=g[0], b1=g[1], W2=g[2], b2=g[3])

    def forward(self, Y, stream=None):
        N, p1, p2 = _check_Y(Y)
        out = torch.empty((N, self.shape[2] * self.shape[3]), dtype=torch.float32, device=Y.device)
        _check(self._lib.sdl_mlp_forward(self._h, _ptr(Y), N, _ptr(out), _stream(stream)),
               "sdl_mlp_forward")
        return out

    def sparse_code(self, Y, D1, D2, s, k=32, out: Codes | None = None, stream=None):
        """``sdl_sparse_code_learned``: returns (codes, fallback flags, n_fallback,
        guard) with guard = device float[3]: the learned and the full coder's RMSE
        on the judging sample, and 1.0 when the guard re-coded every signal."""
        N, p1, p2 = _check_Y(Y)
        n1, n2 = _check_D(D1, p1, "D1"), _check_D(D2, p2, "D2")
        if out is None:
            out = Codes.empty(N, s, Y.device, with_energy=True)
        flags = torch.empty(N, dtype=torch.int32, device=Y.device)
        nfb = torch.zeros(1, dtype=torch.int32, device=Y.device)
        guard = torch.zeros(3, dtype=torch.float32, device=Y.device)
        _check(self._lib.sdl_sparse_code_learned(
            self.ctx._h, self._h, _ptr(Y), p1, p2, N, _ptr(D1), n1, _ptr(D2), n2, s, k,
            _ptr(out.support), _ptr(out.coef), _ptr(out.nnz), _ptr(out.res_energy), _ptr(flags),
            _ptr(nfb), _ptr(guard), _stream(stream)), "sdl_sparse_code_learned")
        return out, flags, nfb, guard

    def close(self):
        if getattr(self, "_h", None):
            self._lib.sdl_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
