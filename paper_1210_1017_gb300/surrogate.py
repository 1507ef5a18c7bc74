"""Python binding of the surrogate's C ABI (include/sur.h), same names as
the C functions; argument marshalling only."""
from __future__ import annotations

import ctypes as C

from . import sph as _sph

EXPORTED = ["sur_linear", "sur_wgrad_scratch_bytes", "sur_wgrad"]
SUR_EPI_NONE, SUR_EPI_RELU, SUR_EPI_RESIDUAL, SUR_EPI_RELU_MASK = 0, 1, 2, 4

_ready = False


def lib():
    global _ready
    L = _sph.lib()
    if not _ready:
        vp, u32, u64, i32 = C.c_void_p, C.c_uint32, C.c_uint64, C.c_int
        L.sur_linear.argtypes = [vp, vp, vp, u32, u32, u32, i32, vp, vp, vp, vp]
        L.sur_wgrad_scratch_bytes.argtypes = [u32]
        L.sur_wgrad_scratch_bytes.restype = u64
        L.sur_wgrad.argtypes = [vp, vp, u32, u32, C.c_float, vp, vp, u64, vp]
        _ready = True
    return L


def _p(t):
    return None if t is None else t.data_ptr()


def sur_linear(A, Bt, bias, M, K, N, epilogue, res, out_bf16, out_f32, stream):
    _sph._check(lib().sur_linear(_p(A), _p(Bt), _p(bias), M, K, N, epilogue, _p(res),
                                 _p(out_bf16), _p(out_f32), stream), what="sur_linear")


def sur_wgrad_scratch_bytes(N):
    return int(lib().sur_wgrad_scratch_bytes(N))


def sur_wgrad(P, Q, M, N, scale, dW, scratch, scratch_bytes, stream):
    _sph._check(lib().sur_wgrad(_p(P), _p(Q), M, N, scale, _p(dW), _p(scratch), scratch_bytes,
                                stream), what="sur_wgrad")
