"""GB300 block-DCT-domain filtering (arXiv 1710.07193), Python binding.

A thin ctypes binding over ``libdctf.so``: the same entry points as the C ABI
in ``include/dctf.h``, with arguments marshalled from numpy arrays, torch
tensors (device pointers taken with ``data_ptr()``) or raw integer pointers.
Every step of the filtering runs in the library's CUDA kernels; there is no
Python or CPU fallback: if the library is missing, ``load()`` raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

__all__ = [
    "ZERO", "REPLICATE", "FP32_SIMT", "F16X3", "BF16X6", "TF32X1", "TF32X3",
    "DctfError", "load", "lib_path", "exported_symbols", "build_operator", "Operator",
    "apply", "apply_f64in", "apply_host", "forward_dct", "inverse_dct_u8", "last_error",
    "version",
]

ZERO, REPLICATE = 0, 1
FP32_SIMT, F16X3, BF16X6, TF32X1, TF32X3 = 0, 1, 2, 3, 4
_STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "EBUDGET", 5: "ETIMEOUT",
           6: "EUNSUPPORTED"}

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None

_vp, _i32, _i64, _u32 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_uint32

# name -> (restype, argtypes); mirrors include/dctf.h
_SIGS = {
    "dctf_build_operator": (_i32, [_vp, _i32, _i32, _vp, _i32, _i32, _vp, _vp]),
    "dctf_operator_rebuild": (_i32, [_vp, _vp, _i32, _i32, _vp, _i32, _vp]),
    "dctf_operator_set_precision": (_i32, [_vp, _i32]),
    "dctf_operator_download": (_i32, [_vp, _vp, _vp]),
    "dctf_operator_status": (_i32, [_vp, _vp, _i32]),
    "dctf_release_operator": (None, [_vp]),
    "dctf_apply": (_i32, [_vp, _vp, _i64, _vp, _vp]),
    "dctf_apply_f64in": (_i32, [_vp, _vp, _i64, _vp, _vp]),
    "dctf_apply_host": (_i32, [_vp, _vp, _i64, _vp]),
    "dctf_forward_dct": (_i32, [_vp, _i32, _i32, _i64, _i32, _vp, _vp]),
    "dctf_forward_dct_f64": (_i32, [_vp, _i32, _i32, _i64, _i32, _vp, _vp]),
    "dctf_inverse_dct_u8": (_i32, [_vp, _i32, _i32, _i32, _vp, _i64, _vp]),
    "dctf_build_matrix_noalloc": (_i32, [_vp, _i32, _i32, _vp, _i32, _i32, _vp, _vp, _vp]),
    "dctf_last_error": (ctypes.c_char_p, []),
    "dctf_version": (_i32, []),
}


class DctfError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


def lib_path() -> str:
    return os.path.join(_HERE, "libdctf.so")


def load():
    """Load libdctf.so (built by ``__graft_entry__.build()``); raises if absent."""
    global _LIB
    if _LIB is None:
        path = lib_path()
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is not built; run __graft_entry__.build()")
        lib = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = lib
    return _LIB


def exported_symbols() -> list[str]:
    return list(_SIGS)


def last_error() -> str:
    return load().dctf_last_error().decode()


def version() -> int:
    return load().dctf_version()


def _check(status: int) -> None:
    if status != 0:
        raise DctfError(status, last_error())


def _ptr(x) -> int:
    if x is None:
        return 0
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError(f"cannot take a pointer of {type(x)}")


def _stream(stream) -> int:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class Operator:
    """Owns a dctf_operator handle (the FP64-built M and its pieces)."""

    def __init__(self, handle: int, n: int):
        self.handle = handle
        self.n = n
        self.n2 = n * n

    def rebuild(self, mask, anchor, boundary: int, stream=None) -> None:
        m = np.ascontiguousarray(mask, dtype=np.float64)
        a = (ctypes.c_int * 2)(*anchor)
        _check(load().dctf_operator_rebuild(self.handle, m.ctypes.data, m.shape[0], m.shape[1],
                                            ctypes.addressof(a), boundary, _stream(stream)))

    def set_precision(self, p: int) -> None:
        _check(load().dctf_operator_set_precision(self.handle, p))

    def download(self) -> tuple[np.ndarray, np.ndarray]:
        m = np.empty((self.n2, self.n2), dtype=np.float64)
        h = np.empty((self.n2, self.n2), dtype=np.float64)
        _check(load().dctf_operator_download(self.handle, m.ctypes.data, h.ctypes.data))
        return m, h

    def status(self, clear: bool = False) -> int:
        code = ctypes.c_uint32(0)
        _check(load().dctf_operator_status(self.handle, ctypes.addressof(code), int(clear)))
        return code.value

    def release(self) -> None:
        if self.handle:
            load().dctf_release_operator(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.release()
        except Exception:
            pass


def build_operator(mask, anchor, n: int, boundary: int, stream=None) -> Operator:
    m = np.ascontiguousarray(mask, dtype=np.float64)
    if m.ndim != 2:
        raise ValueError("mask must be 2-D")
    a = (ctypes.c_int * 2)(*anchor)
    h = ctypes.c_void_p(0)
    _check(load().dctf_build_operator(m.ctypes.data, m.shape[0], m.shape[1], ctypes.addressof(a),
                                      n, boundary, _stream(stream), ctypes.addressof(h)))
    return Operator(h.value, n)


def apply(op: Operator, coeffs, nblocks: int, out, stream=None) -> None:
    """out[b] = M coeffs[b] for b < nblocks (device FP32 [nblocks][n2])."""
    _check(load().dctf_apply(op.handle, _ptr(coeffs), nblocks, _ptr(out), _stream(stream)))


def apply_f64in(op: Operator, coeffs, nblocks: int, out, stream=None) -> None:
    _check(load().dctf_apply_f64in(op.handle, _ptr(coeffs), nblocks, _ptr(out), _stream(stream)))


def forward_dct(image, height: int, width: int, n: int, coeffs, pitch: int | None = None,
                stream=None, f64: bool = False) -> None:
    """Device uint8 image -> [nblocks][n*n] coefficients (FP32, or FP64)."""
    fn = load().dctf_forward_dct_f64 if f64 else load().dctf_forward_dct
    _check(fn(_ptr(image), height, width, pitch or width, n, _ptr(coeffs), _stream(stream)))


def inverse_dct_u8(coeffs, height: int, width: int, n: int, image, pitch: int | None = None,
                   stream=None) -> None:
    """Device FP32 coefficients -> uint8 image (rounded half away, saturated)."""
    _check(load().dctf_inverse_dct_u8(_ptr(coeffs), height, width, n, _ptr(image),
                                      pitch or width, _stream(stream)))


def apply_host(op: Operator, host_in, nblocks: int, host_out) -> None:
    """Host buffers in and out; copies and compute pipelined inside the library."""
    _check(load().dctf_apply_host(op.handle, _ptr(host_in), nblocks, _ptr(host_out)))
