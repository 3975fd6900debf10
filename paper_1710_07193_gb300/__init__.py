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
    "ZERO", "REPLICATE", "FP32_SIMT", "F16X3", "BF16X6", "TF32X1", "TF32X3", "KRON_FP32", "BF16X3",
    "KRON_F16X3",
    "DctfError", "load", "lib_path", "exported_symbols", "build_operator", "Operator",
    "apply", "apply_f64in", "apply_host", "host_buffer_direct", "apply_pixels", "apply_planar", "forward_dct", "forward_dct_i16", "inverse_dct_u8", "last_error",
    "version", "IO_F32", "IO_I16", "Group", "group_create", "group_create_pixels", "apply_grouped",
    "Server",
]

ZERO, REPLICATE = 0, 1
IO_F32, IO_I16 = 0, 1
APPLY_INPUTS_READY = 1
MASK_CONVOLUTION, BUILD_KRON = 1, 2
FP32_SIMT, F16X3, BF16X6, TF32X1, TF32X3, KRON_FP32, BF16X3, KRON_F16X3 = 0, 1, 2, 3, 4, 5, 6, 7
_STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "EBUDGET", 5: "ETIMEOUT",
           6: "EUNSUPPORTED"}

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None

_vp, _i32, _i64, _u32 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_uint32

# name -> (restype, argtypes); mirrors include/dctf.h
_SIGS = {
    "dctf_build_operator": (_i32, [_vp, _i32, _i32, _vp, _i32, _i32, _vp, _vp]),
    "dctf_build_operator_ex": (_i32, [_vp, _i32, _i32, _vp, _i32, _i32, _u32, _vp, _vp]),
    "dctf_operator_rebuild": (_i32, [_vp, _vp, _i32, _i32, _vp, _i32, _vp]),
    "dctf_operator_set_precision": (_i32, [_vp, _i32]),
    "dctf_operator_set_flags": (_i32, [_vp, _u32]),
    "dctf_operator_kron_rank": (_i32, [_vp, _vp]),
    "dctf_operator_download": (_i32, [_vp, _vp, _vp]),
    "dctf_operator_status": (_i32, [_vp, _vp, _i32]),
    "dctf_release_operator": (None, [_vp]),
    "dctf_apply": (_i32, [_vp, _vp, _i64, _vp, _vp]),
    "dctf_apply_f64in": (_i32, [_vp, _vp, _i64, _vp, _vp]),
    "dctf_apply_pixels": (_i32, [_vp, _vp, _i32, _i32, _vp, _i64, _vp]),
    "dctf_apply_planar": (_i32, [_vp, _vp, _i32, _i32, _i64, _vp, _i64, _vp]),
    "dctf_apply_host": (_i32, [_vp, _vp, _i64, _vp]),
    "dctf_host_buffer_direct": (_i32, [_vp, _i64]),
    "dctf_forward_dct": (_i32, [_vp, _i32, _i32, _i64, _i32, _vp, _vp]),
    "dctf_forward_dct_f64": (_i32, [_vp, _i32, _i32, _i64, _i32, _vp, _vp]),
    "dctf_forward_dct_i16": (_i32, [_vp, _i32, _i32, _i64, _i32, _vp, _vp, _vp]),
    "dctf_inverse_dct_u8": (_i32, [_vp, _i32, _i32, _i32, _vp, _i64, _vp]),
    "dctf_build_matrix_noalloc": (_i32, [_vp, _i32, _i32, _vp, _i32, _i32, _vp, _vp, _vp]),
    "dctf_group_create": (_i32, [_vp, _i32, _i32, _vp]),
    "dctf_group_create_pixels": (_i32, [_vp, _i32, _vp]),
    "dctf_group_launch": (_i32, [_vp, _vp]),
    "dctf_group_tune": (_i32, [_vp, _vp, _i32]),
    "dctf_group_config": (_i32, [_vp, _vp, _vp, _vp, _vp]),
    "dctf_group_set_config": (_i32, [_vp, _i32, _i32, _i32, _i32]),
    "dctf_group_set_flags": (_i32, [_vp, ctypes.c_uint32]),
    "dctf_group_status": (_i32, [_vp, _vp, _i32]),
    "dctf_group_destroy": (None, [_vp]),
    "dctf_apply_grouped": (_i32, [_vp, _i32, _i32, _vp]),
    "dctf_selftest_wait_timeout": (_i32, [_u32, _vp, _vp]),
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

    def set_flags(self, flags: int) -> None:
        _check(load().dctf_operator_set_flags(self.handle, flags))

    def kron_rank(self) -> int:
        """Number of Kronecker terms (operators built with kron=True)."""
        r = ctypes.c_int(0)
        _check(load().dctf_operator_kron_rank(self.handle, ctypes.addressof(r)))
        return r.value

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


def build_operator(mask, anchor, n: int, boundary: int, stream=None,
                   convolution: bool = False, kron: bool = False) -> Operator:
    m = np.ascontiguousarray(mask, dtype=np.float64)
    if m.ndim != 2:
        raise ValueError("mask must be 2-D")
    a = (ctypes.c_int * 2)(*anchor)
    h = ctypes.c_void_p(0)
    _check(load().dctf_build_operator_ex(m.ctypes.data, m.shape[0], m.shape[1],
                                         ctypes.addressof(a), n, boundary,
                                         (MASK_CONVOLUTION if convolution else 0)
                                         | (BUILD_KRON if kron else 0),
                                         _stream(stream), ctypes.addressof(h)))
    return Operator(h.value, n)


def apply(op: Operator, coeffs, nblocks: int, out, stream=None) -> None:
    """out[b] = M coeffs[b] for b < nblocks (device FP32 [nblocks][n2])."""
    _check(load().dctf_apply(op.handle, _ptr(coeffs), nblocks, _ptr(out), _stream(stream)))


def apply_pixels(op: Operator, coeffs, height: int, width: int, image,
                 pitch: int | None = None, stream=None) -> None:
    """Device coefficients [nblocks][64] -> filtered uint8 image (device,
    height rows of `pitch` bytes), one fused pass (8x8 operators)."""
    _check(load().dctf_apply_pixels(op.handle, _ptr(coeffs), height, width, _ptr(image),
                                    pitch or width, _stream(stream)))


def apply_planar(op: Operator, coeffs, height: int, width: int, out, pitch: int | None = None,
                 out_pitch: int | None = None, stream=None) -> None:
    """Image-plane coefficients (device FP32, coefficient (u, v) of block
    (by, bx) at row 8 by + u, column 8 bx + v) -> the same layout, filtered."""
    _check(load().dctf_apply_planar(op.handle, _ptr(coeffs), height, width, pitch or width,
                                    _ptr(out), out_pitch or pitch or width, _stream(stream)))


def apply_f64in(op: Operator, coeffs, nblocks: int, out, stream=None) -> None:
    _check(load().dctf_apply_f64in(op.handle, _ptr(coeffs), nblocks, _ptr(out), _stream(stream)))


def forward_dct(image, height: int, width: int, n: int, coeffs, pitch: int | None = None,
                stream=None, f64: bool = False) -> None:
    """Device uint8 image -> [nblocks][n*n] coefficients (FP32, or FP64)."""
    fn = load().dctf_forward_dct_f64 if f64 else load().dctf_forward_dct
    _check(fn(_ptr(image), height, width, pitch or width, n, _ptr(coeffs), _stream(stream)))


def forward_dct_i16(image, height: int, width: int, n: int, q, coeffs,
                    pitch: int | None = None, stream=None) -> None:
    """Device uint8 image -> int16 quantised coefficients with table q (device)."""
    _check(load().dctf_forward_dct_i16(_ptr(image), height, width, pitch or width, n, _ptr(q),
                                       _ptr(coeffs), _stream(stream)))


def inverse_dct_u8(coeffs, height: int, width: int, n: int, image, pitch: int | None = None,
                   stream=None) -> None:
    """Device FP32 coefficients -> uint8 image (rounded half away, saturated)."""
    _check(load().dctf_inverse_dct_u8(_ptr(coeffs), height, width, n, _ptr(image),
                                      pitch or width, _stream(stream)))


def selftest_wait_timeout(limit_us: int = 2000) -> tuple[int, int, int]:
    """Run the bounded-wait self-test; returns (status, code, other_role_aborted)."""
    code, other = ctypes.c_uint32(0), ctypes.c_uint32(0)
    st = load().dctf_selftest_wait_timeout(limit_us, ctypes.addressof(code), ctypes.addressof(other))
    return st, code.value, other.value


def apply_host(op: Operator, host_in, nblocks: int, host_out) -> None:
    """Host buffers in and out: one host-direct launch on page-locked mapped
    buffers (8x8 F16X3), else copies and compute pipelined in the library."""
    _check(load().dctf_apply_host(op.handle, _ptr(host_in), nblocks, _ptr(host_out)))


def host_buffer_direct(buf, nbytes: int) -> bool:
    """True if the device can read and write `buf` (nbytes from its start)
    directly: page-locked, mapped, inside one allocation."""
    return load().dctf_host_buffer_direct(_ptr(buf), nbytes) == 1


class _GroupItem(ctypes.Structure):
    _fields_ = [("op", _vp), ("inp", _vp), ("out", _vp), ("nblocks", _i64),
                ("q_in", _vp), ("q_out", _vp)]


def _items_array(items):
    """items: sequence of (op, in, out, nblocks[, q_in, q_out])."""
    arr = (_GroupItem * max(1, len(items)))()
    for i, it in enumerate(items):
        op, inp, out, nb = it[:4]
        qi = it[4] if len(it) > 4 else None
        qo = it[5] if len(it) > 5 else None
        arr[i] = _GroupItem(op.handle, _ptr(inp), _ptr(out), int(nb), _ptr(qi), _ptr(qo))
    return arr


class Group:
    """A persistent grouped launch plan (dctf_group)."""

    def __init__(self, handle: int, keep):
        self.handle = handle
        self._keep = keep          # the operators must outlive the group

    def launch(self, stream=None) -> None:
        _check(load().dctf_group_launch(self.handle, _stream(stream)))

    def tune(self, reps: int = 5, stream=None) -> None:
        _check(load().dctf_group_tune(self.handle, _stream(stream), reps))

    def config(self) -> tuple[int, int, int, int]:
        """(CTAs, tile rows, input stages, operator slots) in use."""
        v = [ctypes.c_int(0) for _ in range(4)]
        _check(load().dctf_group_config(self.handle, *[ctypes.addressof(x) for x in v]))
        return tuple(x.value for x in v)

    def set_config(self, grid: int, tile_rows: int, stages: int, slots: int) -> None:
        _check(load().dctf_group_set_config(self.handle, grid, tile_rows, stages, slots))

    def set_flags(self, flags: int) -> None:
        """APPLY_INPUTS_READY: later launches use programmatic serialisation."""
        _check(load().dctf_group_set_flags(self.handle, flags))

    def status(self, clear: bool = False) -> int:
        code = ctypes.c_uint32(0)
        _check(load().dctf_group_status(self.handle, ctypes.addressof(code), int(clear)))
        return code.value

    def destroy(self) -> None:
        if self.handle:
            load().dctf_group_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def group_create(items, io: int = IO_F32) -> Group:
    arr = _items_array(items)
    h = ctypes.c_void_p(0)
    _check(load().dctf_group_create(ctypes.addressof(arr), len(items), io, ctypes.addressof(h)))
    return Group(h.value, [it[0] for it in items])


class _PixelItem(ctypes.Structure):
    _fields_ = [("op", _vp), ("coeffs", _vp), ("height", _i32), ("width", _i32),
                ("image", _vp), ("pitch", _i64)]


def group_create_pixels(items) -> Group:
    """items: sequence of (op, coeffs, height, width, image[, pitch]): fused
    pixel output for every item in one persistent launch."""
    arr = (_PixelItem * max(1, len(items)))()
    for i, it in enumerate(items):
        op, x, h, w, img = it[:5]
        pitch = it[5] if len(it) > 5 and it[5] is not None else w
        arr[i] = _PixelItem(op.handle, _ptr(x), int(h), int(w), _ptr(img), int(pitch))
    h = ctypes.c_void_p(0)
    _check(load().dctf_group_create_pixels(ctypes.addressof(arr), len(items), ctypes.addressof(h)))
    return Group(h.value, [it[0] for it in items])


def apply_grouped(items, io: int = IO_F32, stream=None) -> None:
    arr = _items_array(items)
    _check(load().dctf_apply_grouped(ctypes.addressof(arr), len(items), io, _stream(stream)))


# ------------------------------------------------------------------ serving
class _ServerCfg(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_size_t), ("max_inflight", _i32),
                ("max_batch_requests", _i32), ("op_cache_capacity", _i32),
                ("inject_build_failure_every", _i32), ("staged_only", _i32)]


class _Request(ctypes.Structure):
    _fields_ = [("nplanes", _i32), ("inp", _vp * 4), ("out", _vp * 4), ("nblocks", _i64 * 4),
                ("q", _vp * 4), ("mask", _vp), ("mh", _i32), ("mw", _i32),
                ("anchor", _i32 * 2), ("boundary", _i32), ("q_out", _vp * 4)]


class _Stats(ctypes.Structure):
    _fields_ = [("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double),
                ("mean_ms", ctypes.c_double), ("max_ms", ctypes.c_double),
                ("wall_s", ctypes.c_double), ("completed", ctypes.c_uint64),
                ("failed", ctypes.c_uint64), ("batches", ctypes.c_uint64),
                ("blocks", ctypes.c_uint64), ("cache_hits", ctypes.c_uint64),
                ("cache_misses", ctypes.c_uint64), ("max_batch_requests_seen", _i32),
                ("hbm_in_use", ctypes.c_size_t), ("direct_requests", ctypes.c_uint64),
                ("budget_waits", ctypes.c_uint64), ("hbm_peak", ctypes.c_size_t)]


_SIGS.update({
    "dctf_server_create": (_i32, [_vp, _vp]),
    "dctf_server_submit": (_i32, [_vp, _vp, _vp]),
    "dctf_server_wait": (_i32, [_vp, ctypes.c_uint64, _i32]),
    "dctf_server_stats": (_i32, [_vp, _vp]),
    "dctf_server_reset_stats": (_i32, [_vp]),
    "dctf_server_destroy": (None, [_vp]),
})


class Server:
    """Continuous-batching server for int16 quantised 8x8-block planes."""

    def __init__(self, hbm_budget_bytes: int = 1 << 30, max_inflight: int = 3,
                 max_batch_requests: int = 16, op_cache_capacity: int = 64,
                 inject_build_failure_every: int = 0, staged_only: bool = False):
        cfg = _ServerCfg(hbm_budget_bytes, max_inflight, max_batch_requests, op_cache_capacity,
                         inject_build_failure_every, 1 if staged_only else 0)
        h = ctypes.c_void_p(0)
        _check(load().dctf_server_create(ctypes.addressof(cfg), ctypes.addressof(h)))
        self.handle = h.value
        self._keep = {}

    def prepare(self, planes_in, planes_out, qtabs, mask, anchor, boundary: int, qtabs_out=None):
        """Marshal one request (argument conversion only) for submit_prepared.
        planes_in/out: host int16 arrays [nblocks][64] (kept alive until the
        request is waited for); qtabs: uint16 [64] per plane (dequantisation);
        qtabs_out: uint16 [64] per plane for the requantisation, or None for
        qtabs.  Page-locked planes (e.g. views of torch pinned tensors) take
        the server's host-direct route unless it was created staged_only."""
        r = _Request()
        r.nplanes = len(planes_in)
        keep = [np.ascontiguousarray(mask, dtype=np.float64)]
        outs = qtabs_out if qtabs_out is not None else [None] * len(planes_in)
        for p, (xi, xo, q, qo) in enumerate(zip(planes_in, planes_out, qtabs, outs)):
            q = np.ascontiguousarray(q, dtype=np.uint16).ravel()
            keep += [xi, xo, q]
            r.inp[p] = _ptr(xi)
            r.out[p] = _ptr(xo)
            r.nblocks[p] = xi.shape[0]
            r.q[p] = q.ctypes.data
            if qo is not None:
                qo = np.ascontiguousarray(qo, dtype=np.uint16).ravel()
                keep.append(qo)
                r.q_out[p] = qo.ctypes.data
        r.mask = keep[0].ctypes.data
        r.mh, r.mw = keep[0].shape
        r.anchor[0], r.anchor[1] = anchor
        r.boundary = boundary
        return (r, keep)

    def submit_prepared(self, prepared) -> int:
        """One dctf_server_submit call on a request made by prepare()."""
        r, keep = prepared
        t = ctypes.c_uint64(0)
        _check(load().dctf_server_submit(self.handle, ctypes.addressof(r), ctypes.addressof(t)))
        self._keep[t.value] = keep
        return t.value

    def submit(self, planes_in, planes_out, qtabs, mask, anchor, boundary: int,
               qtabs_out=None) -> int:
        """prepare() + submit_prepared()."""
        return self.submit_prepared(self.prepare(planes_in, planes_out, qtabs, mask, anchor,
                                                 boundary, qtabs_out))

    def wait(self, ticket: int, timeout_ms: int = 60000) -> None:
        st = load().dctf_server_wait(self.handle, ticket, timeout_ms)
        if st != 5:                       # a timed-out ticket stays valid
            self._keep.pop(ticket, None)
        _check(st)

    def stats(self) -> dict:
        s = _Stats()
        _check(load().dctf_server_stats(self.handle, ctypes.addressof(s)))
        return {k: getattr(s, k) for k, _ in _Stats._fields_}

    def reset_stats(self) -> None:
        """Start a new statistics window (the operator cache stays warm)."""
        _check(load().dctf_server_reset_stats(self.handle))

    def close(self) -> None:
        if self.handle:
            load().dctf_server_destroy(self.handle)
            self.handle = 0
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
