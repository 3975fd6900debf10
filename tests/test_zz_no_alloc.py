"""GPU: the allocation-free build entry point against the allocating one.

dctf_build_matrix_noalloc serves callers that cannot call cudaMalloc (their
framework's pool owns the device memory, or their path must not trigger
cudaMalloc's device synchronisation): the caller passes the output buffers
and the build's scratch is a static array inside the library.  This test
calls it through the C ABI twice in a row (different masks, block sizes and
boundaries, so a stale scratch would show) and compares each result with
dctf_build_operator's and with the FP64 oracle's M, within the builder
tests' tolerance.  The file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest
import torch

import datagen
import oracle

pytestmark = pytest.mark.gpu


def noalloc_build(so, w, anchor, n, boundary, want_h):
    n2 = n * n
    m_out = torch.full((n2, n2), float("nan"), dtype=torch.float64, device="cuda")
    h_out = torch.full((n2, n2), float("nan"), dtype=torch.float64, device="cuda") if want_h else None
    wm = np.ascontiguousarray(w, dtype=np.float64)
    a = (ctypes.c_int * 2)(*anchor)
    st = so.dctf_build_matrix_noalloc(wm.ctypes.data, wm.shape[0], wm.shape[1], ctypes.addressof(a),
                                      n, boundary, m_out.data_ptr(),
                                      h_out.data_ptr() if want_h else None,
                                      torch.cuda.current_stream().cuda_stream)
    assert st == 0, so.dctf_last_error()
    torch.cuda.synchronize()
    return m_out.cpu().numpy(), (h_out.cpu().numpy() if want_h else None)


def test_noalloc_build_matches_allocating_build(dctf):
    so = dctf.load()
    calls = [(datagen.large_mask(), (4, 4), 16, oracle.REPLICATE, True),
             (datagen.headline_mask(), (1, 3), 8, oracle.ZERO, False)]
    for w, anchor, n, boundary, want_h in calls:
        m, h = noalloc_build(so, w, anchor, n, boundary, want_h)
        op = dctf.build_operator(w, anchor, n, boundary)
        m_ref, h_ref = op.download()
        op.release()
        scale = max(1.0, np.abs(w).sum())
        assert np.abs(m - m_ref).max() <= 1e-12 * scale
        assert np.abs(m - oracle.build_M(w, anchor, n, boundary)).max() <= 1e-12 * scale
        if want_h:
            assert np.array_equal(h, h_ref)
            assert np.array_equal(h, oracle.build_H(w, anchor, n, boundary))
    # a block side beyond the static scratch (2 n^4 doubles > 1 MiB at n = 32):
    # rejected before any launch, with the scratch limit in the message
    wm = np.ones((3, 3))
    a = (ctypes.c_int * 2)(1, 1)
    buf = torch.empty(1024, dtype=torch.float64, device="cuda")
    assert so.dctf_build_matrix_noalloc(wm.ctypes.data, 3, 3, ctypes.addressof(a), 32, 0,
                                        buf.data_ptr(), None, None) == 1
    assert "scratch" in dctf.last_error()
