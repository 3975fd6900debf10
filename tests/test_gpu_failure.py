"""GPU: failure detection without a fault.  A kernel wait that can never
complete must time out after its bound, record a status code, and bring the
CTA's other roles out through the abort flag; the context stays usable."""
import time

import numpy as np
import pytest
import torch

import datagen

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_aborts_other_roles(dctf):
    t0 = time.perf_counter()
    st, code, other = dctf.selftest_wait_timeout(2000)      # 2 ms bound
    dt = time.perf_counter() - t0
    assert st == 5 and code == 0x101 and other == 1
    assert dt < 5.0                                          # far from the 2 s bound of role 2
    # the context is still usable afterwards
    op = dctf.build_operator(datagen.gaussian_mask(3, 1.0), (1, 1), 8, dctf.ZERO)
    x = torch.randn(300, 64, device="cuda")
    y = torch.empty_like(x)
    dctf.apply(op, x, 300, y)
    torch.cuda.synchronize()
    assert torch.isfinite(y).all() and op.status() == 0
    assert dctf.selftest_wait_timeout(0)[0] == 1             # EINVAL, nothing launched
