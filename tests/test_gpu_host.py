"""GPU: dctf_apply_host, both routes.

Page-locked mapped buffers (torch pinned memory) take the host-direct
launch: the 8x8 F16X3 tensor-core kernel reads the input from host memory
and writes the output there itself.  Pageable buffers, unaligned buffers and
other block sizes take the staged route (copies pipelined with applies).
Either way the result equals dctf_apply on device buffers bit for bit (the
same kernel arithmetic in the same per-block order) and is within 1e-3 of
the FP64 oracle; nothing past nblocks is written.
"""
import numpy as np
import pytest
import torch

import datagen
import oracle

pytestmark = pytest.mark.gpu
COEF_TOL = 1e-3


@pytest.fixture(scope="module")
def source():
    img = datagen.synthetic_image(2048, 2048, datagen.rng(97, 0, 0))
    x = oracle.dct2_blocks(oracle.image_to_blocks(img, 8)).astype(np.float32)
    return x                                   # 65,536 blocks


def on_device(dctf, op, x):
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    yd = torch.empty_like(xd)
    dctf.apply(op, xd, x.shape[0], yd)
    torch.cuda.synchronize()
    return yd.cpu().numpy()


def pinned(x):
    t = torch.empty(x.shape, dtype=torch.float32, pin_memory=True)
    t.copy_(torch.from_numpy(np.ascontiguousarray(x)))
    return t


def test_direct_query(dctf):
    h = torch.zeros((100, 64), dtype=torch.float32, pin_memory=True)
    assert dctf.host_buffer_direct(h, h.numel() * 4)
    assert dctf.host_buffer_direct(h, 0)
    assert not dctf.host_buffer_direct(h, 1 << 40)             # past the allocation
    assert not dctf.host_buffer_direct(h, -1)
    assert not dctf.host_buffer_direct(np.zeros((100, 64), np.float32), 25600)   # pageable
    assert not dctf.host_buffer_direct(torch.zeros((100, 64), device="cuda"), 25600)
    assert not dctf.host_buffer_direct(None, 16)


@pytest.mark.parametrize("nb", [1, 63, 64, 65, 127, 129, 1000, 40961, 65536])
def test_direct_matches_device_and_oracle(dctf, source, nb):
    x = source[:nb]
    w, a = datagen.headline_mask(), (1, 3)
    op = dctf.build_operator(w, a, 8, dctf.REPLICATE)
    op.set_precision(dctf.F16X3)
    hin = pinned(x)
    hout = torch.full((nb + 3, 64), 7.0, dtype=torch.float32, pin_memory=True)
    assert dctf.host_buffer_direct(hin, hin.numel() * 4) and dctf.host_buffer_direct(hout, nb * 256)
    dctf.apply_host(op, hin, nb, hout)
    got = hout.numpy()
    assert np.array_equal(got[:nb], on_device(dctf, op, x))
    assert (got[nb:] == 7.0).all()                            # nothing past nblocks
    g = np.random.default_rng(nb)
    idx = np.unique(np.concatenate([np.arange(min(nb, 64)), g.integers(0, nb, 512)]))
    y_ref = oracle.apply_M(oracle.build_M(w, a, 8, oracle.REPLICATE), x[idx].astype(np.float64))
    assert np.abs(got[idx] - y_ref).max() <= COEF_TOL
    assert op.status() == 0
    op.release()


def test_direct_in_place_and_rebuild(dctf, source):
    x = source[:20000]
    op = dctf.build_operator(datagen.headline_mask(), (1, 3), 8, dctf.REPLICATE)
    h = pinned(x)
    dctf.apply_host(op, h, x.shape[0], h)
    assert np.array_equal(h.numpy(), on_device(dctf, op, x))
    # a rebuild changes the pieces' scale (magic square: sum 45); the direct
    # launch reads it per call
    op.rebuild(datagen.magic_square_3(), (1, 1), dctf.ZERO)
    hin, hout = pinned(x), pinned(np.zeros_like(x))
    for _ in range(2):
        dctf.apply_host(op, hin, x.shape[0], hout)
        assert np.array_equal(hout.numpy(), on_device(dctf, op, x))
    op.release()


def test_overlap_rejected(dctf, source):
    x = source[:256]
    op = dctf.build_operator(datagen.headline_mask(), (1, 3), 8, dctf.REPLICATE)
    h = pinned(np.concatenate([x, x]))
    with pytest.raises(dctf.DctfError) as e:
        dctf.apply_host(op, h[1:], 256, h)
    assert e.value.status == 1
    op.release()


def test_staged_routes(dctf, source):
    """Pageable memory, a pinned buffer that is not 16-byte aligned, and a
    16x16 operator all take the staged route and agree with dctf_apply."""
    x = source[:40961]
    op = dctf.build_operator(datagen.headline_mask(), (1, 3), 8, dctf.REPLICATE)
    y_dev = on_device(dctf, op, x)
    hin = np.ascontiguousarray(x)
    hout = np.zeros_like(hin)
    dctf.apply_host(op, hin, x.shape[0], hout)
    assert np.array_equal(hout, y_dev)
    flat_in = torch.empty(x.size + 4, dtype=torch.float32, pin_memory=True)
    flat_out = torch.zeros(x.size + 4, dtype=torch.float32, pin_memory=True)
    vin, vout = flat_in[1:1 + x.size], flat_out[1:1 + x.size]      # 4-byte offset
    vin.copy_(torch.from_numpy(hin.ravel()))
    dctf.apply_host(op, vin, x.shape[0], vout)
    assert np.array_equal(vout.numpy().reshape(x.shape), y_dev)
    assert flat_out[0].item() == 0.0 and flat_out[-3:].abs().sum().item() == 0.0
    op.release()
    img = datagen.synthetic_image(512, 512, datagen.rng(97, 1, 0))
    x16 = oracle.dct2_blocks(oracle.image_to_blocks(img, 16)).astype(np.float32)
    op16 = dctf.build_operator(datagen.large_mask(), (4, 4), 16, dctf.REPLICATE)
    h16, o16 = pinned(x16), pinned(np.zeros_like(x16))
    dctf.apply_host(op16, h16, x16.shape[0], o16)
    assert np.array_equal(o16.numpy(), on_device(dctf, op16, x16))
    op16.release()
