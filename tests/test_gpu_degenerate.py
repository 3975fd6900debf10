"""GPU: the degenerate cases of the method, every arithmetic.

* the identity (1x1 mask of weight 1, and a 3x3 delta): y = x;
* the zero mask: y = 0 exactly;
* constant blocks under replication with a mask summing to 1: only the DC
  coefficient survives, unchanged;
* large coefficients (16x the image's) and a mask whose entries span six
  decades: the error scales with the outputs, nothing overflows;
* a mask as large as the block with the anchor in each corner.
"""
import numpy as np
import pytest
import torch

import datagen
import oracle

pytestmark = pytest.mark.gpu


def run(dctf, op, x, prec):
    op.set_precision(prec)
    xd = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()
    yd = torch.empty_like(xd)
    dctf.apply(op, xd, x.shape[0], yd)
    torch.cuda.synchronize()
    return yd.cpu().numpy().astype(np.float64)


def precisions(dctf, n):
    if n == 16:
        return [dctf.FP32_SIMT, dctf.F16X3, dctf.BF16X6, dctf.TF32X3]
    return [dctf.FP32_SIMT, dctf.F16X3] if n == 8 else [dctf.FP32_SIMT]


def coeffs(n, seed, shape=(256, 320)):
    img = datagen.synthetic_image(*shape, datagen.rng(95, seed, n))
    return oracle.dct2_blocks(oracle.image_to_blocks(img, n))


@pytest.mark.parametrize("n", [4, 8, 16])
def test_identity_masks(dctf, n):
    x = coeffs(n, 1)
    for w, a in ((np.array([[1.0]]), (0, 0)), (np.pad([[1.0]], 1), (1, 1))):
        for bnd in (0, 1):
            op = dctf.build_operator(w, a, n, bnd)
            for p in precisions(dctf, n):
                y = run(dctf, op, x, p)
                assert np.abs(y - x.astype(np.float32)).max() <= 1e-3, (n, p, bnd)
            op.release()


@pytest.mark.parametrize("n", [4, 8, 16])
def test_zero_mask_gives_zero(dctf, n):
    x = coeffs(n, 2)
    op = dctf.build_operator(np.zeros((3, 3)), (1, 1), n, dctf.REPLICATE)
    for p in precisions(dctf, n):
        assert not run(dctf, op, x, p).any(), p
    op.release()


@pytest.mark.parametrize("n", [8, 16])
def test_constant_blocks_keep_only_dc(dctf, n):
    g = np.random.default_rng(3)
    levels = g.integers(0, 256, 500).astype(np.float64)
    blocks = np.repeat(levels[:, None, None], n, axis=1).repeat(n, axis=2)
    x = oracle.dct2_blocks(blocks)
    w = datagen.uniform_random_mask(5, 5, datagen.rng(95, 3, n))
    w = w / w.sum()                                   # sum 1: a constant stays constant
    op = dctf.build_operator(w, (1, 3), n, dctf.REPLICATE)
    for p in precisions(dctf, n):
        y = run(dctf, op, x, p)
        assert np.abs(y[:, 1:]).max() <= 1e-3, p
        assert np.abs(y[:, 0] - x[:, 0]).max() <= 1e-3 * max(1.0, np.abs(x[:, 0]).max() / 2048), p
    op.release()


@pytest.mark.parametrize("n", [8, 16])
def test_large_coefficients_and_wide_mask_range(dctf, n):
    x = 16.0 * coeffs(n, 4)
    w = np.array([[1e-6, 0.25, 1e-6], [0.25, 1.0, 0.25], [1e-6, 0.25, 1e-6]])
    op = dctf.build_operator(w, (1, 1), n, dctf.ZERO)
    y_ref = oracle.apply_M(oracle.build_M(w, (1, 1), n, oracle.ZERO),
                           x.astype(np.float32).astype(np.float64))
    scale = np.abs(y_ref).max()
    for p in precisions(dctf, n):
        y = run(dctf, op, x, p)
        # the 1e-3 bar is for outputs on the 0-255 pixel scale (|y| ~ 2e3 at
        # n = 8): here it scales with the outputs
        assert np.abs(y - y_ref).max() <= 1e-3 * max(1.0, scale / 2048), (p, scale)
    op.release()


@pytest.mark.parametrize("n", [8, 16])
def test_block_sized_mask_anchor_in_each_corner(dctf, n):
    x = coeffs(n, 5)
    blocks = oracle.idct2_blocks(x, n)
    w = datagen.uniform_random_mask(n, n, datagen.rng(95, 5, n))
    for a in ((0, 0), (0, n - 1), (n - 1, 0), (n - 1, n - 1)):
        for bnd in (0, 1):
            op = dctf.build_operator(w, a, n, bnd)
            y_ref = oracle.apply_M(oracle.build_M(w, a, n, bnd), x.astype(np.float32).astype(np.float64))
            tol = 1e-3 * max(1.0, np.abs(w).sum())
            for p in precisions(dctf, n):
                y = run(dctf, op, x, p)
                assert np.abs(y - y_ref).max() <= tol, (a, bnd, p)
            op.release()
    del blocks
