"""GPU: the paper-form (Kronecker / sandwich-product) apply, DCTF_KRON_FP32.

M = sum_t A_t kron B_t with one term per rank of the mask, applied as
Y = sum_t A_t X B_t^T in FP32 on CUDA cores.  Same bars as every apply: max
coefficient error <= 1e-3 against the FP64 oracle, uint8 equal to the
oracle's spatial filter outside the 1e-4 tie band.  The number of terms
equals the mask's rank.
"""
import numpy as np
import pytest
import torch

import datagen
import oracle

pytestmark = pytest.mark.gpu
COEF_TOL = 1e-3
BAND = 1e-4


def run(dctf, op, x, inplace=False):
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    yd = xd if inplace else torch.empty_like(xd)
    dctf.apply(op, xd, x.shape[0], yd)
    torch.cuda.synchronize()
    return yd.cpu().numpy().astype(np.float64)


CASES = [   # n, mask, anchor, boundary, expected rank
    (8, "headline", (1, 3), 1, 5),
    (8, "gauss3", (1, 1), 0, 1),
    (8, "laplacian", (1, 1), 0, 2),
    (8, "magic", (1, 1), 1, 3),
    (8, "motion", (0, 2), 1, 1),
    (16, "large", (4, 4), 1, 9),
    (16, "gauss7", (3, 3), 0, 1),
    (4, "rand3x2", (2, 1), 1, 2),
]


def mask_of(name):
    g = np.random.default_rng(61)
    return {"headline": datagen.headline_mask(), "gauss3": datagen.gaussian_mask(3, 1.0),
            "laplacian": datagen.laplacian_sharpen(), "magic": datagen.magic_square_3(),
            "motion": datagen.motion_blur_1x5(), "large": datagen.large_mask(),
            "gauss7": datagen.gaussian_mask(7, 2.0), "rand3x2": g.uniform(-1, 1, (3, 2))}[name]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_kron_matches_oracle(dctf, case):
    n, name, a, bnd, rank = CASES[case]
    w = mask_of(name)
    img = datagen.synthetic_image(256, 320, datagen.rng(98, case, 0))
    blocks = oracle.image_to_blocks(img, n)
    x = oracle.dct2_blocks(blocks).astype(np.float32)
    op = dctf.build_operator(w, a, n, bnd, kron=True)
    assert op.kron_rank() == rank == len(oracle.mask_rank_terms(w))
    op.set_precision(dctf.KRON_FP32)
    y = run(dctf, op, x)
    y_ref = oracle.apply_M(oracle.build_M(w, a, n, bnd), x.astype(np.float64))
    # an unnormalised mask scales the outputs (the magic square: by 45, to
    # ~3e4, where one FP32 ulp is 2e-3): the bar scales with them
    assert np.abs(y - y_ref).max() <= COEF_TOL * max(1.0, abs(w.sum()))
    st = oracle.uint8_compare(oracle.spatial_filter_blocks(blocks, w, a, bnd),
                              oracle.to_uint8(oracle.idct2_blocks(y, n)), BAND)
    assert st["mismatch"] == 0, st
    op.release()


@pytest.mark.parametrize("nb", [1, 15, 17, 1000, 40001])
def test_kron_ragged_and_in_place(dctf, nb):
    img = datagen.synthetic_image(3200, 3200, datagen.rng(98, 100, 0))
    x = oracle.dct2_blocks(oracle.image_to_blocks(img, 16))[:nb].astype(np.float32)
    w, a = datagen.large_mask(), (4, 4)
    op = dctf.build_operator(w, a, 16, dctf.REPLICATE, kron=True)
    op.set_precision(dctf.KRON_FP32)
    y = run(dctf, op, x)
    y_ref = oracle.apply_M(oracle.build_M(w, a, 16, oracle.REPLICATE), x.astype(np.float64))
    assert np.abs(y - y_ref).max() <= COEF_TOL
    assert np.array_equal(run(dctf, op, x, inplace=True), y)
    op.release()


def test_kron_rebuild_and_flags(dctf):
    g = np.random.default_rng(62)
    op = dctf.build_operator(datagen.gaussian_mask(3, 1.0), (1, 1), 8, dctf.ZERO, kron=True)
    assert op.kron_rank() == 1
    w2 = g.uniform(-1, 1, (4, 4))
    op.rebuild(w2, (0, 3), dctf.REPLICATE)
    assert op.kron_rank() == 4
    op.set_precision(dctf.KRON_FP32)
    x = oracle.dct2_blocks(oracle.image_to_blocks(
        datagen.synthetic_image(64, 64, g), 8)).astype(np.float32)
    y = run(dctf, op, x)
    y_ref = oracle.apply_M(oracle.build_M(w2, (0, 3), 8, oracle.REPLICATE), x.astype(np.float64))
    assert np.abs(y - y_ref).max() <= COEF_TOL
    # an all-zero mask has no terms and filters everything to zero
    op.rebuild(np.zeros((3, 3)), (1, 1), dctf.ZERO)
    assert op.kron_rank() == 0
    assert not run(dctf, op, x).any()
    op.release()
    plain = dctf.build_operator(datagen.gaussian_mask(3, 1.0), (1, 1), 8, dctf.ZERO)
    with pytest.raises(dctf.DctfError) as e:
        plain.set_precision(dctf.KRON_FP32)
    assert e.value.status == 6
    with pytest.raises(dctf.DctfError):
        plain.kron_rank()
    plain.release()


def test_kron_convolution(dctf):
    """The convolution flag composes with the Kronecker build."""
    import scipy.ndimage as nd
    g = np.random.default_rng(63)
    w = g.uniform(-1, 1, (3, 5))
    op = dctf.build_operator(w, (1, 2), 8, dctf.REPLICATE, convolution=True, kron=True)
    op.set_precision(dctf.KRON_FP32)
    blocks = g.integers(0, 256, (7, 8, 8)).astype(float)
    x = oracle.dct2_blocks(blocks).astype(np.float32)
    p = oracle.idct2_blocks(run(dctf, op, x), 8)
    for b in range(7):
        assert np.abs(p[b] - nd.convolve(blocks[b], w, mode="nearest")).max() < 2e-3
    op.release()
