"""GPU: the FP64 operator builder against the oracle (steps a1-a2).

H is compared bit for bit (both sides add the same mask entries in the same
order); M = K H K^T within 1e-12 relative to sum|w| (FP64, different but
equivalent summation order: separable DCT passes on the device)."""
import numpy as np
import pytest

import datagen
import oracle

pytestmark = pytest.mark.gpu


def cases():
    g = np.random.default_rng(21)
    out = []
    for n in (4, 8, 16):
        out.append((n, datagen.gaussian_mask(3, 1.0), (1, 1)))
        out.append((n, g.uniform(-1, 1, (min(n, 4), min(n, 3))), (min(n, 4) - 1, 0)))
        out.append((n, np.array([[1.0]]), (0, 0)))
    out.append((8, datagen.headline_mask(), (1, 3)))
    out.append((8, datagen.magic_square_3(), (1, 1)))
    out.append((8, datagen.gaussian_mask(7, 2.0), (3, 3)))
    out.append((8, datagen.motion_blur_1x5(), (0, 2)))
    out.append((8, g.uniform(-1, 1, (8, 8)), (7, 0)))
    out.append((16, datagen.large_mask(), (4, 4)))
    out.append((16, g.uniform(-1, 1, (16, 11)), (3, 10)))
    return out


@pytest.mark.parametrize("boundary", [oracle.ZERO, oracle.REPLICATE])
@pytest.mark.parametrize("case", range(len(cases())))
def test_builder_matches_oracle(dctf, case, boundary):
    n, w, a = cases()[case]
    op = dctf.build_operator(w, a, n, boundary)
    m, h = op.download()
    h_ref = oracle.build_H(w, a, n, boundary)
    assert np.array_equal(h, h_ref)
    m_ref = oracle.build_M(w, a, n, boundary)
    scale = max(1.0, np.abs(w).sum())
    assert np.abs(m - m_ref).max() <= 1e-12 * scale
    op.release()


def test_rebuild_in_place(dctf):
    g = np.random.default_rng(22)
    w1, w2 = g.uniform(-1, 1, (3, 5)), g.uniform(-1, 1, (5, 2))
    op = dctf.build_operator(w1, (1, 1), 8, oracle.ZERO)
    op.rebuild(w2, (4, 0), oracle.REPLICATE)
    m, _ = op.download()
    assert np.abs(m - oracle.build_M(w2, (4, 0), 8, oracle.REPLICATE)).max() < 1e-12 * 8
    with pytest.raises(dctf.DctfError):
        op.rebuild(np.ones((9, 9)), (4, 4), oracle.ZERO)   # larger than the 8x8 block
    op.release()


def test_convolution_flag_matches_scipy_convolve(dctf):
    """DCTF_MASK_CONVOLUTION: the operator filters like scipy.ndimage.convolve
    on each block (checked through the built M and the oracle's inverse DCT)."""
    import scipy.ndimage as nd
    g = np.random.default_rng(23)
    w = g.uniform(-1, 1, (3, 5))
    a = (1, 2)                                 # centred: scipy's default origin
    op = dctf.build_operator(w, a, 8, dctf.REPLICATE, convolution=True)
    m, _ = op.download()
    blocks = g.integers(0, 256, (5, 8, 8)).astype(float)
    y = oracle.apply_M(m, oracle.dct2_blocks(blocks))
    p = oracle.idct2_blocks(y, 8)
    for b in range(5):
        ref = nd.convolve(blocks[b], w, mode="nearest")
        assert np.abs(p[b] - ref).max() < 1e-9
    op.release()
