"""Pins for the oracle's DCT (Sec. II.A, Eq. 1-3) against closed forms and an
independent library transform (scipy.fft's orthonormal DCT-II)."""
import math

import numpy as np
import pytest
import scipy.fft

import oracle


@pytest.mark.parametrize("n", [4, 8, 16])
def test_dct_matrix_orthonormal(n):
    c = oracle.dct_matrix(n)
    assert np.abs(c @ c.T - np.eye(n)).max() < 1e-14          # Eq. 2
    assert np.allclose(c[0], 1.0 / math.sqrt(n), atol=1e-15, rtol=0)


@pytest.mark.parametrize("n", [4, 8, 16])
def test_dct_matrix_matches_scipy(n):
    # column x of C is the DCT-II of the unit vector e_x
    ref = scipy.fft.dct(np.eye(n), type=2, norm="ortho", axis=0)
    assert np.abs(oracle.dct_matrix(n) - ref).max() < 1e-14


def test_dct8_known_entries():
    c = oracle.dct_matrix(8)
    assert c[1, 0] == pytest.approx(math.cos(math.pi / 16) / 2, abs=1e-15)
    assert c[4, 0] == pytest.approx(0.5 * math.cos(math.pi / 4), abs=1e-15)
    assert c[7, 7] == pytest.approx(0.5 * math.cos(math.pi * 15 * 7 / 16), abs=1e-15)


@pytest.mark.parametrize("n", [4, 8, 16])
def test_blockwise_dct_matches_scipy(n):
    g = np.random.default_rng(1)
    blocks = g.integers(0, 256, (37, n, n)).astype(np.float64)
    y = oracle.dct2_blocks(blocks)
    ref = scipy.fft.dctn(blocks, type=2, norm="ortho", axes=(1, 2)).reshape(-1, n * n)
    assert np.abs(y - ref).max() < 1e-10
    back = oracle.idct2_blocks(y, n)
    assert np.abs(back - blocks).max() < 1e-10                  # Eq. 3
    ref_back = scipy.fft.idctn(ref.reshape(-1, n, n), type=2, norm="ortho", axes=(1, 2))
    assert np.abs(back - ref_back).max() < 1e-10


def test_vec_order_row_major():
    # coefficient (u, v) of a block sits at u*n + v: a pure horizontal
    # cosine (varies along columns j) lands in row u = 0.
    n = 8
    c = oracle.dct_matrix(n)
    blk = np.tile(c[3], (n, 1))[None]                # rows identical
    y = oracle.dct2_blocks(blk).reshape(n, n)
    assert abs(y[0, 3] - math.sqrt(n)) < 1e-12
    y[0, 3] = 0
    assert np.abs(y).max() < 1e-12


def test_constant_block_and_parseval():
    n = 8
    y = oracle.dct2_blocks(np.full((1, n, n), 100.0))
    assert y[0, 0] == pytest.approx(n * 100.0)
    assert np.abs(y[0, 1:]).max() < 1e-11
    g = np.random.default_rng(2)
    b = g.normal(size=(5, n, n))
    assert np.allclose((oracle.dct2_blocks(b) ** 2).sum(1), (b.reshape(5, -1) ** 2).sum(1))


def test_blocks_roundtrip_raster_order():
    img = np.arange(16 * 24).reshape(16, 24)
    b = oracle.image_to_blocks(img, 8)
    assert b.shape == (6, 8, 8)
    assert b[1, 0, 0] == 8 and b[3, 0, 0] == 8 * 24        # raster order
    assert (oracle.blocks_to_image(b, 16, 24) == img).all()
