"""The paper's validation (Sec. III): DCT-domain filtering and spatial filtering
give the same uint8 pixels, on the paper's two experiments (3x3 Gaussian
sigma=1, zero padding and replication; order-3 magic square, replication),
plus the rounding and int16 requantisation helpers against special cases."""
import numpy as np
import pytest

import datagen
import oracle
from oracle import REPLICATE, ZERO


def routes(img, n, w, a, boundary):
    blocks = oracle.image_to_blocks(img, n)
    p_sp = oracle.spatial_filter_blocks(blocks, w, a, boundary)
    p_dct = oracle.coefficient_route(oracle.dct2_blocks(blocks), n, w, a, boundary)
    return p_sp, p_dct


@pytest.mark.parametrize("boundary", [ZERO, REPLICATE])
def test_experiment1_gaussian_uint8_equal(boundary):
    job = datagen.small_job()
    p_sp, p_dct = routes(job.image, 8, job.mask, job.anchor, boundary)
    assert np.abs(p_sp - p_dct).max() < 1e-10
    st = oracle.uint8_compare(p_sp, oracle.to_uint8(p_dct), band=1e-9)
    assert st["mismatch"] == 0


def test_experiment2_magic_square_uint8_equal():
    img = datagen.synthetic_image(64, 64, datagen.rng(99, 0, 0))
    w = datagen.magic_square_3()
    p_sp, p_dct = routes(img, 8, w, (1, 1), REPLICATE)
    assert np.abs(p_sp - p_dct).max() < 1e-8
    st = oracle.uint8_compare(p_sp, oracle.to_uint8(p_dct), band=1e-9)
    assert st["mismatch"] == 0
    # an unnormalised mask summing to 45 saturates nearly every pixel
    assert (oracle.to_uint8(p_sp) == 255).mean() > 0.9


def test_round_half_away_special_cases():
    v = np.array([-2.5, -1.5, -0.5, -0.49, 0.0, 0.49, 0.5, 1.5, 2.5, 254.5, 255.5])
    assert oracle.round_half_away(v).tolist() == [-3, -2, -1, -0, 0, 0, 1, 2, 3, 255, 256]
    assert oracle.to_uint8(v).tolist() == [0, 0, 0, 0, 0, 0, 1, 2, 3, 255, 255]


def test_uint8_compare_band():
    p = np.array([10.49995, 10.2, 300.0, -7.0, 99.5])
    t = np.array([11, 10, 255, 0, 99], dtype=np.uint8)
    st = oracle.uint8_compare(p, t)
    assert st == {"mismatch": 0, "band": 2, "total": 5}
    st = oracle.uint8_compare(p, np.array([11, 11, 255, 0, 99], dtype=np.uint8))
    assert st["mismatch"] == 1


def test_requantise_special_cases():
    q = np.full(64, 4, dtype=np.uint16)
    y = np.zeros((1, 64))
    y[0, :6] = [2.0, -2.0, 6.0, 1e7, -1e7, 1.9]
    out = oracle.requantise(y, q)
    assert out[0, :6].tolist() == [1, -1, 2, 32767, -32768, 0]
    x = oracle.dequantise(np.array([[3] * 64], dtype=np.int16), datagen.quant_table(2))
    assert x[0, 0] == 3 * 3 and x[0, 63] == 3 * (1 + 2 * 15)


def test_serve_blocks_identity_mask():
    # a delta mask with equal quant tables returns the input exactly
    g = np.random.default_rng(8)
    qin = g.integers(-200, 200, (10, 64)).astype(np.int16)
    qt = datagen.quant_table(2)
    w = np.zeros((3, 3))
    w[1, 1] = 1
    out, _ = oracle.serve_blocks(qin, qt, oracle.build_M(w, (1, 1), 8, ZERO), qt)
    assert (out == qin).all()
