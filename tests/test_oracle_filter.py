"""Pins for the oracle's spatial filter and operators (Sec. II.B-C, Eq. 5-20)
against brute force, scipy.ndimage and algebraic invariants."""
import itertools

import numpy as np
import pytest
import scipy.ndimage as nd

import oracle
from oracle import REPLICATE, ZERO


def brute_filter(block, w, anchor, boundary):
    """Direct per-pixel loops: the mask entry (r, c) reads pixel
    (i + r - ar, j + c - ac); outside the block it reads 0 (zero padding) or
    the nearest in-block pixel (border replication)."""
    n = block.shape[0]
    mh, mw = w.shape
    ar, ac = anchor
    out = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            acc = 0.0
            for r in range(mh):
                for c in range(mw):
                    s, t = i + r - ar, j + c - ac
                    if boundary == ZERO:
                        if 0 <= s < n and 0 <= t < n:
                            acc += w[r, c] * block[s, t]
                    else:
                        acc += w[r, c] * block[min(max(s, 0), n - 1), min(max(t, 0), n - 1)]
            out[i, j] = acc
    return out


@pytest.mark.parametrize("boundary", [ZERO, REPLICATE])
@pytest.mark.parametrize("mh,mw", [(1, 1), (1, 3), (2, 3), (3, 3), (4, 2), (4, 4)])
def test_spatial_filter_brute_force_4x4(boundary, mh, mw):
    g = np.random.default_rng(mh * 10 + mw)
    blocks = g.integers(0, 256, (3, 4, 4)).astype(float)
    w = g.uniform(-1, 1, (mh, mw))
    for anchor in itertools.product(range(mh), range(mw)):
        out = oracle.spatial_filter_blocks(blocks, w, anchor, boundary)
        for b in range(3):
            assert np.abs(out[b] - brute_filter(blocks[b], w, anchor, boundary)).max() < 1e-11
        # H is the same filter on the vectorised block
        h = oracle.build_H(w, anchor, 4, boundary)
        hv = blocks.reshape(3, 16) @ h.T
        assert np.abs(hv - out.reshape(3, 16)).max() < 1e-11


@pytest.mark.parametrize("boundary,mode", [(ZERO, "constant"), (REPLICATE, "nearest")])
def test_spatial_filter_matches_scipy_correlate(boundary, mode):
    g = np.random.default_rng(7)
    blocks = g.integers(0, 256, (4, 8, 8)).astype(float)
    for (mh, mw), anchor in [((3, 3), (1, 1)), ((5, 5), (1, 3)), ((1, 5), (0, 2)),
                             ((7, 7), (3, 3)), ((4, 6), (3, 0)), ((8, 8), (0, 7))]:
        w = g.uniform(-1, 1, (mh, mw))
        out = oracle.spatial_filter_blocks(blocks, w, anchor, boundary)
        origin = (anchor[0] - mh // 2, anchor[1] - mw // 2)
        for b in range(4):
            ref = nd.correlate(blocks[b], w, mode=mode, cval=0.0, origin=origin)
            assert np.abs(out[b] - ref).max() < 1e-10


def test_delta_mask_is_identity():
    for n in (4, 8, 16):
        for boundary in (ZERO, REPLICATE):
            w = np.zeros((3, 3))
            w[1, 1] = 1.0
            assert np.abs(oracle.build_H(w, (1, 1), n, boundary) - np.eye(n * n)).max() == 0
            assert np.abs(oracle.build_M(w, (1, 1), n, boundary) - np.eye(n * n)).max() < 1e-13


def test_mask_must_fit_block():
    with pytest.raises(ValueError):
        oracle.build_H(np.ones((5, 5)), (2, 2), 4, ZERO)
    with pytest.raises(ValueError):
        oracle.build_H(np.ones((3, 3)), (3, 1), 8, ZERO)


def one_d_operator(v, a, n, boundary):
    """1-D filter along one axis: out[i] = sum_r v[r] x[P(i + r - a)]."""
    h = np.zeros((n, n))
    for i in range(n):
        for r in range(len(v)):
            s = i + r - a
            if boundary == ZERO:
                if 0 <= s < n:
                    h[i, s] += v[r]
            else:
                h[i, min(max(s, 0), n - 1)] += v[r]
    return h


@pytest.mark.parametrize("boundary", [ZERO, REPLICATE])
@pytest.mark.parametrize("n", [4, 8, 16])
def test_separable_mask_gives_kronecker_operator(boundary, n):
    g = np.random.default_rng(n + boundary)
    mh, mw = min(n, 5), min(n, 3)
    v, hh = g.uniform(-1, 1, mh), g.uniform(-1, 1, mw)
    anchor = (mh - 2, 0)
    m = oracle.build_M(np.outer(v, hh), anchor, n, boundary)
    c = oracle.dct_matrix(n)
    mv = c @ one_d_operator(v, anchor[0], n, boundary) @ c.T
    mh_ = c @ one_d_operator(hh, anchor[1], n, boundary) @ c.T
    assert np.abs(m - np.kron(mv, mh_)).max() < 1e-12


@pytest.mark.parametrize("boundary", [ZERO, REPLICATE])
def test_operator_linear_in_mask(boundary):
    g = np.random.default_rng(3)
    w1, w2 = g.normal(size=(5, 5)), g.normal(size=(5, 5))
    m = lambda w: oracle.build_M(w, (1, 3), 8, boundary)
    assert np.abs(m(2.5 * w1 - 0.75 * w2) - (2.5 * m(w1) - 0.75 * m(w2))).max() < 1e-12


def test_replicate_constant_block_stays_constant():
    # border replication maps a constant block c to (sum w) c: column 0 of M
    g = np.random.default_rng(4)
    for n, (mh, mw) in [(4, (3, 2)), (8, (5, 5)), (16, (9, 9))]:
        w = g.uniform(-1, 1, (mh, mw))
        m = oracle.build_M(w, (mh // 2, mw - 1), n, REPLICATE)
        e0 = np.zeros(n * n)
        e0[0] = w.sum()
        assert np.abs(m[:, 0] - e0).max() < 1e-12


def test_zero_padding_transpose_is_rotated_mask():
    # with zero padding H[p, q] = w[q - p + a]; its transpose is the
    # rotated mask with the mirrored anchor
    g = np.random.default_rng(5)
    w = g.uniform(-1, 1, (3, 5))
    a = (0, 3)
    mt = oracle.build_M(w[::-1, ::-1], (2 - a[0], 4 - a[1]), 8, ZERO)
    assert np.abs(mt - oracle.build_M(w, a, 8, ZERO).T).max() < 1e-12


def test_operator_route_equals_spatial_route_fp64():
    # vec(F) = M vec(BLOCK) is the spatial filter seen through the DCT
    g = np.random.default_rng(6)
    for n, boundary in [(4, ZERO), (8, REPLICATE), (16, ZERO), (16, REPLICATE)]:
        blocks = g.integers(0, 256, (6, n, n)).astype(float)
        w = g.uniform(-1, 1, (min(n, 7), min(n, 4)))
        a = (1, 2)
        p_spatial = oracle.spatial_filter_blocks(blocks, w, a, boundary)
        p_dct = oracle.idct2_blocks(
            oracle.apply_M(oracle.build_M(w, a, n, boundary), oracle.dct2_blocks(blocks)), n)
        assert np.abs(p_spatial - p_dct).max() < 1e-9


def test_convolution_is_rotated_correlation():
    """The convolution reading of Eq. 5 equals the correlation of the oracle
    with the rotated mask and mirrored anchor (scipy.ndimage.convolve)."""
    g = np.random.default_rng(24)
    w = g.uniform(-1, 1, (3, 5))
    blocks = g.integers(0, 256, (3, 8, 8)).astype(float)
    out = oracle.spatial_filter_blocks(blocks, w[::-1, ::-1], (3 - 1 - 1, 5 - 1 - 2), REPLICATE)
    for b in range(3):
        assert np.abs(out[b] - nd.convolve(blocks[b], w, mode="nearest")).max() < 1e-10
