"""Pins for the oracle's Kronecker (sandwich-product) form of the operator
(Sec. II.B Eq. 11-12, Sec. II.C Eq. 20): M = sum_t A_t kron B_t with as many
terms as the mask's rank.

The Kronecker factors come from the mask's SVD and 1-D filters; build_M
comes from the 2-D loops of build_H.  The two constructions share nothing
but the DCT matrix, so their agreement pins both."""
import numpy as np
import pytest

import datagen
import oracle
from oracle import REPLICATE, ZERO


def kron_sum(factors):
    return sum(np.kron(a, b) for a, b in factors)


MASKS = [
    ("random 5x5", lambda g: g.uniform(-1, 1, (5, 5)), (1, 3)),
    ("random 3x7", lambda g: g.uniform(-1, 1, (3, 7)), (2, 0)),
    ("magic square", lambda g: datagen.magic_square_3(), (1, 1)),
    ("laplacian", lambda g: datagen.laplacian_sharpen(), (1, 1)),
    ("gaussian 7x7", lambda g: datagen.gaussian_mask(7, 2.0), (3, 3)),
    ("motion blur 1x5", lambda g: datagen.motion_blur_1x5(), (0, 2)),
    ("perturbed 9x9", lambda g: datagen.large_mask(), (4, 4)),
]


@pytest.mark.parametrize("boundary", [ZERO, REPLICATE])
@pytest.mark.parametrize("k", range(len(MASKS)))
def test_kron_sum_equals_dense_operator(k, boundary):
    name, make, a = MASKS[k]
    w = make(np.random.default_rng(40 + k))
    n = 16 if w.shape[0] > 8 or w.shape[1] > 8 else 8
    f = oracle.kron_factors(w, a, n, boundary)
    assert np.abs(kron_sum(f) - oracle.build_M(w, a, n, boundary)).max() < 1e-12 * max(1, np.abs(w).sum())


def test_number_of_terms_is_the_mask_rank():
    g = np.random.default_rng(41)
    assert len(oracle.mask_rank_terms(np.outer(g.normal(size=4), g.normal(size=6)))) == 1
    assert len(oracle.mask_rank_terms(datagen.gaussian_mask(7, 2.0))) == 1     # separable
    assert len(oracle.mask_rank_terms(datagen.laplacian_sharpen())) == 2       # cross: 2 terms
    assert len(oracle.mask_rank_terms(datagen.magic_square_3())) == 3          # full rank
    assert len(oracle.mask_rank_terms(g.uniform(-1, 1, (5, 5)))) == 5
    assert len(oracle.mask_rank_terms(np.zeros((3, 3)))) == 0


def test_paper_3x3_zero_padding_has_three_terms():
    """Eq. 11 writes the zero-padding operator of a 3x3 mask as three
    Kronecker terms; a generic 3x3 mask has rank 3, so the sum of three
    rank-1 terms is the whole operator and no fewer can be."""
    g = np.random.default_rng(42)
    w = g.uniform(-1, 1, (3, 3))
    f = oracle.kron_factors(w, (1, 1), 8, ZERO)
    assert len(f) == 3
    m = oracle.build_M(w, (1, 1), 8, ZERO)
    # Kronecker rank of M (rearrangement: rows (a-row, b-row), cols (a-col, b-col))
    r = m.reshape(8, 8, 8, 8).transpose(0, 2, 1, 3).reshape(64, 64)
    s = np.linalg.svd(r, compute_uv=False)
    assert (s > 1e-10 * s[0]).sum() == 3


@pytest.mark.parametrize("boundary", [ZERO, REPLICATE])
def test_sandwich_apply_equals_dense_apply(boundary):
    g = np.random.default_rng(43)
    img = datagen.synthetic_image(64, 96, g)
    x = oracle.dct2_blocks(oracle.image_to_blocks(img, 16))
    w, a = datagen.large_mask(), (4, 4)
    y_k = oracle.apply_kron(oracle.kron_factors(w, a, 16, boundary), x, 16)
    y_m = oracle.apply_M(oracle.build_M(w, a, 16, boundary), x)
    assert np.abs(y_k - y_m).max() < 1e-9


def test_filter_1d_brute_force():
    g = np.random.default_rng(44)
    v = g.uniform(-1, 1, 5)
    for boundary in (ZERO, REPLICATE):
        h = oracle.filter_1d(v, 3, 8, boundary)
        x = g.uniform(0, 255, 8)
        for i in range(8):
            acc = 0.0
            for r in range(5):
                s = i + r - 3
                if boundary == ZERO:
                    acc += v[r] * x[s] if 0 <= s < 8 else 0.0
                else:
                    acc += v[r] * x[min(max(s, 0), 7)]
            assert abs((h @ x)[i] - acc) < 1e-12
