"""Pin of the oracle's operator M to the paper's own construction.

The paper builds the 3x3-mask filter of an 8x8 block from printed matrices
(Sec. II.B, Eq. 6-11, zero padding) plus six border-replication terms
(Sec. II.C, Eq. 13-20).  Those matrices are transcribed symbolically in
tests/golden/paper_matrices_3x3_n8.txt; this test substitutes a mask into
them, forms the DCT-domain versions X = C x C^T (the reading of Eq. 7 that
agrees with Eq. 1 and 3), evaluates Eq. 8-11 and Eq. 13-20, and compares
with the oracle's M = K H K^T.  A wrong sign, index, anchor, transposition
or boundary rule in the oracle fails here.
"""
import os

import numpy as np
import pytest

import oracle
from oracle import REPLICATE, ZERO

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_matrices_3x3_n8.txt")


def load_symbolic():
    mats, cur = {}, None
    with open(GOLDEN) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if not line:
                continue
            if line.startswith("matrix"):
                cur = line.split()[1]
                mats[cur] = []
            else:
                mats[cur].append(line.split())
    for k, v in mats.items():
        assert len(v) == 8 and all(len(r) == 8 for r in v), k
    return mats


def evaluate(sym, w):
    """Substitute mask values: wRC (Eq. 4) and wK (Sec. II.C, row-major)."""
    val = {}
    for r in range(3):
        for c in range(3):
            val[f"w{r + 1}{c + 1}"] = w[r, c]
            val[f"w{3 * r + c + 1}"] = w[r, c]
    out = np.zeros((8, 8))
    for i in range(8):
        for j in range(8):
            tot = 0.0
            for term in sym[i][j].split("+"):
                tot += float(term) if term in ("0", "1") else val[term]
            out[i, j] = tot
    return out


@pytest.fixture(scope="module")
def sym():
    return load_symbolic()


def paper_filter(sym, w, block_dct, replicate):
    c = oracle.dct_matrix(8)
    D = {k: c @ evaluate(v, w) @ c.T for k, v in sym.items()}   # X = C x C^T
    X = block_dct
    P = D["a"] @ X @ D["b"]                          # Eq. 8
    Q = X @ D["c"]                                   # Eq. 9
    R = D["d"] @ X @ D["e"]                          # Eq. 10
    F = P + Q + R                                    # Eq. 11
    if not replicate:
        return F
    repl = (D["b_r"] @ X @ D["bott_cor"]             # Eq. 13
            + D["u_l"] @ X @ D["up_cor"]             # Eq. 14
            + D["right"] @ X @ D["b_r"]              # Eq. 15
            + D["left"] @ X @ D["u_l"]               # Eq. 16
            + D["u_l"] @ X @ D["up"]                 # Eq. 17
            + D["b_r"] @ X @ D["bottom"])            # Eq. 18, 19
    return F + repl                                  # Eq. 20


@pytest.mark.parametrize("boundary", [ZERO, REPLICATE])
def test_paper_equations_equal_oracle_operator(sym, boundary):
    g = np.random.default_rng(11)
    for trial in range(5):
        w = g.uniform(-1, 1, (3, 3))                 # asymmetric, inseparable
        m = oracle.build_M(w, (1, 1), 8, boundary)
        blocks = g.integers(0, 256, (4, 8, 8)).astype(float)
        x = oracle.dct2_blocks(blocks)
        y = oracle.apply_M(m, x)
        for b in range(4):
            f = paper_filter(sym, w, x[b].reshape(8, 8), boundary == REPLICATE)
            assert np.abs(f.ravel() - y[b]).max() < 1e-10


def test_paper_magic_square_replicate(sym):
    # second experiment of Sec. III: order-3 magic square, border replication
    w = np.array([[8., 1., 6.], [3., 5., 7.], [4., 9., 2.]])
    m = oracle.build_M(w, (1, 1), 8, REPLICATE)
    g = np.random.default_rng(12)
    x = oracle.dct2_blocks(g.integers(0, 256, (3, 8, 8)).astype(float))
    y = oracle.apply_M(m, x)
    for b in range(3):
        f = paper_filter(sym, w, x[b].reshape(8, 8), True)
        assert np.abs(f.ravel() - y[b]).max() < 1e-9


def test_symmetric_simplification_eq12(sym):
    # when mask rows 1 and 3 agree, b = e and F = (A + D) BLOCK E + BLOCK C
    g = np.random.default_rng(13)
    w = g.uniform(-1, 1, (3, 3))
    w[2] = w[0]
    c = oracle.dct_matrix(8)
    D = {k: c @ evaluate(v, w) @ c.T for k, v in sym.items()}
    assert np.abs(D["b"] - D["e"]).max() < 1e-14
    x = oracle.dct2_blocks(g.integers(0, 256, (1, 8, 8)).astype(float))
    X = x[0].reshape(8, 8)
    f12 = (D["a"] + D["d"]) @ X @ D["e"] + X @ D["c"]
    y = oracle.apply_M(oracle.build_M(w, (1, 1), 8, ZERO), x)
    assert np.abs(f12.ravel() - y[0]).max() < 1e-10


def test_spatial_matrices_are_the_correlation(sym):
    # the printed spatial products a x b + x c + d x e (Eq. 6, 9, 10 before
    # the DCT) equal the zero-padded correlation with the centred anchor
    g = np.random.default_rng(14)
    w = g.uniform(-1, 1, (3, 3))
    blk = g.integers(0, 256, (8, 8)).astype(float)
    s = {k: evaluate(v, w) for k, v in sym.items()}
    p = s["a"] @ blk @ s["b"] + blk @ s["c"] + s["d"] @ blk @ s["e"]
    ref = oracle.spatial_filter_blocks(blk[None], w, (1, 1), ZERO)[0]
    assert np.abs(p - ref).max() < 1e-11
