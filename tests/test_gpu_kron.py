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


# ------------------------------------------- the sandwich products on tensor cores
TC_CASES = [   # mask, anchor, boundary, expected rank (terms: 1-4 groups of four)
    ("gauss7", (3, 3), 0, 1),
    ("gauss9", (4, 4), 1, 1),
    ("laplacian", (1, 1), 1, 2),
    ("magic", (1, 1), 1, 3),
    ("rand5", (1, 3), 0, 5),
    ("large", (4, 4), 1, 9),
    ("pgauss16", (7, 2), 1, 16),
]


def tc_mask(name):
    g = np.random.default_rng(64)
    if name == "gauss9":
        return datagen.gaussian_mask(9, 2.5)
    if name == "rand5":
        return g.uniform(-1, 1, (5, 5))
    if name == "pgauss16":      # full rank: a block-sized perturbed Gaussian
        return datagen.perturbed_gaussian(16, 4.0, 0.05, datagen.rng(98, 300, 0))
    return mask_of(name)


@pytest.fixture(scope="module")
def tc_source():
    img = datagen.synthetic_image(512, 768, datagen.rng(98, 200, 0))
    blocks = oracle.image_to_blocks(img, 16)
    return blocks, oracle.dct2_blocks(blocks).astype(np.float32)


@pytest.mark.parametrize("case", range(len(TC_CASES)))
def test_kron_tc_matches_oracle(dctf, tc_source, case):
    """DCTF_KRON_F16X3: Z_t = X B_t^T and Y = sum_t A_t Z_t as F16X3
    tensor-core products, held to the same bars as every exact arithmetic."""
    name, a, bnd, rank = TC_CASES[case]
    w = tc_mask(name)
    blocks, x = tc_source
    op = dctf.build_operator(w, a, 16, bnd, kron=True)
    assert op.kron_rank() == rank == len(oracle.mask_rank_terms(w))
    op.set_precision(dctf.KRON_F16X3)
    y = run(dctf, op, x)
    assert op.status() == 0
    y_ref = oracle.apply_M(oracle.build_M(w, a, 16, bnd), x.astype(np.float64))
    err = np.abs(y - y_ref).max()
    op_dense = dctf.build_operator(w, a, 16, bnd)
    err_dense = np.abs(run(dctf, op_dense, x) - y_ref).max()     # dense F16X3, for the record
    op_dense.release()
    print(f"KRON_F16X3 {name} rank {rank}: max coefficient error {err:.3g} "
          f"(dense F16X3 {err_dense:.3g})")
    assert err <= COEF_TOL * max(1.0, abs(w.sum()))
    # the same operator in its Kronecker form, applied by the oracle
    y_kron = oracle.apply_kron(oracle.kron_factors(w, a, 16, bnd), x, 16)
    assert np.abs(y - y_kron).max() <= COEF_TOL * max(1.0, abs(w.sum()))
    st = oracle.uint8_compare(oracle.spatial_filter_blocks(blocks, w, a, bnd),
                              oracle.to_uint8(oracle.idct2_blocks(y, 16)), BAND)
    assert st["mismatch"] == 0, st
    op.release()


@pytest.mark.parametrize("nb", [1, 7, 8, 9, 1000, 40001])
def test_kron_tc_ragged_and_in_place(dctf, nb):
    """Units of 8 blocks: counts that leave a partial unit and CTAs without
    work; in place gives the same bits."""
    img = datagen.synthetic_image(3200, 3200, datagen.rng(98, 101, 0))
    x = oracle.dct2_blocks(oracle.image_to_blocks(img, 16))[:nb].astype(np.float32)
    w, a = datagen.large_mask(), (4, 4)
    op = dctf.build_operator(w, a, 16, dctf.REPLICATE, kron=True)
    op.set_precision(dctf.KRON_F16X3)
    y = run(dctf, op, x)
    y_ref = oracle.apply_M(oracle.build_M(w, a, 16, oracle.REPLICATE), x.astype(np.float64))
    assert np.abs(y - y_ref).max() <= COEF_TOL
    assert np.array_equal(run(dctf, op, x, inplace=True), y)
    assert op.status() == 0
    op.release()


def test_kron_tc_rebuild_zero_mask_and_support(dctf, tc_source):
    """The number of terms is read on the device at each launch: a rebuild
    that changes it needs nothing from the host; a zero mask (no terms)
    filters to zero; the variant exists for 16 x 16 blocks only."""
    _, x = tc_source
    op = dctf.build_operator(datagen.gaussian_mask(9, 2.5), (4, 4), 16, dctf.ZERO, kron=True)
    op.set_precision(dctf.KRON_F16X3)
    for w, a, bnd in ((datagen.magic_square_3(), (1, 1), 1), (tc_mask("rand5"), (2, 2), 0),
                      (datagen.gaussian_mask(3, 1.0), (1, 1), 1)):
        op.rebuild(w, a, bnd)
        y = run(dctf, op, x)
        y_ref = oracle.apply_M(oracle.build_M(w, a, 16, bnd), x.astype(np.float64))
        assert np.abs(y - y_ref).max() <= COEF_TOL * max(1.0, abs(w.sum()))
    op.rebuild(np.zeros((5, 5)), (2, 2), dctf.ZERO)
    assert op.kron_rank() == 0
    assert not run(dctf, op, x).any()
    assert op.status() == 0
    op.release()
    op8 = dctf.build_operator(datagen.gaussian_mask(3, 1.0), (1, 1), 8, dctf.ZERO, kron=True)
    with pytest.raises(dctf.DctfError) as e:
        op8.set_precision(dctf.KRON_F16X3)
    assert e.value.status == 6
    op8.release()


def test_kron_tc_inputs_ready_same_bits(dctf, tc_source):
    """DCTF_KRON_F16X3 under DCTF_APPLY_INPUTS_READY (programmatic stream
    serialisation): applies queued back to back into different outputs give
    the bits of an ordinary launch."""
    _, x = tc_source
    op = dctf.build_operator(datagen.large_mask(), (4, 4), 16, dctf.REPLICATE, kron=True)
    op.set_precision(dctf.KRON_F16X3)
    y_plain = run(dctf, op, x)
    op.set_flags(dctf.APPLY_INPUTS_READY)
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    outs = [torch.full_like(xd, float("nan")) for _ in range(4)]
    for _ in range(2):
        for yd in outs:
            dctf.apply(op, xd, x.shape[0], yd)
    torch.cuda.synchronize()
    for yd in outs:
        assert np.array_equal(yd.cpu().numpy().astype(np.float64), y_plain)
    assert op.status() == 0
    op.release()
