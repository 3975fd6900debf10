"""GPU: y_b = M x_b through the C ABI against the FP64 oracle.

Bars (stated once, used everywhere):
  * coefficients: max |y_gpu - y_oracle| <= 1e-3 (0-255 pixel scale), the
    oracle applied to the same FP32 input coefficients;
  * pixels: uint8 of the GPU result (inverse DCT, round half away, saturate)
    equals uint8 of the oracle's spatial-domain filter for every pixel whose
    FP64 value is not within 1e-4 of a .5 rounding boundary (those are counted).
"""
import numpy as np
import pytest
import torch

import datagen
import oracle

pytestmark = pytest.mark.gpu

COEF_TOL = 1e-3
BAND = 1e-4


def coeffs_of(img, n):
    blocks = oracle.image_to_blocks(img, n)
    return blocks, oracle.dct2_blocks(blocks)


def run(dctf, op, x32, prec, inplace=False):
    op.set_precision(prec)
    xd = torch.from_numpy(np.ascontiguousarray(x32)).cuda()
    yd = xd if inplace else torch.empty_like(xd)
    dctf.apply(op, xd, x32.shape[0], yd)
    torch.cuda.synchronize()
    return yd.cpu().numpy().astype(np.float64)


def check(y, x32, blocks, w, a, n, boundary, pixels=True):
    y_ref = oracle.apply_M(oracle.build_M(w, a, n, boundary), x32.astype(np.float64))
    err = np.abs(y - y_ref).max()
    assert err <= COEF_TOL, f"max coefficient error {err}"
    if pixels:
        p_sp = oracle.spatial_filter_blocks(blocks, w, a, boundary)
        st = oracle.uint8_compare(p_sp, oracle.to_uint8(oracle.idct2_blocks(y, n)), BAND)
        assert st["mismatch"] == 0, st
    return err


def precisions(n, dctf):
    """The variants held to the bar for block size n (TF32X1 and BF16X3 are
    not: see test_tf32x1_error_bound, test_bf16x3_error_bound)."""
    if n == 16:
        return [dctf.FP32_SIMT, dctf.F16X3, dctf.BF16X6, dctf.TF32X3]
    return [dctf.FP32_SIMT, dctf.F16X3] if n == 8 else [dctf.FP32_SIMT]


def n16_tc(dctf):
    return [dctf.F16X3, dctf.BF16X6, dctf.TF32X3, dctf.TF32X1, dctf.BF16X3]


@pytest.fixture(scope="module")
def ragged_source():
    img = datagen.synthetic_image(2048, 1280, datagen.rng(90, 0, 0))
    blocks, x = coeffs_of(img, 8)
    return blocks, x.astype(np.float32)


@pytest.mark.parametrize("nb", [1, 5, 127, 128, 129, 255, 1000, 16384 + 77, 40960])
@pytest.mark.parametrize("prec", ["simt", "f16x3"])
def test_ragged_block_counts(dctf, ragged_source, nb, prec):
    blocks, x = ragged_source
    w, a = datagen.headline_mask(), (1, 3)
    op = dctf.build_operator(w, a, 8, dctf.REPLICATE)
    p = dctf.FP32_SIMT if prec == "simt" else dctf.F16X3
    y = run(dctf, op, x[:nb], p)
    check(y, x[:nb], blocks[:nb], w, a, 8, oracle.REPLICATE)
    assert op.status() == 0


def test_simt_tile_configs_agree(dctf, ragged_source):
    """Below 128 x (SM count) blocks the CUDA-core kernel uses 16-block
    tiles; each output sums the same terms in the same order, so both tile
    shapes give the same bits."""
    blocks, x = ragged_source
    w, a = datagen.headline_mask(), (1, 3)
    op = dctf.build_operator(w, a, 8, dctf.REPLICATE)
    cut = 128 * torch.cuda.get_device_properties(0).multi_processor_count
    assert x.shape[0] > cut
    y_big = run(dctf, op, x[:cut], dctf.FP32_SIMT)           # 128-block tiles
    y_small = run(dctf, op, x[:cut - 1], dctf.FP32_SIMT)     # 16-block tiles
    assert np.array_equal(y_big[:cut - 1], y_small)
    check(y_small[:2000], x[:2000], blocks[:2000], w, a, 8, oracle.REPLICATE)
    op.release()


@pytest.mark.parametrize("nb", [1, 31, 33, 63, 65, 1000, 40000])
def test_simt16_double_buffered_same_bits(dctf, n16_source, nb):
    """16x16 FP32 CUDA cores: the kernel that streams M's chunks double-
    buffered (FP32 input) gives the same bits as the single-buffered kernel
    (taken by the FP64-input entry point, fed the same values), and both meet
    the oracle."""
    blocks, x = n16_source
    x, blocks = x[:nb], blocks[:nb]
    w, a = datagen.large_mask(), (4, 4)
    op = dctf.build_operator(w, a, 16, dctf.REPLICATE)
    y_db = run(dctf, op, x, dctf.FP32_SIMT)
    xd = torch.from_numpy(x.astype(np.float64)).cuda()
    yd = torch.empty(x.shape, dtype=torch.float32, device="cuda")
    dctf.apply_f64in(op, xd, nb, yd)
    torch.cuda.synchronize()
    assert np.array_equal(y_db, yd.cpu().numpy().astype(np.float64))
    check(y_db, x, blocks, w, a, 16, oracle.REPLICATE)
    assert np.array_equal(run(dctf, op, x, dctf.FP32_SIMT, inplace=True), y_db)
    op.release()


def test_small_workload_fp64_coefficients(dctf):
    """256x256, 3x3 Gaussian sigma=1, zero padding, FP64 coefficients in."""
    job = datagen.small_job()
    blocks, x64 = coeffs_of(job.image, 8)
    op = dctf.build_operator(job.mask, job.anchor, 8, job.boundary)
    xd = torch.from_numpy(x64).cuda()
    yd = torch.empty(x64.shape, dtype=torch.float32, device="cuda")
    dctf.apply_f64in(op, xd, x64.shape[0], yd)
    torch.cuda.synchronize()
    y = yd.cpu().numpy().astype(np.float64)
    y_ref = oracle.apply_M(oracle.build_M(job.mask, job.anchor, 8, job.boundary), x64)
    assert np.abs(y - y_ref).max() <= COEF_TOL
    p_sp = oracle.spatial_filter_blocks(blocks, job.mask, job.anchor, job.boundary)
    assert oracle.uint8_compare(p_sp, oracle.to_uint8(oracle.idct2_blocks(y, 8)))["mismatch"] == 0
    for p in precisions(8, dctf):
        check(run(dctf, op, x64.astype(np.float32), p), x64.astype(np.float32), blocks,
              job.mask, job.anchor, 8, job.boundary)


@pytest.mark.parametrize("prec", ["simt", "f16x3"])
def test_headline_mask_1024(dctf, prec):
    job = datagen.headline_job(1024, 1024)
    blocks, x = coeffs_of(job.image, 8)
    x = x.astype(np.float32)
    op = dctf.build_operator(job.mask, job.anchor, 8, job.boundary)
    p = dctf.FP32_SIMT if prec == "simt" else dctf.F16X3
    check(run(dctf, op, x, p), x, blocks, job.mask, job.anchor, 8, job.boundary)


@pytest.mark.parametrize("i", range(8))
def test_grouped_masks(dctf, i):
    """The four masks of the grouped batch with both boundary modes."""
    w, a, boundary, _ = datagen.grouped_mask(i)
    img = datagen.synthetic_image(256, 384, datagen.rng(91, i, 0))
    blocks, x = coeffs_of(img, 8)
    x = x.astype(np.float32)
    op = dctf.build_operator(w, a, 8, boundary)
    for p in precisions(8, dctf):
        check(run(dctf, op, x, p), x, blocks, w, a, 8, boundary)


def test_magic_square_replicate(dctf):
    """Second experiment of Sec. III: unnormalised order-3 magic square."""
    img = datagen.synthetic_image(256, 256, datagen.rng(92, 0, 0))
    blocks, x = coeffs_of(img, 8)
    x = x.astype(np.float32)
    w = datagen.magic_square_3()
    op = dctf.build_operator(w, (1, 1), 8, dctf.REPLICATE)
    for p in precisions(8, dctf):
        y = run(dctf, op, x, p)
        y_ref = oracle.apply_M(oracle.build_M(w, (1, 1), 8, oracle.REPLICATE), x.astype(np.float64))
        # outputs reach 45 x 2040: the bar scales with the output magnitude
        assert np.abs(y - y_ref).max() <= COEF_TOL * 45
        p_sp = oracle.spatial_filter_blocks(blocks, w, (1, 1), oracle.REPLICATE)
        st = oracle.uint8_compare(p_sp, oracle.to_uint8(oracle.idct2_blocks(y, 8)), BAND)
        assert st["mismatch"] == 0


@pytest.mark.parametrize("n", [4, 16])
def test_other_block_sizes(dctf, n):
    img = datagen.synthetic_image(256, 320, datagen.rng(93, n, 0))
    blocks, x = coeffs_of(img, n)
    x = x.astype(np.float32)
    if n == 16:
        w, a = datagen.large_mask(), (4, 4)
    else:
        w, a = datagen.uniform_random_mask(3, 4, datagen.rng(93, n, 1)), (2, 1)
    for boundary in (oracle.ZERO, oracle.REPLICATE):
        op = dctf.build_operator(w, a, n, boundary)
        for p in precisions(n, dctf):
            check(run(dctf, op, x, p), x, blocks, w, a, n, boundary)
        if n == 4:
            with pytest.raises(dctf.DctfError):
                op.set_precision(dctf.F16X3)
        else:
            for p in n16_tc(dctf):
                with pytest.raises(dctf.DctfError):
                    run(dctf, op, x, p, inplace=True)


def test_split_variants_need_16x16(dctf):
    op = dctf.build_operator(datagen.gaussian_mask(3, 1.0), (1, 1), 8, dctf.ZERO)
    for p in (dctf.BF16X6, dctf.TF32X1, dctf.TF32X3, dctf.BF16X3):
        with pytest.raises(dctf.DctfError) as e:
            op.set_precision(p)
        assert e.value.status == 6                          # EUNSUPPORTED
    op.release()


@pytest.mark.parametrize("prec", ["simt", "f16x3"])
def test_in_place(dctf, ragged_source, prec):
    blocks, x = ragged_source
    x = x[:3000]
    w, a = datagen.headline_mask(), (1, 3)
    op = dctf.build_operator(w, a, 8, dctf.REPLICATE)
    p = dctf.FP32_SIMT if prec == "simt" else dctf.F16X3
    y_sep = run(dctf, op, x, p)
    y_inp = run(dctf, op, x, p, inplace=True)
    assert np.array_equal(y_sep, y_inp)


def test_zero_blocks_and_bad_pointers(dctf):
    op = dctf.build_operator(datagen.gaussian_mask(3, 1.0), (1, 1), 8, dctf.ZERO)
    dctf.apply(op, 0, 0, 0)                       # nothing to do, nothing touched
    buf = torch.zeros(2 * 64 + 4, device="cuda")
    with pytest.raises(dctf.DctfError):
        dctf.apply(op, buf.data_ptr() + 4, 2, buf.data_ptr() + 4 + 512)   # misaligned
    with pytest.raises(dctf.DctfError):
        dctf.apply(op, buf.data_ptr(), 2, buf.data_ptr() + 256)           # partial overlap
    with pytest.raises(dctf.DctfError):
        dctf.apply(op, buf.data_ptr(), -1, buf.data_ptr())


def test_forward_and_inverse_dct(dctf):
    img = datagen.synthetic_image(64, 96, datagen.rng(94, 0, 0))
    for n in (4, 8, 16):
        blocks, x_ref = coeffs_of(img, n)
        imd = torch.from_numpy(img).cuda()
        c64 = torch.empty(x_ref.shape, dtype=torch.float64, device="cuda")
        dctf.forward_dct(imd, 64, 96, n, c64, f64=True)
        c32 = torch.empty(x_ref.shape, dtype=torch.float32, device="cuda")
        dctf.forward_dct(imd, 64, 96, n, c32)
        torch.cuda.synchronize()
        assert np.abs(c64.cpu().numpy() - x_ref).max() < 1e-10
        assert np.abs(c32.cpu().numpy() - x_ref).max() < 2e-4
        back = torch.empty_like(imd)
        dctf.inverse_dct_u8(c32, 64, 96, n, back)
        torch.cuda.synchronize()
        assert np.array_equal(back.cpu().numpy(), img)


def test_apply_host_matches_device(dctf, ragged_source):
    _, x = ragged_source
    op = dctf.build_operator(datagen.headline_mask(), (1, 3), 8, dctf.REPLICATE)
    y_dev = run(dctf, op, x, dctf.F16X3)
    hin = torch.from_numpy(x).pin_memory()
    hout = torch.empty_like(hin).pin_memory()
    dctf.apply_host(op, hin, x.shape[0], hout)
    assert np.array_equal(hout.numpy().astype(np.float64), y_dev)
    # more blocks than one 8 MB chunk (full chunks take the pre-encoded
    # pipe items, the tail the general path), after a rebuild that changes
    # the operator's scale, and with the inputs-ready flag set (which the
    # host path must not apply: each apply follows its input copy)
    xx = np.concatenate([x] * 3)
    w2 = datagen.magic_square_3()
    op.rebuild(w2, (1, 1), dctf.REPLICATE)
    op.set_flags(dctf.APPLY_INPUTS_READY)
    y2 = run(dctf, op, xx, dctf.F16X3)
    hin2 = torch.from_numpy(xx).pin_memory()
    hout2 = torch.empty_like(hin2).pin_memory()
    for _ in range(2):
        hout2.zero_()
        dctf.apply_host(op, hin2, xx.shape[0], hout2)
        assert np.array_equal(hout2.numpy().astype(np.float64), y2)
    op.release()


@pytest.fixture(scope="module")
def headline_full():
    job = datagen.headline_job()           # 4096 x 4096, 262,144 blocks
    blocks, x = coeffs_of(job.image, 8)
    return job, blocks, x.astype(np.float32)


def test_full_size_headline_every_block(dctf, headline_full):
    """The full 4096x4096 workload in the benchmark's launch configuration:
    every block of both kernels against the oracle (coefficients and uint8
    pixels of the spatial filter), and the two kernels agree."""
    job, blocks, x = headline_full
    op = dctf.build_operator(job.mask, job.anchor, 8, job.boundary)
    y_tc = run(dctf, op, x, dctf.F16X3)
    y_simt = run(dctf, op, x, dctf.FP32_SIMT)
    for y in (y_tc, y_simt):
        check(y, x, blocks, job.mask, job.anchor, 8, job.boundary)
    assert np.abs(y_tc - y_simt).max() <= 2 * COEF_TOL
    assert op.status() == 0


@pytest.fixture(scope="module")
def n16_source():
    img = datagen.synthetic_image(3200, 3200, datagen.rng(96, 0, 0))
    blocks, x = coeffs_of(img, 16)
    return blocks, x.astype(np.float32)


@pytest.mark.parametrize("nb", [1, 127, 129, 255, 257, 1000, 40000])
@pytest.mark.parametrize("prec", ["F16X3", "BF16X6", "TF32X3"])
def test_n16_tensor_core_ragged(dctf, n16_source, nb, prec):
    """16x16 blocks, perturbed 9x9 Gaussian, border replication: the
    tensor-core kernels (outputs split over 2 or 4 CTAs, K-chunked input)
    on block counts that leave partial tiles (one block, a tile minus or
    plus one, two tiles minus or plus one) and idle CTA groups."""
    blocks, x = n16_source
    x, blocks = x[:nb], blocks[:nb]
    w, a = datagen.large_mask(), (4, 4)
    op = dctf.build_operator(w, a, 16, dctf.REPLICATE)
    check(run(dctf, op, x, getattr(dctf, prec)), x, blocks, w, a, 16, oracle.REPLICATE)
    assert op.status() == 0
    op.release()


def tf32x1_bound(m, x):
    """Bound on |y - M x| for TF32X1 from its arithmetic: x_k and M_jk each
    carry a relative rounding error <= 2^-11 (10 explicit mantissa bits,
    round to nearest), so each product is off by <= (2^-10 + 2^-22)|M_jk x_k|;
    the FP32 accumulation (32 chunked additions per accumulator, truncating)
    adds <= 2^-18 sum_k |M_jk x_k|; the DC term is exact to FP32 rounding."""
    s = np.abs(x[:, 1:]) @ np.abs(m[:, 1:]).T
    return (2.0**-10 + 2.0**-17) * s + 1e-5 * (1 + np.abs(x[:, :1]) * np.abs(m[:, 0])[None, :])


@pytest.mark.parametrize("boundary", [0, 1])
def test_tf32x1_error_bound(dctf, n16_source, boundary):
    """TF32X1 is not exact; its error stays inside the bound its arithmetic
    gives, and is far above the other splits' (so the variant is really
    running at TF32 precision)."""
    _, x = n16_source
    x = x[:5000]
    w, a = datagen.large_mask(), (4, 4)
    op = dctf.build_operator(w, a, 16, boundary)
    y = run(dctf, op, x, dctf.TF32X1)
    m = oracle.build_M(w, a, 16, boundary)
    y_ref = oracle.apply_M(m, x.astype(np.float64))
    err = np.abs(y - y_ref)
    assert (err <= tf32x1_bound(m, x.astype(np.float64))).all()
    assert err.max() > 1e-2
    op.release()


def bf16x3_bound(m, x):
    """Bound on |y - M x| for BF16X3 from its arithmetic.  BF16 keeps 8
    significant bits, so x0 = rn(x) is off by <= 2^-8 |x| and x1 = rn(x - x0)
    leaves x - x0 - x1 <= 2^-16 |x|; the same holds for M's pieces m0, m1.
    The three products miss x0 (M - m0 - m1) + x1 (M - m0) + (x - x0 - x1) M,
    <= 3 (1 + 2^-7) 2^-16 |M_jk x_k|; the truncating FP32 accumulation of 48
    MMAs per accumulator adds <= 2^-16 sum_k |M_jk x_k|; the DC term is exact
    to FP32 rounding."""
    s = np.abs(x[:, 1:]) @ np.abs(m[:, 1:]).T
    return (3 * (1 + 2.0**-7) + 1) * 2.0**-16 * s + 1e-5 * (1 + np.abs(x[:, :1]) * np.abs(m[:, 0])[None, :])


@pytest.mark.parametrize("boundary", [0, 1])
def test_bf16x3_error_bound(dctf, n16_source, boundary):
    """BF16X3 (the three-term split with BF16 hi/lo pieces) is not exact:
    its error stays inside the bound its arithmetic gives and lies well
    above the exact splits' (so the two-piece variant is what runs)."""
    _, x = n16_source
    x = x[:5000]
    w, a = datagen.large_mask(), (4, 4)
    op = dctf.build_operator(w, a, 16, boundary)
    y = run(dctf, op, x, dctf.BF16X3)
    m = oracle.build_M(w, a, 16, boundary)
    y_ref = oracle.apply_M(m, x.astype(np.float64))
    err = np.abs(y - y_ref)
    assert (err <= bf16x3_bound(m, x.astype(np.float64))).all()
    assert err.max() > 5e-4
    op.release()


def test_error_table_16x16(dctf, capsys):
    """Max coefficient error vs the FP64 oracle for each arithmetic on the
    16x16 workload's mask (perturbed 9x9 Gaussian, border replication),
    printed for the record; both stay within the bar."""
    img = datagen.synthetic_image(2048, 2048, datagen.rng(datagen.W_LARGE, 0, 0))
    blocks, x = coeffs_of(img, 16)
    x = x.astype(np.float32)
    w, a = datagen.large_mask(), (4, 4)
    op = dctf.build_operator(w, a, 16, dctf.REPLICATE)
    errs = {}
    for name in ("FP32_SIMT", "F16X3", "BF16X6", "TF32X3"):
        errs[name] = check(run(dctf, op, x, getattr(dctf, name)), x, blocks, w, a, 16,
                           oracle.REPLICATE)
    for name in ("TF32X1", "BF16X3"):
        y = run(dctf, op, x, getattr(dctf, name))
        errs[name] = np.abs(y - oracle.apply_M(oracle.build_M(w, a, 16, oracle.REPLICATE),
                                               x.astype(np.float64))).max()
    with capsys.disabled():
        print(f"\n16x16 max coefficient error: {errs}")


def test_inputs_ready_flag(dctf, ragged_source):
    """DCTF_APPLY_INPUTS_READY (programmatic dependent launch): chained
    applies give the same bits as ordinary launches, including when a launch
    overwrites the buffer the previous launch is still reading."""
    _, x = ragged_source
    w, a = datagen.headline_mask(), (1, 3)
    op = dctf.build_operator(w, a, 8, dctf.REPLICATE)
    xs = [torch.from_numpy(x).cuda() for _ in range(3)]
    ref = [torch.empty_like(xs[0]) for _ in range(3)]
    for i in range(3):
        dctf.apply(op, xs[i], x.shape[0], ref[i])
    torch.cuda.synchronize()
    op.set_flags(dctf.APPLY_INPUTS_READY)
    outs = [torch.full_like(xs[0], float("nan")) for _ in range(3)]
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        dctf.apply(op, xs[0], x.shape[0], outs[0], stream=s)
        torch.cuda.synchronize()
        with torch.cuda.graph(g, stream=s):
            for i in range(3):
                dctf.apply(op, xs[i], x.shape[0], outs[i], stream=s)
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    for i in range(3):
        assert torch.equal(outs[i], ref[i])
    # write-after-read: the second launch writes the first launch's input
    src = torch.from_numpy(x).cuda()
    y = torch.empty_like(src)
    other = torch.from_numpy(x[::-1].copy()).cuda()
    dctf.apply(op, src, x.shape[0], y)
    dctf.apply(op, other, x.shape[0], src)
    torch.cuda.synchronize()
    assert torch.equal(y, ref[0])
    op.set_flags(0)
    assert op.status() == 0


@pytest.mark.parametrize("prec", ["F16X3", "BF16X6", "TF32X3"])
def test_n16_inputs_ready_same_bits(dctf, n16_source, prec):
    """The 16x16 tensor-core applies under DCTF_APPLY_INPUTS_READY
    (programmatic stream serialisation): applies queued back to back, each
    writing a different output while the previous one finishes, give the
    bits of an ordinary launch."""
    _, x = n16_source
    x = x[:5000]
    w, a = datagen.large_mask(), (4, 4)
    op = dctf.build_operator(w, a, 16, dctf.REPLICATE)
    y_plain = run(dctf, op, x, getattr(dctf, prec))
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
