"""GPU: fused coefficients -> filtered uint8 pixels (dctf_apply_pixels).

The image the kernel writes must equal uint8 of the oracle's spatial-domain
filter (Sec. II.B-C, round half away from zero, saturate: Sec. III) for every
pixel whose FP64 value is not within 1e-4 of a .5 rounding boundary; those
are counted.  Pitch padding must stay untouched.
"""
import numpy as np
import pytest
import torch

import datagen
import oracle

pytestmark = pytest.mark.gpu
BAND = 1e-4


def run_pixels(dctf, op, img, pitch=None, flags=0):
    h, w = img.shape
    x = oracle.dct2_blocks(oracle.image_to_blocks(img, 8)).astype(np.float32)
    xd = torch.from_numpy(x).cuda()
    pitch = pitch or w
    out = torch.full((h, pitch), 77, dtype=torch.uint8, device="cuda")
    op.set_flags(flags)
    dctf.apply_pixels(op, xd, h, w, out, pitch)
    torch.cuda.synchronize()
    op.set_flags(0)
    return out.cpu().numpy(), x


def check_image(u8, img, w, a, boundary):
    h, wd = img.shape
    blocks = oracle.image_to_blocks(img, 8)
    p_ref = oracle.spatial_filter_blocks(blocks, w, a, boundary)
    got = oracle.image_to_blocks(u8[:, :wd], 8)
    st = oracle.uint8_compare(p_ref, got, BAND)
    assert st["mismatch"] == 0, st
    return st


CASES = [   # (height, width, mask, anchor, boundary)
    (8, 8, "gauss3", (1, 1), 0),
    (136, 264, "headline", (1, 3), 1),
    (512, 520, "magic", (1, 1), 1),
    (1024, 1024, "headline", (1, 3), 1),
    (720, 1288, "laplacian", (1, 1), 0),
    (64, 8000, "gauss7", (3, 3), 1),
]


def mask_of(name):
    return {"gauss3": datagen.gaussian_mask(3, 1.0), "headline": datagen.headline_mask(),
            "magic": datagen.magic_square_3(), "laplacian": datagen.laplacian_sharpen(),
            "gauss7": datagen.gaussian_mask(7, 2.0)}[name]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_pixels_match_spatial_filter(dctf, case):
    h, wd, name, a, bnd = CASES[case]
    img = datagen.synthetic_image(h, wd, datagen.rng(97, case, 0))
    w = mask_of(name)
    op = dctf.build_operator(w, a, 8, bnd)
    u8, _ = run_pixels(dctf, op, img)
    check_image(u8, img, w, a, bnd)
    assert op.status() == 0
    op.release()


def test_pitch_padding_untouched_and_inputs_ready(dctf):
    img = datagen.synthetic_image(264, 136, datagen.rng(97, 100, 0))
    w, a = datagen.headline_mask(), (1, 3)
    op = dctf.build_operator(w, a, 8, dctf.REPLICATE)
    u8, _ = run_pixels(dctf, op, img, pitch=200)
    check_image(u8, img, w, a, oracle.REPLICATE)
    assert (u8[:, 136:] == 77).all()
    u8b, _ = run_pixels(dctf, op, img, pitch=200, flags=dctf.APPLY_INPUTS_READY)
    assert np.array_equal(u8, u8b)
    op.release()


@pytest.mark.parametrize("hw", [(1024, 1024), (2048, 1536)])
def test_pixels_one_cta_per_sm_under_inputs_ready(dctf, hw):
    """With DCTF_APPLY_INPUTS_READY an image of up to 2,048 half tiles goes
    out with one CTA an SM (two otherwise): the same pixels either way, and
    the oracle's."""
    h, wd = hw
    img = datagen.synthetic_image(h, wd, datagen.rng(97, 102, h))
    w, a = datagen.headline_mask(), (1, 3)
    op = dctf.build_operator(w, a, 8, dctf.REPLICATE)
    u8, _ = run_pixels(dctf, op, img)
    u8b, _ = run_pixels(dctf, op, img, flags=dctf.APPLY_INPUTS_READY)
    assert np.array_equal(u8, u8b)
    check_image(u8b, img, w, a, oracle.REPLICATE)
    assert op.status() == 0
    op.release()


def test_pixels_agree_with_coefficient_route(dctf):
    """The fused kernel and dctf_apply followed by the inverse DCT give the
    same uint8 image outside the tie band (two device routes, one result)."""
    img = datagen.synthetic_image(512, 768, datagen.rng(97, 101, 0))
    w, a = datagen.headline_mask(), (1, 3)
    op = dctf.build_operator(w, a, 8, dctf.REPLICATE)
    u8, x = run_pixels(dctf, op, img)
    xd = torch.from_numpy(x).cuda()
    y = torch.empty_like(xd)
    dctf.apply(op, xd, x.shape[0], y)
    u8c = torch.empty((512, 768), dtype=torch.uint8, device="cuda")
    dctf.inverse_dct_u8(y, 512, 768, 8, u8c)
    torch.cuda.synchronize()
    p_ref = oracle.spatial_filter_blocks(oracle.image_to_blocks(img, 8), w, a, oracle.REPLICATE)
    inband = np.abs(np.abs(p_ref - np.floor(p_ref)) - 0.5) < BAND
    diff = oracle.image_to_blocks(u8, 8) != oracle.image_to_blocks(u8c.cpu().numpy(), 8)
    assert not (diff & ~inband).any()
    op.release()


def test_pixels_argument_checks(dctf):
    op8 = dctf.build_operator(datagen.gaussian_mask(3, 1.0), (1, 1), 8, dctf.ZERO)
    x = torch.zeros((4, 64), device="cuda")
    img = torch.zeros((16, 24), dtype=torch.uint8, device="cuda")
    with pytest.raises(dctf.DctfError):
        dctf.apply_pixels(op8, x, 16, 20, img, 24)          # width not a multiple of 8
    with pytest.raises(dctf.DctfError):
        dctf.apply_pixels(op8, x, 16, 16, img, 12)          # pitch < width
    with pytest.raises(dctf.DctfError):
        dctf.apply_pixels(op8, x, 16, 16, x, 64)            # image overlaps the coefficients
    op16 = dctf.build_operator(datagen.gaussian_mask(3, 1.0), (1, 1), 16, dctf.ZERO)
    with pytest.raises(dctf.DctfError) as e:
        dctf.apply_pixels(op16, x, 16, 16, img, 24)
    assert e.value.status == 6
    op8.release()
    op16.release()


def test_grouped_pixels_match_single_launches_and_oracle(dctf):
    """Many images, each with its own operator, to uint8 in one persistent
    launch: every image equals its own dctf_apply_pixels launch bit for bit
    (same arithmetic) and the oracle's spatial filter outside the tie band;
    pitch padding stays untouched; tuning and CUDA-graph replay give the
    same images."""
    jobs = datagen.grouped_jobs(count=16, scale=0.2)
    items = []
    for i, job in enumerate(jobs):
        h, w = job.image.shape
        x = oracle.dct2_blocks(oracle.image_to_blocks(job.image, 8)).astype(np.float32)
        pitch = w + 8 * (i % 3)
        img = torch.full((h, pitch), 77, dtype=torch.uint8, device="cuda")
        op = dctf.build_operator(job.mask, job.anchor, 8, job.boundary)
        items.append((op, torch.from_numpy(x).cuda(), h, w, img, pitch))
    g = dctf.group_create_pixels(items)
    g.launch()
    torch.cuda.synchronize()
    assert g.status() == 0
    singles = []
    for (op, xd, h, w, img, pitch), job in zip(items, jobs):
        u8 = img.cpu().numpy()
        assert (u8[:, w:] == 77).all()
        check_image(u8, job.image, job.mask, job.anchor, job.boundary)
        one = torch.full_like(img, 77)
        dctf.apply_pixels(op, xd, h, w, one, pitch)
        torch.cuda.synchronize()
        assert torch.equal(one, img)
        singles.append(one)
    g.tune(reps=2)
    for it in items:
        it[4].fill_(0)
    s = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s, capture_error_mode="thread_local"):
        g.launch(stream=s)
    graph.replay()
    torch.cuda.synchronize()
    for it, one in zip(items, singles):
        assert torch.equal(it[4][:, :it[3]], one[:, :it[3]])
    g.destroy()
    for it in items:
        it[0].release()


def test_grouped_pixels_reject_bad_items(dctf):
    op = dctf.build_operator(datagen.gaussian_mask(3, 1.0), (1, 1), 8, dctf.ZERO)
    op16 = dctf.build_operator(datagen.gaussian_mask(3, 1.0), (1, 1), 16, dctf.ZERO)
    x = torch.zeros((16, 64), device="cuda")
    img = torch.zeros((32, 32), dtype=torch.uint8, device="cuda")
    with pytest.raises(dctf.DctfError) as e:
        dctf.group_create_pixels([(op16, x, 32, 32, img)])
    assert e.value.status == 6                              # EUNSUPPORTED
    for bad in ([(op, x, 32, 30, img)],                      # width not a multiple of 8
                [(op, x, 32, 32, img, 24)],                  # pitch < width
                [(op, x, 0, 32, img)],                       # empty image
                [(op, x[:, 1:], 32, 32, img)]):              # misaligned coefficients
        with pytest.raises(dctf.DctfError) as e:
            dctf.group_create_pixels(bad)
        assert e.value.status == 1                          # EINVAL
    op.release()
    op16.release()
