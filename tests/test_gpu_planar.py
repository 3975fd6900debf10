"""GPU: the image-plane coefficient layout (dctf_apply_planar).

Coefficient (u, v) of block (by, bx) sits at row 8 by + u, column 8 bx + v of
an image-shaped FP32 plane.  The result must equal, element for element, the
block-major dctf_apply on the same coefficients (same arithmetic, same
order), and stay within 1e-3 of the FP64 oracle; pitch padding and the
pixels outside the plane are never written.
"""
import numpy as np
import pytest
import torch

import datagen
import oracle

pytestmark = pytest.mark.gpu
COEF_TOL = 1e-3


def planes(img):
    h, w = img.shape
    xb = oracle.dct2_blocks(oracle.image_to_blocks(img, 8)).astype(np.float32)
    plane = oracle.blocks_to_image(xb.reshape(-1, 8, 8), h, w).astype(np.float32)
    return xb, plane


SIZES = [(8, 8), (64, 1024), (136, 264), (512, 1032), (1088, 1920), (40, 2056)]


@pytest.mark.parametrize("size", SIZES)
def test_planar_matches_block_major_and_oracle(dctf, size):
    h, w = size
    img = datagen.synthetic_image(h, w, datagen.rng(99, h, w))
    xb, plane = planes(img)
    m, a = datagen.headline_mask(), (1, 3)
    op = dctf.build_operator(m, a, 8, dctf.REPLICATE)
    pd = torch.from_numpy(plane).cuda()
    out = torch.empty_like(pd)
    dctf.apply_planar(op, pd, h, w, out)
    xd = torch.from_numpy(xb).cuda()
    yb = torch.empty_like(xd)
    dctf.apply(op, xd, xb.shape[0], yb)
    torch.cuda.synchronize()
    got = oracle.image_to_blocks(out.cpu().numpy(), 8).reshape(-1, 64)
    assert np.array_equal(got, yb.cpu().numpy().astype(np.float64))
    y_ref = oracle.apply_M(oracle.build_M(m, a, 8, oracle.REPLICATE), xb.astype(np.float64))
    assert np.abs(got - y_ref).max() <= COEF_TOL
    assert op.status() == 0
    op.release()


def test_planar_pitch_and_in_place(dctf):
    h, w, pitch = 136, 264, 300
    img = datagen.synthetic_image(h, w, datagen.rng(99, 1, 1))
    _, plane = planes(img)
    m, a = datagen.gaussian_mask(7, 2.0), (3, 3)
    op = dctf.build_operator(m, a, 8, dctf.ZERO)
    buf = torch.full((h, pitch), -7.0, device="cuda")
    buf[:, :w] = torch.from_numpy(plane).cuda()
    out = torch.full((h, pitch), 5.0, device="cuda")
    dctf.apply_planar(op, buf, h, w, out, pitch=pitch, out_pitch=pitch)
    torch.cuda.synchronize()
    o = out.cpu().numpy()
    assert (o[:, w:] == 5.0).all()
    dctf.apply_planar(op, buf, h, w, buf, pitch=pitch, out_pitch=pitch)     # in place
    torch.cuda.synchronize()
    b = buf.cpu().numpy()
    assert np.array_equal(b[:, :w], o[:, :w]) and (b[:, w:] == -7.0).all()
    op.release()


def test_planar_argument_checks(dctf):
    op = dctf.build_operator(datagen.gaussian_mask(3, 1.0), (1, 1), 8, dctf.ZERO)
    p = torch.zeros((16, 32), device="cuda")
    with pytest.raises(dctf.DctfError):
        dctf.apply_planar(op, p, 16, 20, p)                      # width not a multiple of 8
    with pytest.raises(dctf.DctfError):
        dctf.apply_planar(op, p, 16, 32, p, pitch=34, out_pitch=34)   # pitch not a multiple of 4
    with pytest.raises(dctf.DctfError):
        dctf.apply_planar(op, p, 8, 32, p[4:], pitch=32, out_pitch=32)  # partial overlap
    op16 = dctf.build_operator(datagen.gaussian_mask(3, 1.0), (1, 1), 16, dctf.ZERO)
    with pytest.raises(dctf.DctfError) as e:
        dctf.apply_planar(op16, p, 16, 32, torch.zeros_like(p))
    assert e.value.status == 6
    op.release()
    op16.release()
