"""GPU: the full-size workloads in the launch configurations the benchmark
times, checked against the oracle on EVERY block (the oracle's apply and its
spatial filter are vectorised FP64 passes) and by properties that hold at
any size.

* the grouped workload: 64 images of seeded sizes (~870k blocks), each with
  its own operator, in one persistent launch after autotuning;
* 8192 x 8192 with 16 x 16 blocks (262,144 blocks), every arithmetic;
* 4096 x 4096 with 8 x 8 blocks: the fused pixel output and the
  image-plane layout.

Bars as everywhere: coefficients within 1e-3 of the FP64 oracle (the
variants that are not exact by construction within the bound their
arithmetic gives), uint8 pixels equal to the oracle's spatial filter
outside the 1e-4 tie band.
"""
import numpy as np
import pytest
import torch

import datagen
import oracle
from tests.test_gpu_apply import bf16x3_bound, tf32x1_bound

pytestmark = pytest.mark.gpu
COEF_TOL = 1e-3
BAND = 1e-4


def _pinned_sample(nb):
    return np.unique(np.linspace(0, nb - 1, 257).astype(int))


def dct_full(blocks):
    """C X C^T for every block as two FP64 GEMMs (the oracle's einsum is
    too slow for 262,144 16 x 16 blocks); pinned to oracle.dct2_blocks on a
    sample before use."""
    nb, n, _ = blocks.shape
    c = oracle.dct_matrix(n)
    t = (blocks.reshape(-1, n) @ c.T).reshape(nb, n, n)              # X C^T
    out = (t.transpose(0, 2, 1).reshape(-1, n) @ c.T).reshape(nb, n, n).transpose(0, 2, 1)
    x = np.ascontiguousarray(out).reshape(nb, n * n)
    idx = _pinned_sample(nb)
    assert np.abs(x[idx] - oracle.dct2_blocks(blocks[idx])).max() < 1e-9
    return x


def idct_full(y, n):
    """C^T Y C for every block as two FP64 GEMMs; pinned to
    oracle.idct2_blocks on a sample before use.  [nb, n, n]."""
    y = np.asarray(y, dtype=np.float64).reshape(-1, n, n)
    nb = y.shape[0]
    c = oracle.dct_matrix(n)
    t = (y.reshape(-1, n) @ c).reshape(nb, n, n)                     # Y C
    out = (t.transpose(0, 2, 1).reshape(-1, n) @ c).reshape(nb, n, n).transpose(0, 2, 1)
    out = np.ascontiguousarray(out)
    idx = _pinned_sample(nb)
    assert np.abs(out[idx] - oracle.idct2_blocks(y[idx].reshape(-1, n * n), n)).max() < 1e-9
    return out


def check_all(y, x32, p_sp, m, n, bound=None):
    """Every block: coefficients against the oracle's y = M x in FP64, and
    (exact arithmetics) uint8 pixels against the oracle's spatial filter."""
    y_ref = oracle.apply_M(m, x32.astype(np.float64))
    err = np.abs(y - y_ref)
    if bound is None:
        assert err.max() <= COEF_TOL, err.max()
        st = oracle.uint8_compare(p_sp, oracle.to_uint8(idct_full(y, n)), BAND)
        assert st["mismatch"] == 0, st
    else:
        assert (err <= bound(m, x32.astype(np.float64))).all()
    return err.max()


@pytest.fixture(scope="module")
def grouped_full():
    jobs = datagen.grouped_jobs(64)
    data = []
    for job in jobs:
        blocks = oracle.image_to_blocks(job.image, 8)
        p_sp = oracle.spatial_filter_blocks(blocks, job.mask, job.anchor, job.boundary)
        data.append((job, p_sp, dct_full(blocks).astype(np.float32)))
    return data


def test_grouped_full_workload(dctf, grouped_full):
    items = []
    for job, _, x in grouped_full:
        xd = torch.from_numpy(x).cuda()
        yd = torch.full_like(xd, float("nan"))
        items.append((dctf.build_operator(job.mask, job.anchor, 8, job.boundary), xd, yd, x.shape[0]))
    assert sum(it[3] for it in items) > 500_000
    g = dctf.group_create(items)
    g.tune(reps=3)
    g.launch()
    torch.cuda.synchronize()
    assert g.status() == 0
    for (op, xd, yd, nb), (job, p_sp, x) in zip(items, grouped_full):
        y = yd.cpu().numpy()
        assert np.isfinite(y).all()                        # every block written
        check_all(y.astype(np.float64), x, p_sp, oracle.build_M(job.mask, job.anchor, 8,
                                                                  job.boundary), 8)
        y1 = torch.empty_like(xd)
        dctf.apply(op, xd, nb, y1)                         # one plain launch: the same bits
        torch.cuda.synchronize()
        assert np.array_equal(y1.cpu().numpy(), y)
    g.destroy()
    for it in items:
        it[0].release()


@pytest.fixture(scope="module")
def large_full():
    job = datagen.large_job()
    blocks = oracle.image_to_blocks(job.image, 16)
    x = dct_full(blocks).astype(np.float32)
    p_sp = oracle.spatial_filter_blocks(blocks, job.mask, job.anchor, job.boundary)
    return job, p_sp, x, oracle.build_M(job.mask, job.anchor, 16, job.boundary)


@pytest.mark.parametrize("prec", ["F16X3", "BF16X6", "TF32X3", "FP32_SIMT", "BF16X3", "TF32X1",
                                  "KRON_FP32", "KRON_F16X3"])
def test_large_16x16_full_workload(dctf, large_full, prec):
    job, p_sp, x, m = large_full
    nb = x.shape[0]
    assert nb == 262144
    op = dctf.build_operator(job.mask, job.anchor, 16, job.boundary, kron=prec.startswith("KRON"))
    op.set_precision(getattr(dctf, prec))
    xd = torch.from_numpy(x).cuda()
    yd = torch.full_like(xd, float("nan"))
    dctf.apply(op, xd, nb, yd)
    torch.cuda.synchronize()
    assert op.status() == 0
    y = yd.cpu().numpy()
    assert np.isfinite(y).all()
    bound = {"BF16X3": bf16x3_bound, "TF32X1": tf32x1_bound}.get(prec)
    check_all(y.astype(np.float64), x, p_sp, m, 16, bound)
    op.release()


@pytest.fixture(scope="module")
def headline_full():
    job = datagen.headline_job()
    blocks = oracle.image_to_blocks(job.image, 8)
    p_sp = oracle.spatial_filter_blocks(blocks, job.mask, job.anchor, job.boundary)
    return job, p_sp, dct_full(blocks).astype(np.float32)


def test_pixels_and_planar_full_workload(dctf, headline_full):
    job, p_sp, x = headline_full
    h, w = job.image.shape
    m = oracle.build_M(job.mask, job.anchor, 8, job.boundary)
    op = dctf.build_operator(job.mask, job.anchor, 8, job.boundary)
    xd = torch.from_numpy(x).cuda()
    # fused pixel output: uint8 of the spatial filter on every block
    img = torch.full((h, w), 77, dtype=torch.uint8, device="cuda")
    dctf.apply_pixels(op, xd, h, w, img)
    torch.cuda.synchronize()
    got = oracle.image_to_blocks(img.cpu().numpy(), 8)
    st = oracle.uint8_compare(p_sp, got, BAND)
    assert st["mismatch"] == 0, st
    # image-plane layout: the same bits as the block-major apply, everywhere
    yb = torch.empty_like(xd)
    dctf.apply(op, xd, x.shape[0], yb)
    plane = torch.from_numpy(oracle.blocks_to_image(x.reshape(-1, 8, 8), h, w).astype(np.float32)).cuda()
    out = torch.empty_like(plane)
    dctf.apply_planar(op, plane, h, w, out)
    torch.cuda.synchronize()
    assert op.status() == 0
    got = oracle.image_to_blocks(out.cpu().numpy(), 8).reshape(-1, 64)
    assert np.array_equal(got, yb.cpu().numpy())
    check_all(got.astype(np.float64), x, p_sp, m, 8)
    op.release()
