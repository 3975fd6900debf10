"""GPU: the persistent grouped apply (many images, each with its own operator,
one launch) against the oracle, and against one dctf_apply per image.

Same bars as tests/test_gpu_apply.py: coefficients within 1e-3 of the FP64
oracle, uint8 pixels equal outside the 1e-4 tie band; int16 requantised
outputs equal outside the same band (in units of y / q)."""
import numpy as np
import pytest
import torch

import datagen
import oracle

pytestmark = pytest.mark.gpu

COEF_TOL = 1e-3
BAND = 1e-4


def make_items(dctf, jobs):
    items, refs = [], []
    for job in jobs:
        blocks = oracle.image_to_blocks(job.image, 8)
        x = oracle.dct2_blocks(blocks).astype(np.float32)
        xd = torch.from_numpy(x).cuda()
        yd = torch.full_like(xd, float("nan"))
        op = dctf.build_operator(job.mask, job.anchor, 8, job.boundary)
        items.append((op, xd, yd, x.shape[0]))
        refs.append((job, blocks, x))
    return items, refs


def check_item(y, job, blocks, x):
    y_ref = oracle.apply_M(oracle.build_M(job.mask, job.anchor, 8, job.boundary),
                           x.astype(np.float64))
    assert np.abs(y - y_ref).max() <= COEF_TOL
    p_sp = oracle.spatial_filter_blocks(blocks, job.mask, job.anchor, job.boundary)
    st = oracle.uint8_compare(p_sp, oracle.to_uint8(oracle.idct2_blocks(y, 8)), BAND)
    assert st["mismatch"] == 0, st


@pytest.fixture(scope="module")
def small_batch():
    return datagen.grouped_jobs(count=16, scale=0.2)


def test_group_matches_oracle_and_single_applies(dctf, small_batch):
    items, refs = make_items(dctf, small_batch)
    g = dctf.group_create(items)
    g.launch()
    torch.cuda.synchronize()
    assert g.status() == 0
    for (op, xd, yd, nb), (job, blocks, x) in zip(items, refs):
        y = yd.cpu().numpy().astype(np.float64)
        check_item(y, job, blocks, x)
        # one plain launch per image gives the same bits
        y1 = torch.empty_like(xd)
        dctf.apply(op, xd, nb, y1)
        torch.cuda.synchronize()
        assert np.array_equal(y1.cpu().numpy(), yd.cpu().numpy())


def test_group_graph_replay_and_tune(dctf, small_batch):
    items, refs = make_items(dctf, small_batch)
    g = dctf.group_create(items)
    g.tune(reps=2)
    # the tuner's last candidate ran half the CTAs with 64-row tiles
    torch.cuda.synchronize()
    for (_, _, yd, _), (job, blocks, x) in zip(items, refs):
        check_item(yd.cpu().numpy().astype(np.float64), job, blocks, x)
    grid, rows, stages, slots = g.config()
    assert grid >= 1 and rows in (64, 128) and (stages, slots) in ((3, 2), (2, 2), (4, 1))
    for _, _, yd, _ in items:
        yd.fill_(float("nan"))
    s = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(graph, stream=s):
            g.launch(stream=s)
    graph.replay()
    torch.cuda.synchronize()
    for (_, _, yd, _), (job, blocks, x) in zip(items, refs):
        check_item(yd.cpu().numpy().astype(np.float64), job, blocks, x)
    assert g.status() == 0


def test_group_edge_items(dctf):
    """Empty items, a 1-block item, a ragged item, an in-place item, and the
    64-row tile mode."""
    img = datagen.synthetic_image(512, 264, datagen.rng(97, 0, 0))   # 2112 blocks
    blocks = oracle.image_to_blocks(img, 8)
    x = oracle.dct2_blocks(blocks).astype(np.float32)
    w, a = datagen.headline_mask(), (1, 3)
    op = dctf.build_operator(w, a, 8, dctf.REPLICATE)
    y_ref = oracle.apply_M(oracle.build_M(w, a, 8, oracle.REPLICATE), x.astype(np.float64))
    sizes = [0, 1, 63, 65, 128, 0, 1000, 129]
    items, views = [], []
    off = 0
    xin = torch.from_numpy(x).cuda()
    for nb in sizes:
        xi = xin[off:off + nb].clone() if nb else xin[:1].clone()
        yi = torch.full_like(xi, float("nan"))
        items.append((op, xi, yi, nb))
        views.append((off, nb, yi))
        off += nb
    # in place: the last item writes over its own input
    xi = xin[:300].clone()
    items.append((op, xi, xi, 300))
    views.append((0, 300, xi))
    g = dctf.group_create(items)
    g.launch()
    torch.cuda.synchronize()
    for o, nb, yi in views:
        if nb:
            assert np.abs(yi.cpu().numpy().astype(np.float64) - y_ref[o:o + nb]).max() <= COEF_TOL
    assert g.status() == 0
    with pytest.raises(dctf.DctfError):
        g.tune()                   # an in-place item: refused


def test_group_rejects_bad_items(dctf):
    op8 = dctf.build_operator(datagen.gaussian_mask(3, 1.0), (1, 1), 8, dctf.ZERO)
    op16 = dctf.build_operator(datagen.gaussian_mask(3, 1.0), (1, 1), 16, dctf.ZERO)
    buf = torch.zeros(64 * 10 + 4, device="cuda")
    with pytest.raises(dctf.DctfError):
        dctf.group_create([(op16, buf, buf, 2)])
    with pytest.raises(dctf.DctfError):
        dctf.group_create([(op8, buf.data_ptr() + 4, buf.data_ptr() + 4, 2)])
    with pytest.raises(dctf.DctfError):
        dctf.group_create([(op8, buf, buf.data_ptr() + 256, 2)])
    with pytest.raises(dctf.DctfError):
        dctf.group_create([(op8, buf, buf, 2)], io=dctf.IO_I16)     # no q tables


def quantised_plane(img, s):
    q = datagen.quant_table(s)
    x = oracle.dct2_blocks(oracle.image_to_blocks(img, 8))
    qin = np.clip(oracle.round_half_away(x / q.ravel()[None, :].astype(np.float64)),
                  -32768, 32767).astype(np.int16)
    return qin, q


def test_group_int16_dequant_requant(dctf):
    """JPEG-style int16 planes, each with its own mask, input table and a
    different output table: dequantise with q_in, filter, requantise with
    q_out in one pass (swapping the tables changes the result)."""
    planes = []
    for j in range(6):
        img = datagen.synthetic_image(128 + 64 * (j % 3), 192, datagen.rng(98, j, 0))
        s = [1, 2, 4][j % 3]
        w, a, bnd = datagen.serving_mask(j)
        planes.append((img, s, w, a, bnd))
    items, refs, keep = [], [], []
    for j, (img, s, w, a, bnd) in enumerate(planes):
        qin, q = quantised_plane(img, s)
        op = dctf.build_operator(w, a, 8, bnd)
        xd = torch.from_numpy(qin).cuda()
        yd = torch.zeros_like(xd)
        qo = datagen.quant_table([4, 1, 2][j % 3])       # another scale than q's
        qd = torch.from_numpy(q.ravel().astype(np.int16).view(np.int16)).cuda()
        qod = torch.from_numpy(qo.ravel().astype(np.int16).view(np.int16)).cuda()
        keep += [qd, qod]
        items.append((op, xd, yd, qin.shape[0], qd, qod))
        refs.append((qin, q, qo, w, a, bnd))
    g = dctf.group_create(items, io=dctf.IO_I16)
    g.launch()
    torch.cuda.synchronize()
    assert g.status() == 0
    for (op, xd, yd, nb, _, _), (qin, q, qo, w, a, bnd) in zip(items, refs):
        m = oracle.build_M(w, a, 8, bnd)
        _, v = oracle.serve_blocks(qin, q, m, qo)
        got = yd.cpu().numpy()
        st = oracle.int16_compare(v, got, BAND)
        assert st["mismatch"] == 0, st
        # the tables are not interchangeable: the swapped order disagrees
        _, v_swapped = oracle.serve_blocks(qin, qo, m, q)
        assert oracle.int16_compare(v_swapped, got, BAND)["mismatch"] > 0


def test_group_layouts_same_bits(dctf, small_batch):
    """Every shared-memory layout the tuner chooses from (input stages x
    operator slots), with either tile height, gives the same bits as the
    default launch, for FP32 coefficient groups and pixel groups."""
    items, refs = make_items(dctf, small_batch)
    g = dctf.group_create(items)
    g.launch()
    torch.cuda.synchronize()
    want = [yd.cpu().numpy().copy() for _, _, yd, _ in items]
    imgs = [torch.zeros(job.image.shape, dtype=torch.uint8, device="cuda") for job, _, _ in refs]
    gp = dctf.group_create_pixels([(op, xd, job.image.shape[0], job.image.shape[1], im)
                                   for (op, xd, _, _), (job, _, _), im in zip(items, refs, imgs)])
    gp.launch()
    torch.cuda.synchronize()
    want_px = [im.cpu().numpy().copy() for im in imgs]
    for grp, layouts, outs, ref in ((g, ((3, 2), (2, 2), (4, 1)), [it[2] for it in items], want),
                                    (gp, ((4, 2), (5, 2), (6, 1)), imgs, want_px)):
        for stages, slots in layouts:
            for rows in (128, 64):
                grp.set_config(57, rows, stages, slots)
                assert grp.config() == (57, rows, stages, slots)
                for o in outs:
                    o.zero_()
                grp.launch()
                torch.cuda.synchronize()
                for o, w in zip(outs, ref):
                    assert np.array_equal(o.cpu().numpy(), w)
        with pytest.raises(dctf.DctfError) as e:
            grp.set_config(0, 128, 7, 2)
        assert e.value.status == 6
        assert grp.status() == 0
    g.destroy()
    gp.destroy()


def test_group_int16_layouts_same_bits(dctf):
    img = datagen.synthetic_image(256, 320, datagen.rng(98, 77, 0))
    qin, q = quantised_plane(img, 2)
    w, a, bnd = datagen.serving_mask(5)
    op = dctf.build_operator(w, a, 8, bnd)
    xd = torch.from_numpy(qin).cuda()
    qd = torch.from_numpy(q.ravel().astype(np.int16)).cuda()
    outs = [torch.zeros_like(xd) for _ in range(3)]
    g = dctf.group_create([(op, xd, o, qin.shape[0] // (k + 1), qd, qd) for k, o in enumerate(outs)],
                          io=dctf.IO_I16)
    res = []
    for stages, slots in ((4, 2), (6, 2), (8, 1)):
        g.set_config(0, 128, stages, slots)
        for o in outs:
            o.zero_()
        g.launch()
        torch.cuda.synchronize()
        res.append([o.cpu().numpy().copy() for o in outs])
    for r in res[1:]:
        for a_, b_ in zip(res[0], r):
            assert np.array_equal(a_, b_)
    _, v = oracle.serve_blocks(qin, q, oracle.build_M(w, a, 8, bnd), q)
    assert oracle.int16_compare(v, res[0][0], BAND)["mismatch"] == 0
    g.destroy()


_TUNE_CHILD = """
import sys, json
sys.path.insert(0, sys.argv[1])
import numpy as np, torch
import datagen, oracle
import paper_1710_07193_gb300 as dctf
dctf.load()
jobs = datagen.grouped_jobs(count=6, scale=0.2)
items = []
for j in jobs:
    x = oracle.dct2_blocks(oracle.image_to_blocks(j.image, 8)).astype(np.float32)
    xd = torch.from_numpy(x).cuda()
    items.append((dctf.build_operator(j.mask, j.anchor, 8, j.boundary), xd, torch.empty_like(xd),
                  x.shape[0]))
g = dctf.group_create(items)
if sys.argv[2] == "tune":
    g.tune(reps=2)
print(json.dumps(list(g.config())))
"""


def test_tune_cache_persists_across_processes(dctf, tmp_path):
    """DCTF_TUNE_CACHE: a tuning is written to the file, and a new process
    creating a group of the same size class starts from that choice."""
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, DCTF_TUNE_CACHE=str(tmp_path / "tune.txt"))
    run = lambda mode: json.loads(subprocess.run(
        [sys.executable, "-c", _TUNE_CHILD, root, mode], env=env, capture_output=True, text=True,
        timeout=300, check=True).stdout.strip().splitlines()[-1])
    tuned = run("tune")
    lines = (tmp_path / "tune.txt").read_text().split("\n")
    assert any(len(ln.split()) == 7 for ln in lines)
    assert run("none") == tuned


def test_group_inputs_ready_flag_same_bits(dctf, small_batch):
    """DCTF_APPLY_INPUTS_READY on a group (programmatic serialisation):
    several launches back to back, directly and in a graph, give the bits of
    an ordinary launch; unknown flags are refused."""
    items, refs = make_items(dctf, small_batch)
    g = dctf.group_create(items)
    g.launch()
    torch.cuda.synchronize()
    plain = [yd.clone() for _, _, yd, _ in items]
    g.set_flags(dctf.APPLY_INPUTS_READY)
    for _, _, yd, _ in items:
        yd.fill_(float("nan"))
    for _ in range(4):
        g.launch()
    torch.cuda.synchronize()
    for (_, _, yd, _), p in zip(items, plain):
        assert torch.equal(yd, p)
    s = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(graph, stream=s):
            for _ in range(3):
                g.launch(stream=s)
    for _, _, yd, _ in items:
        yd.fill_(float("nan"))
    graph.replay()
    graph.replay()
    torch.cuda.synchronize()
    for (_, _, yd, _), p in zip(items, plain):
        assert torch.equal(yd, p)
    assert g.status() == 0
    with pytest.raises(dctf.DctfError):
        g.set_flags(2)
    g.destroy()
