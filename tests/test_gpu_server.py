"""GPU: the continuous-batching server (int16 quantised planes).

* each request's result is bit-identical whether it runs alone or in a
  mixed burst (continuous batching must not change results), and equal to
  the oracle's requantised output outside the 1e-4 tie band;
* admission by HBM budget (a request that can never fit is refused),
  operator cache hits / eviction, bounded waits, and an injected operator
  build failure that fails only its own request while the server carries on.
"""
import numpy as np
import pytest
import torch

import datagen
import oracle

pytestmark = pytest.mark.gpu
BAND = 1e-4


def quantised(img, s):
    q = datagen.quant_table(s)
    x = oracle.dct2_blocks(oracle.image_to_blocks(img, 8))
    qin = np.clip(oracle.round_half_away(x / q.ravel()[None, :].astype(np.float64)),
                  -32768, 32767).astype(np.int16)
    return qin, q.ravel()


@pytest.fixture(scope="module")
def requests():
    """A small stream: scaled-down 4:2:0 frames (3 planes) and stills (1 plane)."""
    out = []
    for r in datagen.serving_stream(10, 2000.0, scale=0.15):
        planes = [quantised(img, s) for img, s in zip(r.planes, r.q_scale)]
        w, a, bnd = datagen.serving_mask(r.mask_id)
        out.append((planes, w, a, bnd))
    return out


def run_one(srv, req):
    planes, w, a, bnd = req
    outs = [np.zeros_like(p[0]) for p in planes]
    t = srv.submit([p[0] for p in planes], outs, [p[1] for p in planes], w, a, bnd)
    return t, outs


def test_alone_equals_mixed_and_oracle(dctf, requests):
    srv = dctf.Server(hbm_budget_bytes=512 << 20, max_inflight=2, max_batch_requests=4)
    alone = []
    for req in requests:
        t, outs = run_one(srv, req)
        srv.wait(t)
        alone.append(outs)
    # the burst arrives while the worker stages a 64 MB pageable request
    # (milliseconds of host copying), so it queues and must be batched
    big = np.zeros((1 << 19, 64), dtype=np.int16)
    w0, a0, b0 = requests[0][1:]
    t_big = srv.submit([big], [np.empty_like(big)], [requests[0][0][0][1]], w0, a0, b0)
    burst = [run_one(srv, req) for req in requests]
    srv.wait(t_big)
    for t, _ in burst:
        srv.wait(t)
    for (planes, w, a, bnd), outs_alone, (_, outs_mix) in zip(requests, alone, burst):
        m = oracle.build_M(w, a, 8, bnd)
        for (qin, q), ya, ym in zip(planes, outs_alone, outs_mix):
            assert np.array_equal(ya, ym)
            _, v = oracle.serve_blocks(qin, q, m, q)
            st = oracle.int16_compare(v, ya, BAND)
            assert st["mismatch"] == 0, st
    st = srv.stats()
    assert st["completed"] == 2 * len(requests) + 1 and st["failed"] == 0
    assert st["cache_hits"] > 0 and 0 < st["p50_ms"] <= st["p99_ms"]
    assert st["max_batch_requests_seen"] > 1          # the burst really batched
    assert st["hbm_in_use"] == 0
    srv.close()


def test_budget_cache_and_timeouts(dctf, requests):
    srv = dctf.Server(hbm_budget_bytes=2 << 20, max_inflight=2, max_batch_requests=2,
                      op_cache_capacity=2)
    big = np.zeros((40000, 64), dtype=np.int16)           # 2 x 5 MB > 2 MB budget
    with pytest.raises(dctf.DctfError) as e:
        srv.submit([big], [np.zeros_like(big)], [datagen.quant_table(1)],
                   datagen.gaussian_mask(3, 1.0), (1, 1), 0)
    assert e.value.status == 4                            # EBUDGET
    with pytest.raises(dctf.DctfError):
        srv.wait(123456)                                  # unknown ticket
    # stills only (fit the small budget), more distinct masks than the cache holds
    stills = [r for r in requests if len(r[0]) == 1]
    tickets = []
    for j, (planes, _, _, _) in enumerate(stills * 2):
        w, a, bnd = datagen.serving_mask(j % 5)
        outs = [np.zeros_like(planes[0][0])]
        tickets.append((srv.submit([planes[0][0]], outs, [planes[0][1]], w, a, bnd),
                        outs, planes[0], (w, a, bnd)))
    for t, outs, (qin, q), (w, a, bnd) in tickets:
        try:
            srv.wait(t, 0)                                # may still be running
        except dctf.DctfError as err:
            assert err.status == 5                        # ETIMEOUT: ticket stays valid
            srv.wait(t)
        _, v = oracle.serve_blocks(qin, q, oracle.build_M(w, a, 8, bnd), q)
        assert oracle.int16_compare(v, outs[0], BAND)["mismatch"] == 0
    st = srv.stats()
    assert st["failed"] == 0 and st["cache_misses"] >= 5
    srv.close()


def test_injected_build_failure(dctf, requests):
    srv = dctf.Server(hbm_budget_bytes=64 << 20, max_inflight=2, max_batch_requests=2,
                      op_cache_capacity=1, inject_build_failure_every=2)
    results = []
    for j in range(6):
        planes, _, _, _ = requests[j % len(requests)]
        w, a, bnd = datagen.serving_mask(j)                 # a new operator every time
        outs = [np.zeros_like(p[0]) for p in planes]
        t = srv.submit([p[0] for p in planes], outs, [p[1] for p in planes], w, a, bnd)
        try:
            srv.wait(t)
            results.append("ok")
        except dctf.DctfError as err:
            assert err.status == 3                        # the injected ECUDA
            results.append("fail")
    assert results.count("fail") == 3 and results.count("ok") == 3
    st = srv.stats()
    assert st["failed"] == 3 and st["completed"] == 3
    srv.close()


def staged_result(srv, planes, w, a, bnd):
    """The request on pageable buffers: the staged route."""
    outs = [np.zeros_like(p[0]) for p in planes]
    srv.wait(srv.submit([p[0] for p in planes], outs, [p[1] for p in planes], w, a, bnd))
    return outs


def test_pinned_buffers_take_the_direct_path(dctf, requests):
    """Page-locked caller buffers take the host-direct route (the batch
    kernel reads and writes them over the host link, no HBM staging); the
    results are bit-identical to the staged route, whether the two kinds of
    request share a batch or not."""
    srv = dctf.Server(hbm_budget_bytes=64 << 20, max_inflight=2, max_batch_requests=4)
    keep = []
    for planes, w, a, bnd in requests[:6]:
        pin_in = [torch.from_numpy(p[0]).pin_memory() for p in planes]
        pin_out = [torch.zeros_like(t).pin_memory() for t in pin_in]
        keep += pin_in + pin_out
        t1 = srv.submit([t.numpy() for t in pin_in], [t.numpy() for t in pin_out],
                        [p[1] for p in planes], w, a, bnd)
        outs = [np.zeros_like(p[0]) for p in planes]
        t2 = srv.submit([p[0] for p in planes], outs, [p[1] for p in planes], w, a, bnd)
        srv.wait(t1)
        srv.wait(t2)
        for tp, o in zip(pin_out, outs):
            assert np.array_equal(tp.numpy(), o)
    st = srv.stats()
    assert st["failed"] == 0 and st["direct_requests"] == 6 and st["completed"] == 12
    assert st["hbm_in_use"] == 0
    srv.close()


def test_direct_in_place_overlap_and_budget(dctf, requests):
    """In place (out == in) stays host-direct; a request whose planes'
    buffers overlap otherwise takes the staged route (inputs read before any
    output is written); a host-direct request needs none of the HBM budget."""
    srv = dctf.Server(hbm_budget_bytes=1 << 20, max_inflight=2, max_batch_requests=4)
    ref = dctf.Server(hbm_budget_bytes=64 << 20, max_inflight=1, max_batch_requests=1)
    planes, w, a, bnd = next(r for r in requests if len(r[0]) == 3)
    want = staged_result(ref, planes, w, a, bnd)
    buf = [torch.from_numpy(p[0].copy()).pin_memory() for p in planes]
    srv.wait(srv.submit([b.numpy() for b in buf], [b.numpy() for b in buf],
                        [p[1] for p in planes], w, a, bnd))
    for b, o in zip(buf, want):
        assert np.array_equal(b.numpy(), o)
    assert srv.stats()["direct_requests"] == 1
    # planes 1 and 2 (same size): plane 2's output is plane 1's input buffer
    p1 = torch.from_numpy(planes[1][0].copy()).pin_memory()
    p2 = torch.from_numpy(planes[2][0].copy()).pin_memory()
    o1 = torch.zeros_like(p1).pin_memory()
    srv.wait(srv.submit([p1.numpy(), p2.numpy()], [o1.numpy(), p1.numpy()],
                        [planes[1][1], planes[2][1]], w, a, bnd))
    assert np.array_equal(o1.numpy(), want[1]) and np.array_equal(p1.numpy(), want[2])
    assert srv.stats()["direct_requests"] == 1                # staged
    # 2.5 MiB of int16 planes in and out against a 1 MiB budget
    g = np.random.default_rng(5)
    x = g.integers(-300, 300, (20480, 64)).astype(np.int16)
    q = planes[0][1]
    big = [(x, q)]
    want_big = staged_result(ref, big, w, a, bnd)
    hin = torch.from_numpy(x).pin_memory()
    hout = torch.zeros_like(hin).pin_memory()
    srv.wait(srv.submit([hin.numpy()], [hout.numpy()], [q], w, a, bnd))
    assert np.array_equal(hout.numpy(), want_big[0])
    with pytest.raises(dctf.DctfError):
        srv.submit([x], [np.zeros_like(x)], [q], w, a, bnd)     # staged: over the budget
    st = srv.stats()
    assert st["failed"] == 0 and st["direct_requests"] == 2 and st["hbm_in_use"] == 0
    srv.close()
    ref.close()


def test_distinct_output_table_both_routes(dctf, requests):
    """Each plane requantised with its own output table (q_out != q): the
    host-direct and the staged route give the same bits, equal to the
    oracle's dequantise-with-q, requantise-with-q_out result."""
    srv = dctf.Server(hbm_budget_bytes=64 << 20, max_inflight=2, max_batch_requests=4)
    for j, (planes, w, a, bnd) in enumerate(requests[:4]):
        qouts = [datagen.quant_table([4, 1, 2][(j + p) % 3]).ravel() for p in range(len(planes))]
        pin_in = [torch.from_numpy(p[0]).pin_memory() for p in planes]
        pin_out = [torch.zeros_like(t).pin_memory() for t in pin_in]
        outs = [np.zeros_like(p[0]) for p in planes]
        t1 = srv.submit([t.numpy() for t in pin_in], [t.numpy() for t in pin_out],
                        [p[1] for p in planes], w, a, bnd, qtabs_out=qouts)
        t2 = srv.submit([p[0] for p in planes], outs, [p[1] for p in planes], w, a, bnd,
                        qtabs_out=qouts)
        srv.wait(t1)
        srv.wait(t2)
        m = oracle.build_M(w, a, 8, bnd)
        for (qin, q), qo, tp, o in zip(planes, qouts, pin_out, outs):
            assert np.array_equal(tp.numpy(), o)
            _, v = oracle.serve_blocks(qin, q, m, qo)
            assert oracle.int16_compare(v, o, BAND)["mismatch"] == 0
            if not np.array_equal(q, qo):
                _, vs = oracle.serve_blocks(qin, qo, m, q)
                assert oracle.int16_compare(vs, o, BAND)["mismatch"] > 0
    st = srv.stats()
    assert st["failed"] == 0 and st["direct_requests"] == 4
    srv.close()


def test_admission_waits_for_budget(dctf):
    """A staged_only server with a 1 MiB HBM budget: each request needs
    0.77 MiB (in + out), so only one fits at a time and the others are
    admitted as earlier ones complete.  Every result is correct, the server
    counts the waits, and the budget is never exceeded."""
    budget = 1 << 20
    srv = dctf.Server(hbm_budget_bytes=budget, max_inflight=4, max_batch_requests=4,
                      staged_only=True)
    w, a, bnd = datagen.serving_mask(3)
    m = oracle.build_M(w, a, 8, bnd)
    qo = datagen.quant_table(1).ravel()
    reqs = []
    for k in range(5):
        # a 384 x 512 image's quantised coefficients: 3072 blocks, 384 KiB
        img = datagen.synthetic_image(384, 512, datagen.rng(97, k, 0))
        x, q = quantised(img, 2)
        xin = torch.from_numpy(x).pin_memory()                      # page-locked, yet staged
        xout = torch.zeros_like(xin).pin_memory()
        reqs.append((x, xin, xout))
    tickets = [srv.submit([xin.numpy()], [xout.numpy()], [q], w, a, bnd, qtabs_out=[qo])
               for _, xin, xout in reqs]
    for t in tickets:
        srv.wait(t)
    for x, _, xout in reqs:
        _, v = oracle.serve_blocks(x, q, m, qo)
        assert oracle.int16_compare(v, xout.numpy(), BAND)["mismatch"] == 0
    st = srv.stats()
    assert st["failed"] == 0 and st["completed"] == 5 and st["direct_requests"] == 0
    assert st["budget_waits"] >= 1
    assert 0 < st["hbm_peak"] <= budget and st["hbm_in_use"] == 0
    srv.close()


def test_reset_stats_starts_a_new_window(dctf):
    """dctf_server_reset_stats clears the latencies and counters but keeps
    the operator cache: the same mask after a reset is a cache hit, and the
    new window counts only the requests that complete in it."""
    srv = dctf.Server(hbm_budget_bytes=64 << 20, max_inflight=2, max_batch_requests=4)
    w, a, bnd = datagen.serving_mask(5)
    img = datagen.synthetic_image(256, 256, datagen.rng(97, 9, 0))
    x, q = quantised(img, 1)
    outs = [np.zeros_like(x) for _ in range(3)]
    srv.wait(srv.submit([x], [outs[0]], [q], w, a, bnd))
    st = srv.stats()
    assert st["completed"] == 1 and st["cache_misses"] == 1
    srv.reset_stats()
    st = srv.stats()
    assert st["completed"] == 0 and st["cache_misses"] == 0 and st["cache_hits"] == 0
    assert st["p99_ms"] == 0 and st["batches"] == 0 and st["budget_waits"] == 0
    for o in outs[1:]:
        srv.wait(srv.submit([x], [o], [q], w, a, bnd))
    st = srv.stats()
    assert st["completed"] == 2 and st["cache_misses"] == 0 and st["cache_hits"] == 2
    assert st["p50_ms"] > 0 and st["failed"] == 0
    assert np.array_equal(outs[1], outs[0]) and np.array_equal(outs[2], outs[0])
    srv.close()
