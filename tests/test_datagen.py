"""The seeded generators: determinism, shapes and closed-form masks."""
import numpy as np

import datagen


def test_gaussian_3x3_sigma1_closed_form():
    g = datagen.gaussian_mask(3, 1.0)
    e = np.exp(-0.5)
    tot = 1 + 4 * e + 4 * e * e
    assert abs(g[1, 1] - 1 / tot) < 1e-15 and abs(g[1, 1] - 0.20418) < 1e-5
    assert abs(g[0, 1] - e / tot) < 1e-15 and abs(g[0, 1] - 0.12384) < 1e-5
    assert abs(g[0, 0] - e * e / tot) < 1e-15 and abs(g[0, 0] - 0.07511) < 1e-5


def test_image_deterministic_and_in_range():
    a = datagen.synthetic_image(64, 72, datagen.rng(1, 0, 0))
    b = datagen.synthetic_image(64, 72, datagen.rng(1, 0, 0))
    assert a.dtype == np.uint8 and a.shape == (64, 72)
    assert (a == b).all()
    assert 80 < a.mean() < 180 and a.std() > 5


def test_masks():
    w = datagen.headline_mask()
    assert w.shape == (5, 5) and abs(w.sum() - 1) < 1e-12
    assert np.abs(w - w[::-1, ::-1]).max() > 0.01        # asymmetric
    assert np.linalg.matrix_rank(w) > 1                   # inseparable
    m = datagen.magic_square_3()
    assert (m.sum(0) == 15).all() and (m.sum(1) == 15).all() and np.trace(m) == 15
    lg = datagen.large_mask()
    assert lg.shape == (9, 9) and abs(lg.sum() - 1) < 1e-12
    for j in range(32):
        w, a, bnd = datagen.serving_mask(j)
        assert 3 <= w.shape[0] <= 7 and abs(w.sum() - 1) < 1e-12 and bnd in (0, 1)


def test_grouped_sizes():
    s = datagen.grouped_sizes()
    assert len(s) == 64
    assert all(h % 8 == 0 and w % 8 == 0 and 64 <= h <= 2048 and 64 <= w <= 2048 for h, w in s)
    kinds = {datagen.grouped_mask(i)[3] for i in range(8)}
    assert kinds == {"laplace3", "gauss7", "motion1x5", "rand5x5"}
    assert {datagen.grouped_mask(i)[2] for i in range(8)} == {0, 1}


def test_quant_table():
    q = datagen.quant_table(4)
    assert q[0, 0] == 5 and q[7, 7] == 1 + 4 * 15


def test_serving_stream():
    r = datagen.serving_stream(20, 1000.0, with_pixels=False)
    assert all(r[i].arrival_s < r[i + 1].arrival_s for i in range(19))
    kinds = {x.kind for x in r}
    assert kinds == {"frame", "still"}
    f = next(x for x in r if x.kind == "frame")
    assert f.planes == [(1088, 1920), (544, 960), (544, 960)]
