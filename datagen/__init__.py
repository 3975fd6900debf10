"""Seeded synthetic inputs for block-DCT filtering.

This module holds no arithmetic of the filtering method: it draws pixel
images, filter masks, quantisation tables and request streams, and nothing
else.  The orthonormal DCT, the filter operator and every comparison live in
``oracle/`` (CPU, test infrastructure) and in the CUDA library; both take the
arrays made here as their inputs.

Random streams.  Every array comes from its own ``numpy.random.Generator``
seeded by ``SeedSequence(0, spawn_key=(workload, item, kind))``, so any one
image or mask can be regenerated alone, in any order, on any machine.

Workloads (sizes follow the paper's 8x8 blocks and 3x3 masks, scaled up):

* ``W_SMALL``    256x256 image, 8x8 blocks, 3x3 Gaussian sigma=1, zero padding.
* ``W_HEADLINE`` 4096x4096 image, 8x8 blocks, random asymmetric 5x5 mask,
                 anchor (1, 3), border replication.
* ``W_GROUPED``  64 images of seeded sizes (multiples of 8 in [64, 2048]),
                 one mask and boundary mode per image.
* ``W_LARGE``    8192x8192 image, 16x16 blocks, perturbed 9x9 Gaussian,
                 border replication.
* ``W_SERVING``  Poisson stream of 1920x1088 4:2:0 frames and 512x512
                 stills, int16 quantised coefficients, 32 seeded masks.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

W_SMALL, W_HEADLINE, W_GROUPED, W_LARGE, W_SERVING = 1, 2, 3, 4, 5

ZERO, REPLICATE = 0, 1

# kinds of random stream within one workload item
_K_IMAGE, _K_MASK, _K_SIZE, _K_QUANT, _K_ARRIVAL = 0, 1, 2, 3, 4


def rng(workload: int, item: int = 0, kind: int = 0) -> np.random.Generator:
    """The generator for one (workload, item, kind) stream."""
    return np.random.default_rng(
        np.random.SeedSequence(0, spawn_key=(workload, item, kind)))


def _round_half_away(v: np.ndarray) -> np.ndarray:
    return np.sign(v) * np.floor(np.abs(v) + 0.5)


def synthetic_image(h: int, w: int, g: np.random.Generator) -> np.ndarray:
    """uint8 image: 128 + 8 low-frequency 2-D cosines + N(0, 10^2) noise.

    I(y, x) = 128 + sum_k a_k cos(2 pi (fy_k y / h + fx_k x / w) + phi_k)
              + n(y, x),  a_k ~ U[10, 40], fy_k, fx_k ~ U{0..7},
    phi_k ~ U[0, 2 pi), n ~ N(0, 10^2); rounded half away from zero and
    clipped to [0, 255].  Rows are made in chunks to bound host memory.
    """
    a = g.uniform(10.0, 40.0, 8)
    fy = g.integers(0, 8, 8)
    fx = g.integers(0, 8, 8)
    phi = g.uniform(0.0, 2.0 * math.pi, 8)
    out = np.empty((h, w), dtype=np.uint8)
    xs = np.arange(w, dtype=np.float64)[None, :]
    chunk = max(1, (1 << 22) // max(w, 1))
    for y0 in range(0, h, chunk):
        y1 = min(h, y0 + chunk)
        ys = np.arange(y0, y1, dtype=np.float64)[:, None]
        v = np.full((y1 - y0, w), 128.0)
        for k in range(8):
            v += a[k] * np.cos(2.0 * math.pi * (fy[k] * ys / h + fx[k] * xs / w) + phi[k])
        v += g.normal(0.0, 10.0, (y1 - y0, w))
        out[y0:y1] = np.clip(_round_half_away(v), 0, 255).astype(np.uint8)
    return out


# ----------------------------------------------------------------- masks
def gaussian_mask(m: int, sigma: float) -> np.ndarray:
    """m x m isotropic Gaussian centred on ((m-1)/2, (m-1)/2), sum 1."""
    c = (m - 1) / 2.0
    r = np.arange(m, dtype=np.float64) - c
    g = np.exp(-(r[:, None] ** 2 + r[None, :] ** 2) / (2.0 * sigma * sigma))
    return g / g.sum()


def uniform_random_mask(mh: int, mw: int, g: np.random.Generator,
                        min_abs_sum: float = 0.5) -> np.ndarray:
    """Entries U[-1, 1], redrawn until |sum| >= min_abs_sum, then scaled
    to sum 1 (the redraw keeps sum(|w|) bounded by mh*mw/min_abs_sum)."""
    while True:
        w = g.uniform(-1.0, 1.0, (mh, mw))
        s = w.sum()
        if abs(s) >= min_abs_sum:
            return w / s


def laplacian_sharpen() -> np.ndarray:
    """3x3 sharpen: centre 5, 4-neighbours -1 (sum 1)."""
    return np.array([[0., -1., 0.], [-1., 5., -1.], [0., -1., 0.]])


def motion_blur_1x5() -> np.ndarray:
    """1x5 horizontal box of 0.2."""
    return np.full((1, 5), 0.2)


def perturbed_gaussian(m: int, sigma: float, amp: float,
                       g: np.random.Generator) -> np.ndarray:
    """Gaussian + amp * U[-1, 1] per entry, rescaled to sum 1 (asymmetric)."""
    w = gaussian_mask(m, sigma) + amp * g.uniform(-1.0, 1.0, (m, m))
    return w / w.sum()


def magic_square_3() -> np.ndarray:
    """The order-3 magic square (rows, columns and diagonals sum to 15)."""
    return np.array([[8., 1., 6.], [3., 5., 7.], [4., 9., 2.]])


def centred_anchor(mh: int, mw: int) -> tuple[int, int]:
    return ((mh - 1) // 2, (mw - 1) // 2)


# ------------------------------------------------------------- workloads
@dataclass
class FilterJob:
    """One image and the mask applied to it."""
    image: np.ndarray          # uint8 [h, w], h and w multiples of n
    n: int                     # block size
    mask: np.ndarray           # float64 [mh, mw]
    anchor: tuple[int, int]    # (row, col) in the mask, 0-based
    boundary: int              # ZERO or REPLICATE
    name: str = ""


def small_job() -> FilterJob:
    img = synthetic_image(256, 256, rng(W_SMALL, 0, _K_IMAGE))
    return FilterJob(img, 8, gaussian_mask(3, 1.0), (1, 1), ZERO,
                     "256x256 8x8 gauss3 zero")


def headline_mask() -> np.ndarray:
    return uniform_random_mask(5, 5, rng(W_HEADLINE, 0, _K_MASK))


def headline_job(h: int = 4096, w: int = 4096) -> FilterJob:
    img = synthetic_image(h, w, rng(W_HEADLINE, 0, _K_IMAGE))
    return FilterJob(img, 8, headline_mask(), (1, 3), REPLICATE,
                     f"{h}x{w} 8x8 rand5x5 replicate")


def grouped_mask(i: int) -> tuple[np.ndarray, tuple[int, int], int, str]:
    """Image i of the grouped batch: mask kind i mod 4, boundary (i div 4) mod 2."""
    kind = i % 4
    boundary = (i // 4) % 2
    if kind == 0:
        w, a, nm = laplacian_sharpen(), (1, 1), "laplace3"
    elif kind == 1:
        w, a, nm = gaussian_mask(7, 2.0), (3, 3), "gauss7"
    elif kind == 2:
        w, a, nm = motion_blur_1x5(), (0, 2), "motion1x5"
    else:
        w, a, nm = uniform_random_mask(5, 5, rng(W_GROUPED, i, _K_MASK)), (2, 2), "rand5x5"
    return w, a, boundary, nm


def grouped_sizes(count: int = 64) -> list[tuple[int, int]]:
    g = rng(W_GROUPED, 0, _K_SIZE)
    hw = 8 * g.integers(8, 257, (count, 2))
    return [(int(h), int(w)) for h, w in hw]


def grouped_jobs(count: int = 64, scale: float = 1.0) -> list[FilterJob]:
    """The grouped batch; ``scale`` < 1 shrinks every side (for fast tests),
    keeping multiples of 8 and at least one block."""
    jobs = []
    for i, (h, w) in enumerate(grouped_sizes(count)):
        if scale != 1.0:
            h = max(8, 8 * int(round(h * scale / 8)))
            w = max(8, 8 * int(round(w * scale / 8)))
        mask, anchor, boundary, nm = grouped_mask(i)
        img = synthetic_image(h, w, rng(W_GROUPED, i, _K_IMAGE))
        jobs.append(FilterJob(img, 8, mask, anchor, boundary, f"{h}x{w} {nm}"))
    return jobs


def large_mask() -> np.ndarray:
    return perturbed_gaussian(9, 2.5, 0.05, rng(W_LARGE, 0, _K_MASK))


def large_job(h: int = 8192, w: int = 8192) -> FilterJob:
    img = synthetic_image(h, w, rng(W_LARGE, 0, _K_IMAGE))
    return FilterJob(img, 16, large_mask(), (4, 4), REPLICATE,
                     f"{h}x{w} 16x16 pgauss9 replicate")


# --------------------------------------------------------------- serving
def quant_table(s: int, n: int = 8) -> np.ndarray:
    """q[u, v] = 1 + round(s (1 + u + v)), uint16 [n, n]."""
    u = np.arange(n)[:, None]
    v = np.arange(n)[None, :]
    return (1 + np.round(s * (1 + u + v))).astype(np.uint16)


def serving_mask(j: int) -> tuple[np.ndarray, tuple[int, int], int]:
    """Mask j of 32: size 3..7, even j symmetric Gaussian (sigma from the
    seed), odd j asymmetric uniform; boundary (j div 2) mod 2."""
    m = 3 + (j % 5)
    g = rng(W_SERVING, j, _K_MASK)
    if j % 2 == 0:
        w = gaussian_mask(m, float(g.uniform(0.6, 2.0)))
    else:
        w = uniform_random_mask(m, m, g)
    return w, centred_anchor(m, m), (j // 2) % 2


FRAME_PLANES = ((1088, 1920), (544, 960), (544, 960))
STILL_PLANES = ((512, 512),)


@dataclass
class Request:
    rid: int
    arrival_s: float
    planes: list = field(default_factory=list)   # uint8 images
    q_scale: list = field(default_factory=list)  # s per plane
    mask_id: int = 0
    kind: str = "still"


def serving_stream(count: int, rate_hz: float, scale: float = 1.0,
                   with_pixels: bool = True) -> list[Request]:
    """``count`` requests with Poisson arrivals at ``rate_hz``: half
    1920x1088 4:2:0 frames, half 512x512 stills.  ``scale`` < 1 shrinks
    plane sides (multiples of 16 kept) for fast tests."""
    g = rng(W_SERVING, 0, _K_ARRIVAL)
    t = np.cumsum(g.exponential(1.0 / rate_hz, count))
    reqs = []
    for i in range(count):
        gi = rng(W_SERVING, 1000 + i, _K_QUANT)
        frame = bool(gi.integers(0, 2))
        shapes = FRAME_PLANES if frame else STILL_PLANES
        if scale != 1.0:
            shapes = tuple((max(16, 16 * int(round(h * scale / 16))),
                            max(16, 16 * int(round(w * scale / 16))))
                           for h, w in shapes)
        r = Request(i, float(t[i]), mask_id=int(gi.integers(0, 32)),
                    kind="frame" if frame else "still")
        for p, (h, w) in enumerate(shapes):
            r.q_scale.append(int(gi.choice([1, 2, 4])))
            if with_pixels:
                r.planes.append(synthetic_image(h, w, rng(W_SERVING, 1000 + i, 10 + p)))
            else:
                r.planes.append((h, w))
        reqs.append(r)
    return reqs
