"""Plain FP64 reference implementation of block-DCT-domain filtering.

Test infrastructure only (tests, smoke check, CPU baseline); never imported
by the library.  No blocking, fusion or reordering beyond the definitions.

Conventions
-----------
* A block is an N x N array ``x[i, j]`` (i = row, j = column).
* ``vec`` is row-major: element (i, j) of a block sits at index i*N + j, and
  coefficient (u, v) of a DCT block at u*N + v (u vertical, v horizontal
  frequency).  With this order vec(C X C^T) = (C kron C) vec(X).
* Coefficient arrays are ``[nblocks, N*N]``, blocks in raster order of the
  image.
* A mask ``w`` is ``[mh, mw]`` with an anchor (ar, ac): the mask entry that
  sits on the output pixel.  The filter is a correlation (Eq. 5 as the
  printed matrices of Eq. 6-18 implement it):
      out(i, j) = sum_{r, c} w[r, c] * x(i + r - ar, j + c - ac)
  with x outside the block either 0 (zero padding, Sec. II.B) or the nearest
  pixel of the same block (border replication, Sec. II.C).
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "ZERO", "REPLICATE", "dct_matrix", "image_to_blocks", "blocks_to_image",
    "dct2_blocks", "idct2_blocks", "spatial_filter_blocks", "build_H",
    "kron_dct", "build_M", "apply_M", "round_half_away", "to_uint8",
    "dequantise", "requantise", "serve_blocks", "pixel_route",
    "coefficient_route", "uint8_compare", "int16_compare",
    "mask_rank_terms", "filter_1d", "kron_factors", "apply_kron",
]

ZERO, REPLICATE = 0, 1


# ------------------------------------------------------------ Sec. II.A
def dct_matrix(n: int) -> np.ndarray:
    """Orthonormal DCT-II matrix C (Sec. II.A, Eq. 1-2).

    C[u, x] = alpha(u) cos(pi (2x + 1) u / (2n)), alpha(0) = sqrt(1/n),
    alpha(u > 0) = sqrt(2/n); these alphas make C orthogonal, so
    C^-1 = C^T (Eq. 2).
    """
    c = np.empty((n, n), dtype=np.float64)
    for u in range(n):
        alpha = math.sqrt(1.0 / n) if u == 0 else math.sqrt(2.0 / n)
        for x in range(n):
            c[u, x] = alpha * math.cos(math.pi * (2 * x + 1) * u / (2 * n))
    return c


def image_to_blocks(img: np.ndarray, n: int) -> np.ndarray:
    """Split an [h, w] image into [nblocks, n, n] blocks, raster order."""
    h, w = img.shape
    if h % n or w % n:
        raise ValueError("image sides must be multiples of the block size")
    return (img.reshape(h // n, n, w // n, n).transpose(0, 2, 1, 3)
            .reshape(-1, n, n).astype(np.float64))


def blocks_to_image(blocks: np.ndarray, h: int, w: int) -> np.ndarray:
    """Inverse of image_to_blocks (dtype kept)."""
    n = blocks.shape[-1]
    return (blocks.reshape(h // n, w // n, n, n).transpose(0, 2, 1, 3)
            .reshape(h, w))


def dct2_blocks(blocks: np.ndarray) -> np.ndarray:
    """BLOCK = C block C^T for every block (Eq. 1); returns [nb, n*n]."""
    n = blocks.shape[-1]
    c = dct_matrix(n)
    out = np.einsum("ui,bij,vj->buv", c, blocks.astype(np.float64), c)
    return out.reshape(-1, n * n)


def idct2_blocks(coeffs: np.ndarray, n: int) -> np.ndarray:
    """block = C^T BLOCK C for every block (Eq. 3); returns [nb, n, n]."""
    c = dct_matrix(n)
    y = np.asarray(coeffs, dtype=np.float64).reshape(-1, n, n)
    return np.einsum("ui,buv,vj->bij", c, y, c)


# ------------------------------------------------------ Sec. II.B / II.C
def _check_mask(w: np.ndarray, anchor, n: int, boundary: int) -> None:
    mh, mw = w.shape
    ar, ac = anchor
    if not (1 <= mh <= n and 1 <= mw <= n):
        raise ValueError("mask must fit inside the block")
    if not (0 <= ar < mh and 0 <= ac < mw):
        raise ValueError("anchor outside the mask")
    if boundary not in (ZERO, REPLICATE):
        raise ValueError("boundary must be ZERO or REPLICATE")


def spatial_filter_blocks(blocks: np.ndarray, w: np.ndarray, anchor,
                          boundary: int) -> np.ndarray:
    """Per-block spatial filtering (Eq. 5; padding of Sec. II.B / II.C).

    Each block is padded on its own: with zeros (Sec. II.B) or by copying its
    nearest edge pixel (Sec. II.C, Fig. 1); pixels of neighbouring blocks are
    never read.  Then out(i, j) = sum_{r,c} w[r, c] xp(i + r, j + c) where xp
    is the padded block with (ar, ac) rows/columns added before it.
    Returns [nb, n, n] float64.
    """
    blocks = np.asarray(blocks, dtype=np.float64)
    n = blocks.shape[-1]
    w = np.asarray(w, dtype=np.float64)
    _check_mask(w, anchor, n, boundary)
    mh, mw = w.shape
    ar, ac = anchor
    pad = ((0, 0), (ar, mh - 1 - ar), (ac, mw - 1 - ac))
    xp = np.pad(blocks, pad, mode="constant" if boundary == ZERO else "edge")
    out = np.zeros_like(blocks)
    for r in range(mh):
        for c in range(mw):
            out += w[r, c] * xp[:, r:r + n, c:c + n]
    return out


def build_H(w: np.ndarray, anchor, n: int, boundary: int) -> np.ndarray:
    """Spatial operator H with vec(out) = H vec(block) (Eq. 5, Sec. II.C).

    Row (i, j) of H collects w[r, c] at column (s, t), the pixel the mask
    entry reads: s = i + r - ar, t = j + c - ac.  Zero padding drops entries
    whose (s, t) leaves the block; border replication moves them to the
    nearest pixel of the block (clamping s and t to [0, n-1] independently,
    which is how Eq. 13-18 fold the outside neighbours onto edge pixels).
    """
    w = np.asarray(w, dtype=np.float64)
    _check_mask(w, anchor, n, boundary)
    mh, mw = w.shape
    ar, ac = anchor
    h = np.zeros((n * n, n * n), dtype=np.float64)
    for i in range(n):
        for j in range(n):
            for r in range(mh):
                for c in range(mw):
                    s, t = i + r - ar, j + c - ac
                    if boundary == ZERO:
                        if not (0 <= s < n and 0 <= t < n):
                            continue
                    else:
                        s = min(max(s, 0), n - 1)
                        t = min(max(t, 0), n - 1)
                    h[i * n + j, s * n + t] += w[r, c]
    return h


def kron_dct(n: int) -> np.ndarray:
    """K = C kron C, the 2-D DCT of a row-major vectorised block (Eq. 1)."""
    c = dct_matrix(n)
    return np.kron(c, c)


def build_M(w: np.ndarray, anchor, n: int, boundary: int) -> np.ndarray:
    """DCT-domain operator M = K H K^T (Eq. 7 applied to the whole filter).

    Eq. 7 moves each spatial matrix product into the DCT domain by
    conjugation with C; for the vectorised block the spatial filter is H, so
    its DCT-domain form is K H K^-1 = K H K^T (Eq. 2).  Then
    vec(F) = M vec(BLOCK) is Eq. 11 (zero padding) or Eq. 20 (border
    replication).
    """
    k = kron_dct(n)
    return k @ build_H(w, anchor, n, boundary) @ k.T


# ------------------------------------ Sec. II.B-C, Eq. 11 / Eq. 20 (Kronecker form)
def mask_rank_terms(w: np.ndarray, rel_tol: float = 1e-13):
    """w = sum_t u_t v_t^T with as few terms as the mask's rank (its SVD;
    terms whose singular value is below rel_tol * the largest are dropped)."""
    w = np.asarray(w, dtype=np.float64)
    u, s, vt = np.linalg.svd(w)
    if s.size == 0 or s[0] == 0.0:
        return []
    return [(s[t] * u[:, t], vt[t, :]) for t in range(s.size) if s[t] > rel_tol * s[0]]


def filter_1d(v: np.ndarray, a: int, n: int, boundary: int) -> np.ndarray:
    """n x n matrix of the 1-D correlation along one axis of a block:
    out[i] = sum_r v[r] x(i + r - a), x outside [0, n) zero (Sec. II.B) or
    the nearest end value (Sec. II.C)."""
    h = np.zeros((n, n), dtype=np.float64)
    for i in range(n):
        for r in range(len(v)):
            s = i + r - a
            if boundary == ZERO:
                if 0 <= s < n:
                    h[i, s] += v[r]
            else:
                h[i, min(max(s, 0), n - 1)] += v[r]
    return h


def kron_factors(w: np.ndarray, anchor, n: int, boundary: int):
    """M = sum_t A_t kron B_t, the form of Eq. 11 (three Kronecker terms for a
    3x3 mask) for any mask.

    A separable mask u v^T filters along the block's rows and columns
    independently, and both paddings act on each axis on its own (a pixel is
    dropped when either coordinate leaves the block; replication clamps
    each coordinate), so its H is the Kronecker product of the two 1-D
    operators.  Writing w as a sum of rank-1 terms and conjugating by C
    (Eq. 7) gives A_t = C H_u C^T, B_t = C H_v C^T; vec(A X B^T) =
    (A kron B) vec(X) for the row-major vec.
    """
    w = np.asarray(w, dtype=np.float64)
    _check_mask(w, anchor, n, boundary)
    ar, ac = anchor
    c = dct_matrix(n)
    return [(c @ filter_1d(u, ar, n, boundary) @ c.T, c @ filter_1d(v, ac, n, boundary) @ c.T)
            for u, v in mask_rank_terms(w)]


def apply_kron(factors, coeffs: np.ndarray, n: int) -> np.ndarray:
    """y_b = sum_t vec(A_t X_b B_t^T) for every block: the sandwich products
    of Eq. 11 / Eq. 12; [nb, n*n] float64."""
    x = np.asarray(coeffs, dtype=np.float64).reshape(-1, n, n)
    y = np.zeros_like(x)
    for a, b in factors:
        y += np.einsum("ik,bkl,jl->bij", a, x, b)
    return y.reshape(-1, n * n)


def apply_M(m: np.ndarray, coeffs: np.ndarray) -> np.ndarray:
    """y_b = M x_b for every block (Eq. 11 / Eq. 20); [nb, n*n] float64."""
    x = np.asarray(coeffs, dtype=np.float64)
    return x @ np.asarray(m, dtype=np.float64).T


# ---------------------------------------------------------- Sec. III
def round_half_away(v: np.ndarray) -> np.ndarray:
    """Round to nearest, ties away from zero."""
    v = np.asarray(v, dtype=np.float64)
    return np.sign(v) * np.floor(np.abs(v) + 0.5)


def to_uint8(p: np.ndarray) -> np.ndarray:
    """Conversion to uint8 (Sec. III): round half away from zero, saturate."""
    return np.clip(round_half_away(p), 0, 255).astype(np.uint8)


def pixel_route(img: np.ndarray, n: int, w, anchor, boundary) -> np.ndarray:
    """Spatial-domain result as FP64 blocks [nb, n, n] (Sec. III, Fig. 2(d, e))."""
    return spatial_filter_blocks(image_to_blocks(img, n), w, anchor, boundary)


def coefficient_route(coeffs: np.ndarray, n: int, w, anchor, boundary) -> np.ndarray:
    """DCT-domain result mapped back to pixels, FP64 [nb, n, n] (Fig. 2(h))."""
    return idct2_blocks(apply_M(build_M(w, anchor, n, boundary), coeffs), n)


def uint8_compare(p_ref: np.ndarray, u8_test: np.ndarray, band: float = 1e-4):
    """Compare uint8 pixels with an FP64 reference, outside the tie band.

    A reference value whose fractional part lies within ``band`` of 0.5 may
    legitimately round either way; such pixels are counted and excluded.
    Values that saturate (< -0.5 or >= 255.5 by more than the band) cannot
    tie.  Returns dict(mismatch, band, total).
    """
    p = np.asarray(p_ref, dtype=np.float64).ravel()
    t = np.asarray(u8_test).ravel()
    frac = np.abs(p - np.floor(p) - 0.5)
    inside = (frac < band) & (p > -0.5 - band) & (p < 255.5 + band)
    ref = to_uint8(p)
    bad = (ref != t) & ~inside
    return {"mismatch": int(bad.sum()), "band": int(inside.sum()), "total": int(p.size)}


# --------------------------------------------------- serving (int16)
def dequantise(q_in: np.ndarray, qtab: np.ndarray) -> np.ndarray:
    """x[k] = Q_in[k] * q[k] for every block; [nb, n*n] float64."""
    return np.asarray(q_in, dtype=np.float64) * np.asarray(qtab, dtype=np.float64).ravel()[None, :]


def requantise(y: np.ndarray, qtab: np.ndarray) -> np.ndarray:
    """Q_out[k] = sat_int16(round_half_away(y[k] / q[k]))."""
    v = np.asarray(y, dtype=np.float64) / np.asarray(qtab, dtype=np.float64).ravel()[None, :]
    return np.clip(round_half_away(v), -32768, 32767).astype(np.int16)


def serve_blocks(q_in: np.ndarray, qtab_in: np.ndarray, m: np.ndarray,
                 qtab_out: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Quantised coefficients in, quantised filtered coefficients out.

    Returns (Q_out int16, the FP64 value y/q before rounding)."""
    y = apply_M(m, dequantise(q_in, qtab_in))
    v = y / np.asarray(qtab_out, dtype=np.float64).ravel()[None, :]
    return requantise(y, qtab_out), v


def int16_compare(v_ref: np.ndarray, q_test: np.ndarray, band: float = 1e-4):
    """Like uint8_compare for requantised int16 (saturation at +-32767.5)."""
    v = np.asarray(v_ref, dtype=np.float64).ravel()
    t = np.asarray(q_test).ravel()
    frac = np.abs(v - np.floor(v) - 0.5)
    inside = (frac < band) & (v > -32768.5 - band) & (v < 32767.5 + band)
    ref = np.clip(round_half_away(v), -32768, 32767)
    bad = (ref != t) & ~inside
    return {"mismatch": int(bad.sum()), "band": int(inside.sum()), "total": int(v.size)}
