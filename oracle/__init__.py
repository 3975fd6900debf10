"""CPU FP64 oracle for block-DCT-domain filtering (test infrastructure).

This package is test infrastructure, not part of the library: only the
tests, the smoke check and the benchmark's CPU-baseline leg import it.  It
shares no code with the CUDA library and never calls it.

It is the plain definition of what the library computes, in float64 numpy:

* the orthonormal DCT-II matrix and the blockwise 2-D DCT / inverse DCT
  (Sec. II.A, Eq. 1-3);
* per-block spatial filtering with zero padding (Sec. II.B, Eq. 5) or border
  replication (Sec. II.C), the mask applied as a correlation (the reading of
  Eq. 5 that the printed matrices of Eq. 6-18 implement);
* the explicit spatial operator H on a vectorised block, and the DCT-domain
  operator M = (C kron C) H (C kron C)^T obtained from it by Eq. 7;
* y_b = M x_b for every block, uint8 conversion, and the int16
  dequantise / requantise of a JPEG-style serving path.

Every function cites the passage it follows.
"""
from .dctf_oracle import *  # noqa: F401,F403
from .dctf_oracle import __all__  # noqa: F401
