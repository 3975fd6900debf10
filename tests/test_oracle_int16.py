"""Pins of the oracle's int16 serving path against values fixed by hand and by
the mathematics, not by the oracle itself.

The serving form dequantises with the input table, filters, and requantises
with the output table: x = Q_in * q_in, y = M x, Q_out =
sat_int16(round_half_away(y / q_out)).  The paper has no quantisation (it is
JPEG practice around Eq. 1 / Eq. 3); these cases fix the order of the two
tables, the orientation of M, the rounding rule and the int16 saturation.
"""
import numpy as np

import datagen
import oracle
from oracle import REPLICATE

# A 2 x 2 "block" (four coefficients) with an asymmetric operator, so a
# transposed M, swapped tables or another rounding rule each change the result.
M4 = np.array([[1.0, 2.0, 0.0, 0.0],
               [0.0, 1.0, 0.0, 0.0],
               [0.0, 0.0, 1.0, 0.0],
               [0.0, 0.0, 3.0, 1.0]])
Q_IN_TAB = np.array([1, 2, 3, 4], dtype=np.uint16)
Q_OUT_TAB = np.array([2, 4, 5, 1], dtype=np.uint16)


def test_serve_blocks_hand_computed():
    q = np.array([[3, -1, 2, 5],
                  [20000, 20000, -11000, 7]], dtype=np.int16)
    out, v = oracle.serve_blocks(q, Q_IN_TAB, M4, Q_OUT_TAB)
    # block 0: x = (3, -2, 6, 20); y = M x = (-1, -2, 6, 38);
    #          y / q_out = (-0.5, -0.5, 1.2, 38) -> half away from zero
    # block 1: x = (20000, 40000, -33000, 28);
    #          y = (100000, 40000, -33000, -98972);
    #          y / q_out = (50000, 10000, -6600, -98972) -> saturated ends
    assert v.tolist() == [[-0.5, -0.5, 1.2, 38.0], [50000.0, 10000.0, -6600.0, -98972.0]]
    assert out.dtype == np.int16
    assert out.tolist() == [[-1, -1, 1, 38], [32767, 10000, -6600, -32768]]


def test_serve_blocks_tables_not_interchangeable():
    # the same input with the tables swapped gives a different, also
    # hand-computed, answer: x = (6, -4, 10, 5), y = (-2, -4, 10, 35),
    # y / (1, 2, 3, 4) = (-2, -2, 3.33.., 8.75)
    q = np.array([[3, -1, 2, 5]], dtype=np.int16)
    out, _ = oracle.serve_blocks(q, Q_OUT_TAB, M4, Q_IN_TAB)
    assert out.tolist() == [[-2, -2, 3, 9]]


def test_serve_blocks_dc_only_block_replicate():
    # with border replication a constant block stays constant, scaled by the
    # mask sum (the DC column of M is (sum w) e_0, Sec. II.C), so a DC-only
    # input requantises to round(sum(w) * d * q_in[0] / q_out[0]) at index 0
    # and zero elsewhere, for any mask
    w, a = datagen.headline_mask(), (1, 3)
    assert abs(w.sum() - 1.0) < 1e-12
    q_in, q_out = datagen.quant_table(1).ravel(), datagen.quant_table(4).ravel()
    assert (q_in[0], q_out[0]) == (2, 5)
    m = oracle.build_M(w, a, 8, REPLICATE)
    for d, want in ((7, 3), (-9, -4), (12, 5), (16000, 6400)):
        q = np.zeros((1, 64), dtype=np.int16)
        q[0, 0] = d
        out, _ = oracle.serve_blocks(q, q_in, m, q_out)
        # sum(w) = 1: 7*2/5 = 2.8, -18/5 = -3.6, 24/5 = 4.8, 32000/5 = 6400
        assert out[0, 0] == want
        assert not out[0, 1:].any()


def test_int16_compare_saturation_and_band():
    # v: FP64 y / q_out.  Reference rounding saturates at the int16 ends.
    v = np.array([40000.0, 32767.5, 32768.5, -32768.5, -40000.0, 12.50004, 12.5002, -3.5])
    t = np.array([32767, 32767, 32767, -32768, -32768, 12, 13, -4], dtype=np.int16)
    st = oracle.int16_compare(v, t)
    # in the tie band: 32767.5 and -32768.5 (ties at the saturation edges),
    # 12.50004 (within 1e-4 of a tie) and -3.5 (an exact tie); not 12.5002
    assert st == {"mismatch": 0, "band": 4, "total": 8}
    # beyond the saturation bound no value can tie: 32768.5 must be 32767
    bad = t.copy()
    bad[2] = -5
    assert oracle.int16_compare(v, bad)["mismatch"] == 1
    # a saturated negative value must be -32768, not -32767
    bad = t.copy()
    bad[4] = -32767
    assert oracle.int16_compare(v, bad)["mismatch"] == 1
    # outside the band the rounding is checked: 12.5002 -> 13, not 12
    bad = t.copy()
    bad[6] = 12
    assert oracle.int16_compare(v, bad)["mismatch"] == 1
    # inside the band either neighbour is accepted
    ok = t.copy()
    ok[5] = 13
    ok[7] = -3
    assert oracle.int16_compare(v, ok)["mismatch"] == 0
