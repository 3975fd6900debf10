"""The pins must fail on plausible mistakes.

Each case plants one mistake in the oracle (monkeypatched, CPU only) and
checks that at least one pin of the paper-form / brute-force / library
suites then fails.
"""
import math

import numpy as np
import pytest

import oracle
import oracle.dctf_oracle as od
from tests import test_oracle_dct as t_dct
from tests import test_oracle_filter as t_filt
from tests import test_oracle_paper_form as t_paper

_orig_build_H = od.build_H
_orig_dct = od.dct_matrix


def h_convolution(w, anchor, n, boundary):
    mh, mw = np.shape(w)
    return _orig_build_H(np.asarray(w)[::-1, ::-1], (mh - 1 - anchor[0], mw - 1 - anchor[1]), n, boundary)


def h_transposed(w, anchor, n, boundary):
    return _orig_build_H(w, anchor, n, boundary).T


def h_swapped_anchor(w, anchor, n, boundary):
    w = np.asarray(w)
    if w.shape[0] == w.shape[1]:
        return _orig_build_H(w, (anchor[1], anchor[0]), n, boundary)
    return _orig_build_H(w, anchor, n, boundary)


def h_dropped_term(w, anchor, n, boundary):
    w = np.array(w, dtype=float)
    w[-1, -1] = 0.0
    return _orig_build_H(w, anchor, n, boundary)


def h_wrong_boundary(w, anchor, n, boundary):
    return _orig_build_H(w, anchor, n, 1 - boundary)


def dct_no_alpha0(n):
    c = _orig_dct(n).copy()
    c[0] *= math.sqrt(2.0)
    return c


def dct_transposed(n):
    return _orig_dct(n).T.copy()


MUTANTS = {
    "convolution": ("build_H", h_convolution),
    "transposed_H": ("build_H", h_transposed),
    "swapped_anchor": ("build_H", h_swapped_anchor),
    "dropped_term": ("build_H", h_dropped_term),
    "wrong_boundary": ("build_H", h_wrong_boundary),
    "dct_alpha": ("dct_matrix", dct_no_alpha0),
    "dct_transposed": ("dct_matrix", dct_transposed),
}


def _pins():
    sym = t_paper.load_symbolic()
    return [
        lambda: t_paper.test_paper_equations_equal_oracle_operator(sym, oracle.ZERO),
        lambda: t_paper.test_paper_equations_equal_oracle_operator(sym, oracle.REPLICATE),
        lambda: t_filt.test_spatial_filter_brute_force_4x4(oracle.REPLICATE, 2, 3),
        lambda: t_filt.test_operator_route_equals_spatial_route_fp64(),
        lambda: t_dct.test_dct_matrix_matches_scipy(8),
        lambda: t_dct.test_blockwise_dct_matches_scipy(8),
    ]


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, monkeypatch):
    attr, fn = MUTANTS[name]
    monkeypatch.setattr(od, attr, fn)
    monkeypatch.setattr(oracle, attr, fn)
    failures = 0
    for pin in _pins():
        try:
            pin()
        except AssertionError:
            failures += 1
    assert failures > 0, f"mutant {name} passed every pin"


def test_unmutated_oracle_passes_every_pin():
    for pin in _pins():
        pin()


# ----------------------------------------------- Kronecker (sandwich) form
from tests import test_oracle_kron as t_kron  # noqa: E402

_orig_filter_1d = od.filter_1d
_orig_kron_factors = od.kron_factors
_orig_apply_kron = od.apply_kron


def f1d_shifted_anchor(v, a, n, boundary):
    return _orig_filter_1d(v, min(a + 1, len(v) - 1) if len(v) > 1 else a, n, boundary)


def kf_swapped(w, anchor, n, boundary):
    return [(b, a) for a, b in _orig_kron_factors(w, anchor, n, boundary)]


def ak_untransposed(factors, coeffs, n):
    return _orig_apply_kron([(a, b.T) for a, b in factors], coeffs, n)


KRON_MUTANTS = {
    "kron_anchor": ("filter_1d", f1d_shifted_anchor),
    "kron_swapped": ("kron_factors", kf_swapped),
    "kron_untransposed": ("apply_kron", ak_untransposed),
}


def _kron_pins():
    return [
        lambda: t_kron.test_kron_sum_equals_dense_operator(0, oracle.ZERO),
        lambda: t_kron.test_kron_sum_equals_dense_operator(1, oracle.REPLICATE),
        lambda: t_kron.test_sandwich_apply_equals_dense_apply(oracle.REPLICATE),
    ]


@pytest.mark.parametrize("name", sorted(KRON_MUTANTS))
def test_kron_mutant_is_caught(name, monkeypatch):
    attr, fn = KRON_MUTANTS[name]
    monkeypatch.setattr(od, attr, fn)
    monkeypatch.setattr(oracle, attr, fn)
    failures = 0
    for pin in _kron_pins():
        try:
            pin()
        except AssertionError:
            failures += 1
    assert failures > 0, f"mutant {name} passed every pin"


# ----------------------------------------------------- int16 serving path
from tests import test_oracle_int16 as t_i16  # noqa: E402

_orig_serve = od.serve_blocks


def serve_swapped_tables(q_in, qtab_in, m, qtab_out):
    return _orig_serve(q_in, qtab_out, m, qtab_in)


def serve_transposed_M(q_in, qtab_in, m, qtab_out):
    return _orig_serve(q_in, qtab_in, np.asarray(m).T, qtab_out)


def requantise_half_even(y, qtab):
    v = np.asarray(y, dtype=np.float64) / np.asarray(qtab, dtype=np.float64).ravel()[None, :]
    return np.clip(np.round(v), -32768, 32767).astype(np.int16)


def cmp_wrong_saturation(v_ref, q_test, band=1e-4):
    # the saturation bound of the reference rounding off by one at the bottom
    v = np.asarray(v_ref, dtype=np.float64).ravel()
    t = np.asarray(q_test).ravel()
    frac = np.abs(v - np.floor(v) - 0.5)
    inside = (frac < band) & (v > -32768.5 - band) & (v < 32767.5 + band)
    ref = np.clip(oracle.round_half_away(v), -32767, 32767)
    bad = (ref != t) & ~inside
    return {"mismatch": int(bad.sum()), "band": int(inside.sum()), "total": int(v.size)}


def cmp_wide_band_edge(v_ref, q_test, band=1e-4):
    # ties counted past the saturation edge, where both neighbours saturate
    v = np.asarray(v_ref, dtype=np.float64).ravel()
    t = np.asarray(q_test).ravel()
    frac = np.abs(v - np.floor(v) - 0.5)
    inside = (frac < band) & (v > -32769.5 - band) & (v < 32768.5 + band)
    ref = np.clip(oracle.round_half_away(v), -32768, 32767)
    bad = (ref != t) & ~inside
    return {"mismatch": int(bad.sum()), "band": int(inside.sum()), "total": int(v.size)}


I16_MUTANTS = {
    "serve_swapped_tables": ("serve_blocks", serve_swapped_tables),
    "serve_transposed_M": ("serve_blocks", serve_transposed_M),
    "requantise_half_even": ("requantise", requantise_half_even),
    "compare_wrong_saturation": ("int16_compare", cmp_wrong_saturation),
    "compare_wide_band_edge": ("int16_compare", cmp_wide_band_edge),
}


def _i16_pins():
    return [
        t_i16.test_serve_blocks_hand_computed,
        t_i16.test_serve_blocks_tables_not_interchangeable,
        t_i16.test_serve_blocks_dc_only_block_replicate,
        t_i16.test_int16_compare_saturation_and_band,
    ]


@pytest.mark.parametrize("name", sorted(I16_MUTANTS))
def test_int16_mutant_is_caught(name, monkeypatch):
    attr, fn = I16_MUTANTS[name]
    monkeypatch.setattr(od, attr, fn)
    monkeypatch.setattr(oracle, attr, fn)
    failures = 0
    for pin in _i16_pins():
        try:
            pin()
        except AssertionError:
            failures += 1
    assert failures > 0, f"mutant {name} passed every pin"


def test_unmutated_int16_oracle_passes_every_pin():
    for pin in _i16_pins():
        pin()
