"""The LBM_Q16S code reference (tests/q16_ref.py) against properties its definition fixes."""
import numpy as np

from tests import q16_ref as Q
from tests.inputs import uniform


def test_grid_is_increasing_with_the_stated_spacings():
    a = Q.values()
    d = np.diff(a)
    assert (d > 0).all()
    assert a[0] == 0 and a[Q.MAXCODE] == 2 - 2 ** -13
    assert np.all(d[a[:-1] < 0.5] == 2 ** -15)
    assert np.all(d[(a[:-1] >= 0.5) & (a[:-1] < 1)] == 2 ** -14)
    assert np.all(d[a[:-1] >= 1] == 2 ** -13)


def test_roundtrip_of_every_code():
    S = 2.0 ** -6
    codes = np.arange(0x10000)
    codes = codes[(codes & 0x7FFF) != 0]  # -0 and +0 both decode to 0
    assert np.array_equal(Q.encode(Q.decode(codes, S), S), codes)


def test_nearest_by_brute_force():
    """encode picks the code whose value is nearest (ties to even), against a full scan."""
    S = 2.0 ** -5
    h = S * 2.2 * uniform(3, 400)
    grid = np.concatenate([-Q.values()[::-1], Q.values()])
    codes = np.concatenate([np.arange(Q.MAXCODE, -1, -1) | 0x8000, np.arange(Q.MAXCODE + 1)])
    for v in h:
        got = Q.encode(v, S)
        err = np.abs(grid * S - v)
        best = err.min()
        cand = codes[err == best]
        if abs(v) >= Q.values()[-1] * S:
            assert (got & Q.MAXCODE) == Q.MAXCODE
        else:
            assert got in cand
            assert abs(Q.decode(got, S) - v) == best


def test_ties_go_to_even_and_saturation():
    S = 1.0
    lo, hi = Q.values()[100], Q.values()[101]
    assert Q.encode((lo + hi) / 2, S) == 100   # 100 is even
    lo, hi = Q.values()[101], Q.values()[102]
    assert Q.encode((lo + hi) / 2, S) == 102
    assert Q.encode(5.0, S) == Q.MAXCODE and Q.encode(-5.0, S) == Q.MAXCODE | 0x8000
    assert Q.encode(np.nan, S) == Q.MAXCODE


def test_scales_are_powers_of_two_above_the_deviation_bounds():
    for U in (0.01, 0.05, 0.1, 0.2):
        for j in range(9):
            S = Q.scale(j, U)
            w = 4 / 9 if j == 0 else (1 / 9 if j < 5 else 1 / 36)
            K = 2.0 if j == 0 else (5.0 if j < 5 else 5.5)
            assert np.log2(2 * S) == np.round(np.log2(2 * S))
            assert K * w * U <= 2 * S < 2 * K * w * U
