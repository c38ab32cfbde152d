"""Reference of the LBM_Q16S storage code, written from its definition (test helper).

A population's deviation h (from the rest state at the reference density) is stored as a 16-bit
code: sign bit, 2-bit exponent E, 13-bit mantissa M, of a = |h| / S with a per-direction scale S:
    E = 0:       a = M 2^-15
    E = 1, 2, 3: a = (2^13 + M) 2^(E - 16)
i.e. the representable a form the grid M 2^-15 on [0, 1/2), 2^-14 steps on [1/2, 1), 2^-13 steps
on [1, 2).  Encoding rounds a to the nearest grid point, ties to the even code, and saturates at
the largest code 0x7fff (a = 2 - 2^-13); NaN saturates as well.  No arithmetic of the library is
used here: the grid is built by enumeration and searched.
"""
import numpy as np

MAXCODE = 0x7FFF


def values() -> np.ndarray:
    """a of every magnitude code 0 .. 0x7fff (float64, exact)."""
    m = np.arange(MAXCODE + 1)
    E, M = m >> 13, m & 0x1FFF
    return np.where(E == 0, M * 2.0 ** -15, (8192 + M) * 2.0 ** (E - 16))


_GRID = values()


def decode(code, S: float) -> np.ndarray:
    code = np.asarray(code, dtype=np.int64)
    a = _GRID[code & MAXCODE]
    return np.where(code & 0x8000, -a, a) * S


def encode(h, S: float) -> np.ndarray:
    """Nearest code of h / S (ties to the even code), saturating; h is taken as given (float64)."""
    h = np.asarray(h, dtype=np.float64)
    a = np.abs(h) / S
    a = np.where(np.isnan(a), np.inf, a)
    k = np.searchsorted(_GRID, a)               # _GRID[k-1] < a <= _GRID[k]
    k = np.clip(k, 1, MAXCODE)
    lo, hi = _GRID[k - 1], _GRID[k]
    pick_hi = (hi - a < a - lo) | ((hi - a == a - lo) & (k % 2 == 0))
    mag = np.where(pick_hi, k, k - 1)
    mag = np.where(a >= _GRID[MAXCODE], MAXCODE, mag)
    sign = np.where((h < 0) & ~np.isnan(h), 0x8000, 0)
    return (mag | sign).astype(np.int64)


def scale(j: int, U: float) -> float:
    """S_j: 2 S_j is the power of two at or above K_j w_j max(|U|, 0.01), K = 2, 5, 11/2 for the
    rest, axis and diagonal directions."""
    w = 4 / 9 if j == 0 else (1 / 9 if j < 5 else 1 / 36)
    K = 2.0 if j == 0 else (5.0 if j < 5 else 5.5)
    u = max(abs(U), 0.01)
    return 0.5 * 2.0 ** np.ceil(np.log2(K * w * u))
