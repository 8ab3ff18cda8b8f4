"""The integer index forms the CUDA kernels use, checked against the rounding they stand for.

Eq. 1 reads harmonic i of H at output bin n from bin round-half-up(n i / H), and its 2-D form reads
row round-half-up(z i / H), both functions of the reduced fraction p/q = i/H only.  The kernels
evaluate them without division:

* bin:  umulhi(n, F) + (low word of n F) >> 31, F = ceil(2^32 p / q), exact for n < 2^26; the next
  bin n + 1 reads one further exactly when the low word of n F + 2^31 carries on adding F, which the
  pair kernels test as the signed compare (int) lo > (int)(~F ^ 2^31).
* row:  umulhi(2 z p + 65537 q, ceil(2^32 / 2q)) - 32768, exact for |z| <= 32767.

These tests restate those forms in numpy and compare them with floor((2 n p + q) / 2q) over the
whole drift range and over boundary and random bins up to 2^26.
"""
from fractions import Fraction

import numpy as np

M32 = (1 << 32) - 1


def _farey(order):
    return sorted({Fraction(p, q) for q in range(1, order + 1) for p in range(1, q + 1)})


def test_farey_sequence_sizes():
    assert len(_farey(32)) == 324 and len(_farey(16)) == 80


def test_eq1_bin_index_and_pair_carry_exact():
    rng = np.random.default_rng(0)
    n = np.concatenate([np.arange(0, 70000), rng.integers(0, 1 << 26, 300000), np.arange((1 << 26) - 70000, 1 << 26)])
    n = n.astype(np.uint64)
    for f in _farey(32):
        p, q = f.numerator, f.denominator
        if q == 1:
            continue
        F = ((p << 32) + q - 1) // q
        prod = n * np.uint64(F)
        lo, hi = prod & np.uint64(M32), prod >> np.uint64(32)
        k = hi + (lo >> np.uint64(31))
        exact = (np.uint64(2 * p) * n + np.uint64(q)) // np.uint64(2 * q)
        np.testing.assert_array_equal(k, exact, err_msg=str(f))
        bound = np.int64(np.uint32((M32 ^ F) ^ 0x80000000).view(np.int32))
        carry = lo.astype(np.uint32).view(np.int32).astype(np.int64) > bound
        exact1 = (np.uint64(2 * p) * (n + np.uint64(1)) + np.uint64(q)) // np.uint64(2 * q)
        np.testing.assert_array_equal(k + carry.astype(np.uint64), exact1, err_msg=str(f))


def test_2d_row_index_exact_over_the_drift_range():
    z = np.arange(-32767, 32768, dtype=np.int64)
    for f in _farey(16):
        p, q = f.numerator, f.denominator
        a = z * (2 * p) + 65537 * q
        assert (a > 0).all() and (a < (1 << 21)).all()
        R = ((1 << 32) + 2 * q - 1) // (2 * q)
        row = ((a.astype(np.uint64) * np.uint64(R)) >> np.uint64(32)).astype(np.int64) - 32768
        np.testing.assert_array_equal(row, np.floor_divide(2 * z * p + q, 2 * q), err_msg=str(f))
        # rows stay between 0 and z, so every row read exists when the z range holds 0
        assert (np.minimum(z, 0) <= row).all() and (row <= np.maximum(z, 0)).all()
