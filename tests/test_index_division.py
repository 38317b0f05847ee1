"""The generic FV stage splits cell, line and face indices with a float reciprocal instead of the
integer divide: q = trunc(fl((fl(n) + 1/2) * fl(1/d))) in IEEE single precision.  For
0 <= n < 2^15 the quotient (n + 1/2)/d is never an integer and lies at least 1/(2n + 1) (relative)
from one, while the two roundings err by at most 2^-23 (relative), so the result is floor(n/d).
This checks the claim exhaustively, in the same single-precision operations, for every divisor the
kernel can meet (d <= 1024: cells, line cells and faces per group and the box extents)."""
import numpy as np


def test_float_reciprocal_division_is_exact():
    n = np.arange(1 << 15, dtype=np.int64)
    nf = n.astype(np.float32) + np.float32(0.5)
    for d in range(1, 1025):
        r = np.float32(1.0) / np.float32(d)          # IEEE-rounded reciprocal
        q = (nf * r).astype(np.int64)                # product rounded to float, truncated
        assert np.array_equal(q, n // d), d
