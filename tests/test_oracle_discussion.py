"""Pin: the Discussion example of the paper's forward error analysis
(tests/golden/discussion_example.txt) on the cascade restatement."""
import os
from fractions import Fraction

import numpy as np

from oracle import cascade as cs
from tests import exact

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "discussion_example.txt")


def read_example():
    vals = {}
    for line in open(GOLDEN):
        if line.strip() and not line.startswith("#"):
            key, val = line.split()
            vals[key] = int(val) if key == "k" else float.fromhex(val)
    k, eps = vals["k"], vals["eps"]
    x = np.full(k, eps)
    x[0] = 1.0
    y = np.full(k, eps)
    y[1] = 1.0
    closed = 2 * Fraction(eps) + (k - 2) * Fraction(eps) ** 2    # the paper's 2 eps + (k-2) eps^2
    return x, y, closed


def test_discussion_example_exact_and_bin0_cancels():
    x, y, closed = read_example()
    z = np.zeros_like(x)
    c_hi, c_lo, bins, _ = cs.cascade_ddgemm(x[None, :], z[None, :], y[:, None], z[:, None],
                                            return_bins=True)
    got = Fraction(c_hi[0, 0]) + Fraction(c_lo[0, 0])
    assert got == closed
    assert bins[0][0][0, 0] == 0.0           # bin 0 cancels
    assert abs(x) @ abs(y) == float(closed)  # |x|^T |y| = x^T y here
    assert exact.dd_is_normalised(c_hi, c_lo)
