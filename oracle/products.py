"""Reference for the symmetric product Y = A X with A given by its lower
triangle (the product inside the refinement residual R = B - A X): the
definition written out, the strict lower triangle mirrored into the upper
one, and the product taken in numpy's extended precision (np.longdouble,
64-bit significand on x86), so that its own rounding is far below FP64's.
Test infrastructure: only the tests, the smoke check and the benchmark's CPU
baseline use this package.
"""
import numpy as np


def symm_lower(A):
    """The full symmetric matrix whose lower triangle is that of A."""
    L = np.tril(A)
    return L + np.tril(A, -1).T


def symm_product(A, X):
    """A X for symmetric A read from its lower triangle, in extended precision
    (returned as np.longdouble)."""
    S = symm_lower(np.asarray(A, dtype=np.float64)).astype(np.longdouble)
    return S @ np.asarray(X, dtype=np.float64).astype(np.longdouble)
