"""The extended-precision reference of the symmetric product, pinned by exact
rational arithmetic and by what symmetry fixes."""
from fractions import Fraction

import numpy as np

from oracle import products


def test_mirrors_the_lower_triangle():
    A = np.array([[1.0, 9.0, 9.0], [2.0, 3.0, 9.0], [4.0, 5.0, 6.0]])
    S = products.symm_lower(A)
    assert np.array_equal(S, [[1, 2, 4], [2, 3, 5], [4, 5, 6]])
    assert np.array_equal(products.symm_product(A, np.eye(3)).astype(np.float64), S)


def test_matches_exact_rational_product():
    rng = np.random.default_rng(3)
    n, k = 24, 3
    A = rng.standard_normal((n, n)) * 2.0 ** rng.integers(-40, 40, (n, n))
    X = rng.standard_normal((n, k))
    S = products.symm_lower(A)
    got = products.symm_product(A, X)
    for i in range(n):
        for r in range(k):
            exact = sum(Fraction(S[i, j]) * Fraction(X[j, r]) for j in range(n))
            mag = sum(abs(Fraction(S[i, j]) * Fraction(X[j, r])) for j in range(n))
            # extended precision: well below one FP64 rounding of the magnitude
            assert abs(Fraction(float(got[i, r])) - exact) <= mag * Fraction(1, 2 ** 55) + Fraction(
                abs(float(got[i, r]))) * Fraction(1, 2 ** 52)


def test_symmetric_input_gives_the_plain_product():
    rng = np.random.default_rng(4)
    M = rng.integers(-4, 5, (10, 10)).astype(np.float64)
    A = M + M.T
    X = rng.integers(-4, 5, (10, 2)).astype(np.float64)
    assert np.array_equal(products.symm_product(A, X).astype(np.float64), A @ X)
