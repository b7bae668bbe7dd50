"""Pins for the oracle's 1D rules and bases (Sec. 2.1 GLL basis, Sec. 3.1
Gauss rule with m = p+1): closed forms and exactness, not re-derivations."""
import math

import numpy as np
import pytest

from oracle import quadrature as q


def test_gauss3_closed_form():
    x, w = q.gauss_legendre(3)
    s = math.sqrt(3.0 / 5.0)
    np.testing.assert_allclose(x, [(1 - s) / 2, 0.5, (1 + s) / 2], rtol=0, atol=1e-15)
    np.testing.assert_allclose(w, [5 / 18, 8 / 18, 5 / 18], rtol=0, atol=1e-15)


def test_gll_closed_forms():
    x, w = q.gauss_lobatto(4)            # p = 3: {+-1, +-1/sqrt(5)}
    s = 1 / math.sqrt(5.0)
    np.testing.assert_allclose(x, [0, (1 - s) / 2, (1 + s) / 2, 1], atol=1e-15)
    np.testing.assert_allclose(w, [1 / 12, 5 / 12, 5 / 12, 1 / 12], atol=1e-15)
    x, w = q.gauss_lobatto(5)            # p = 4: {0, +-sqrt(3/7), +-1}
    s = math.sqrt(3 / 7)
    np.testing.assert_allclose(x, [0, (1 - s) / 2, 0.5, (1 + s) / 2, 1], atol=1e-15)
    np.testing.assert_allclose(w, np.array([1 / 10, 49 / 90, 32 / 45, 49 / 90, 1 / 10]) / 2, atol=1e-15)
    x, w = q.gauss_lobatto(3)            # p = 2: Simpson
    np.testing.assert_allclose(x, [0, 0.5, 1], atol=1e-15)
    np.testing.assert_allclose(w, [1 / 6, 4 / 6, 1 / 6], atol=1e-15)


@pytest.mark.parametrize("m", range(1, 10))
def test_gauss_exactness(m):
    x, w = q.gauss_legendre(m)
    assert abs(w.sum() - 1.0) < 1e-14
    for k in range(2 * m):
        assert abs(w @ x ** k - 1.0 / (k + 1)) < 1e-14
    assert abs(w @ x ** (2 * m) - 1.0 / (2 * m + 1)) > 1e-13   # degree 2m is not exact


@pytest.mark.parametrize("n", range(2, 10))
def test_gll_exactness_and_nodal_basis(n):
    x, w = q.gauss_lobatto(n)
    for k in range(2 * n - 2):
        assert abs(w @ x ** k - 1.0 / (k + 1)) < 1e-14
    V = q.lagrange_values(x, x)
    np.testing.assert_allclose(V, np.eye(n), atol=1e-14)
    t = np.linspace(0, 1, 17)
    D = q.lagrange_derivatives(x, t)
    # D 1 = 0, and D x^k = k x^(k-1) for k <= p
    np.testing.assert_allclose(D.sum(axis=1), 0.0, atol=1e-11)
    for k in range(1, n):
        np.testing.assert_allclose(D @ x ** k, k * t ** (k - 1), atol=1e-10)
    # values reproduce polynomials of degree <= p
    Vt = q.lagrange_values(x, t)
    for k in range(n):
        np.testing.assert_allclose(Vt @ x ** k, t ** k, atol=1e-12)
