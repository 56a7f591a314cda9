"""Pins of the oracle's 1D point sets and Lagrange tables (Sec. 2.1, Eq. iproduct).

Against: numpy's Gauss-Legendre rule (a library routine), textbook closed
forms (tests/golden/quadrature_closed_forms.json), and polynomial exactness.
"""
import json
import os
from math import sqrt

import numpy as np
import pytest

from oracle.quadrature import gauss_legendre, gauss_lobatto, lagrange_matrix, lagrange_deriv_matrix

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "quadrature_closed_forms.json")


def _ev(s):
    return float(eval(s, {"sqrt": sqrt}))


@pytest.mark.parametrize("q", range(1, 13))
def test_gauss_matches_library(q):
    x, w = gauss_legendre(q)
    xl, wl = np.polynomial.legendre.leggauss(q)
    assert np.allclose(x, xl, rtol=0, atol=2e-15)
    assert np.allclose(w, wl, rtol=0, atol=2e-15)


def test_closed_forms():
    g = json.load(open(GOLDEN))
    for q, d in g["gauss"].items():
        x, w = gauss_legendre(int(q))
        assert np.allclose(x, [_ev(s) for s in d["x"]], atol=1e-15)
        assert np.allclose(w, [_ev(s) for s in d["w"]], atol=1e-15)
    for n, d in g["lobatto"].items():
        x, w = gauss_lobatto(int(n))
        assert np.allclose(x, [_ev(s) for s in d["x"]], atol=1e-15)
        assert np.allclose(w, [_ev(s) for s in d["w"]], atol=1e-15)


def _mono_integral(k):
    return 0.0 if k % 2 else 2.0 / (k + 1)


@pytest.mark.parametrize("q", range(1, 12))
def test_gauss_exactness(q):
    x, w = gauss_legendre(q)
    for k in range(2 * q):
        assert abs(np.sum(w * x ** k) - _mono_integral(k)) < 1e-14
    assert abs(np.sum(w * x ** (2 * q)) - _mono_integral(2 * q)) > 1e-8


@pytest.mark.parametrize("n", range(2, 12))
def test_lobatto_exactness(n):
    x, w = gauss_lobatto(n)
    assert x[0] == -1.0 and x[-1] == 1.0
    for k in range(2 * n - 2):
        assert abs(np.sum(w * x ** k) - _mono_integral(k)) < 1e-14
    k = 2 * n - 2
    assert abs(np.sum(w * x ** k) - _mono_integral(k)) > 1e-6


@pytest.mark.parametrize("n", range(2, 11))
def test_lagrange_interpolation_and_derivative(n):
    nodes, _ = gauss_lobatto(n)
    pts = np.linspace(-1, 1, 17)
    L = lagrange_matrix(nodes, pts)
    D = lagrange_deriv_matrix(nodes, pts)
    assert np.allclose(lagrange_matrix(nodes, nodes), np.eye(n), atol=1e-14)
    for k in range(n):
        f = nodes ** k
        assert np.allclose(L @ f, pts ** k, atol=1e-13)
        df = k * pts ** (k - 1) if k > 0 else np.zeros_like(pts)
        assert np.allclose(D @ f, df, atol=1e-11)
    # derivative of the constant is zero: rows of D sum to 0
    assert np.allclose(D.sum(axis=1), 0.0, atol=1e-12)
    # degree n is NOT reproduced
    assert np.max(np.abs(L @ nodes ** n - pts ** n)) > 1e-6
