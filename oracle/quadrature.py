"""1D point sets and Lagrange bases (Sec. 2.1, Eq. iproduct; Fig. 1 point sets;
Table 1 Lagrange-GLL basis).

* Gauss-Legendre: the Q roots of P_Q, weights 2 / ((1 - x^2) P_Q'(x)^2).
  Integrates polynomials of degree 2Q-1 exactly.
* Gauss-Lobatto-Legendre: +-1 and the roots of P_{N-1}', weights
  2 / (N (N-1) P_{N-1}(x)^2).  Integrates degree 2N-3 exactly.
* Lagrange cardinal functions on a node set, by the product formula.

Plain Newton iteration on the Legendre three-term recurrence; FP64 throughout.
"""
from __future__ import annotations

import numpy as np


def legendre(n: int, x):
    """P_n(x) and P_n'(x) by the three-term recurrence (valid at x = +-1)."""
    x = np.asarray(x, dtype=np.float64)
    p_prev = np.ones_like(x)
    dp_prev = np.zeros_like(x)
    if n == 0:
        return p_prev, dp_prev
    p = x.copy()
    dp = np.ones_like(x)
    for k in range(2, n + 1):
        p_next = ((2 * k - 1) * x * p - (k - 1) * p_prev) / k
        dp_next = ((2 * k - 1) * (p + x * dp) - (k - 1) * dp_prev) / k
        p_prev, p = p, p_next
        dp_prev, dp = dp, dp_next
    return p, dp


def gauss_legendre(q: int):
    """Q-point Gauss-Legendre rule on [-1, 1], nodes ascending."""
    if q < 1:
        raise ValueError("q >= 1")
    i = np.arange(q)
    x = -np.cos(np.pi * (i + 0.75) / (q + 0.5))
    for _ in range(100):
        p, dp = legendre(q, x)
        dx = p / dp
        x = x - dx
        if np.max(np.abs(dx)) < 1e-16:
            break
    _, dp = legendre(q, x)
    w = 2.0 / ((1.0 - x * x) * dp * dp)
    return x, w


def gauss_lobatto(n: int):
    """N-point Gauss-Lobatto-Legendre rule on [-1, 1] (N >= 2), nodes ascending."""
    if n < 2:
        raise ValueError("n >= 2")
    m = n - 1
    x = -np.cos(np.pi * np.arange(n) / m)
    inner = x[1:-1].copy()
    for _ in range(100):
        if inner.size == 0:
            break
        p, dp = legendre(m, inner)
        # P_m'' from Legendre's equation (1 - x^2) P'' - 2 x P' + m (m+1) P = 0
        d2p = (2.0 * inner * dp - m * (m + 1) * p) / (1.0 - inner * inner)
        dx = dp / d2p
        inner = inner - dx
        if np.max(np.abs(dx)) < 1e-16:
            break
    x = np.concatenate([[-1.0], inner, [1.0]])
    p, _ = legendre(m, x)
    w = 2.0 / (n * m * p * p)
    return x, w


def lagrange_matrix(nodes, pts):
    """L[p, j] = l_j(pts[p]) for the cardinal functions of ``nodes``."""
    nodes = np.asarray(nodes, dtype=np.float64)
    pts = np.atleast_1d(np.asarray(pts, dtype=np.float64))
    n = nodes.size
    out = np.ones((pts.size, n))
    for j in range(n):
        for m in range(n):
            if m != j:
                out[:, j] *= (pts - nodes[m]) / (nodes[j] - nodes[m])
    return out


def lagrange_deriv_matrix(nodes, pts):
    """D[p, j] = l_j'(pts[p]) (product rule over the factors of l_j)."""
    nodes = np.asarray(nodes, dtype=np.float64)
    pts = np.atleast_1d(np.asarray(pts, dtype=np.float64))
    n = nodes.size
    out = np.zeros((pts.size, n))
    for j in range(n):
        for k in range(n):
            if k == j:
                continue
            term = np.full(pts.size, 1.0 / (nodes[j] - nodes[k]))
            for m in range(n):
                if m != j and m != k:
                    term *= (pts - nodes[m]) / (nodes[j] - nodes[m])
            out[:, j] += term
    return out
