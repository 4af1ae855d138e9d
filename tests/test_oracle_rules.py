"""Pins of the oracle's 1D rules against closed forms (no GPU).

The paper (Sec. 3.2) fixes an LGL nodal Lagrange basis and Gauss quadrature;
these tests pin the oracle's implementation of both against textbook facts:
exactness degrees, closed-form LGL nodes, Legendre recurrences and cardinality.
"""
import json
import os

import numpy as np
import pytest

from oracle import rules

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def legendre_and_derivative(k, x):
    """Bonnet recurrence (textbook), independent of numpy.polynomial."""
    p0, p1 = np.ones_like(x), x.copy()
    if k == 0:
        return p0, np.zeros_like(x)
    for n in range(1, k):
        p0, p1 = p1, ((2 * n + 1) * x * p1 - n * p0) / (n + 1)
    # (1 - x^2) P_k' = k (P_{k-1} - x P_k) inside; P_k'(+-1) = (+-1)^(k+1) k (k+1) / 2
    dp = np.empty_like(x)
    inner = np.abs(x) < 1.0
    dp[inner] = k * (p0[inner] - x[inner] * p1[inner]) / (1.0 - x[inner] ** 2)
    dp[~inner] = np.sign(x[~inner]) ** (k + 1) * k * (k + 1) / 2.0
    return p1, dp


@pytest.mark.parametrize("n", range(1, 19))
def test_gauss_exactness(n):
    x, w = rules.gauss(n)
    assert abs(w.sum() - 1.0) < 1e-14
    for m in range(2 * n):
        assert abs(np.dot(w, x ** m) - 1.0 / (m + 1)) < 2e-15 * (m + 1)
    # degree 2n is not integrated exactly: it really is an n-point rule
    # (the defect shrinks like 4^-2n, so it is visible only for small n)
    if n <= 8:
        assert abs(np.dot(w, x ** (2 * n)) - 1.0 / (2 * n + 1)) > 1e-12


def test_lgl_closed_forms():
    with open(os.path.join(GOLDEN, "lgl_nodes.json")) as f:
        gold = json.load(f)
    for k, expr in gold["nodes"].items():
        ref = np.array([eval(s, {"sqrt": np.sqrt}) for s in expr])
        assert np.max(np.abs(rules.lgl_nodes(int(k)) - ref)) < 1e-15


@pytest.mark.parametrize("k", range(1, 16))
def test_lgl_properties(k):
    x = rules.lgl_nodes(k)
    assert x[0] == 0.0 and x[-1] == 1.0
    assert np.all(np.diff(x) > 0)
    assert np.max(np.abs(x + x[::-1] - 1.0)) < 1e-15
    t = 2.0 * x[1:-1] - 1.0
    if k > 1:
        _, dp = legendre_and_derivative(k, t)
        assert np.max(np.abs(dp)) < 1e-11 * k * k
    # LGL quadrature w_j = 2 / (k (k+1) P_k(t_j)^2) on [-1, 1] is exact to 2k-1
    pk, _ = legendre_and_derivative(k, 2.0 * x - 1.0)
    w = 1.0 / (k * (k + 1) * pk ** 2)
    for m in range(2 * k):
        assert abs(np.dot(w, x ** m) - 1.0 / (m + 1)) < 1e-14


@pytest.mark.parametrize("k", [1, 2, 3, 5, 8, 11])
def test_lagrange_basis(k):
    x = rules.lgl_nodes(k)
    V, D = rules.lagrange(x, x)
    assert np.max(np.abs(V - np.eye(k + 1))) < 1e-14
    t = np.linspace(-0.3, 1.3, 37)
    V, D = rules.lagrange(x, t)
    assert np.max(np.abs(V.sum(1) - 1.0)) < 1e-11
    assert np.max(np.abs(D.sum(1))) < 1e-9
    # reproduction of a polynomial of degree k and of its derivative
    c = np.random.default_rng(k).uniform(-1, 1, k + 1)
    p = np.polynomial.Polynomial(c)
    assert np.max(np.abs(V @ p(x) - p(t))) < 1e-11
    assert np.max(np.abs(D @ p(x) - p.deriv()(t))) < 1e-9
