"""Pins for the oracle's 1D ingredients: Gauss-Legendre rule and Lagrange basis (Eq. 7).

Each check is against mathematics the paper fixes (Sec. II.B: collocated
Gauss-Legendre quadrature, Lagrange basis on N = p+1 nodes), never against the
oracle's own formula retyped.
"""
import math

import numpy as np
import pytest

import oracle

NS = list(range(1, 10))


@pytest.mark.parametrize("N", NS)
def test_gl_moments_exact(N):
    # an N-point Gauss rule integrates x^m exactly for m <= 2N-1
    xi, w = oracle.gl_nodes(N)
    for m in range(2 * N):
        exact = 0.0 if m % 2 else 2.0 / (m + 1)
        assert abs(np.dot(w, xi ** m) - exact) < 1e-14


@pytest.mark.parametrize("N", NS)
def test_gl_matches_library_rule(N):
    # numpy's Golub-Welsch based leggauss is an independent computation of the same rule
    xr, wr = np.polynomial.legendre.leggauss(N)
    xi, w = oracle.gl_nodes(N)
    assert np.max(np.abs(xi - xr)) < 1e-14
    assert np.max(np.abs(w - wr)) < 1e-14
    # nodes are the roots of P_N
    c = np.zeros(N + 1)
    c[N] = 1.0
    assert np.max(np.abs(np.polynomial.legendre.legval(xi, c))) < 1e-13


def test_gl_closed_forms():
    xi, w = oracle.gl_nodes(1)
    assert xi[0] == 0.0 and w[0] == 2.0
    xi, w = oracle.gl_nodes(2)
    assert abs(xi[1] - 1 / math.sqrt(3)) < 3e-16 and abs(xi[0] + 1 / math.sqrt(3)) < 3e-16
    assert abs(w[0] - 1) < 1e-15 and abs(w[1] - 1) < 1e-15
    xi, w = oracle.gl_nodes(3)
    assert abs(xi[2] - math.sqrt(0.6)) < 1e-15 and abs(xi[1]) < 1e-16
    assert abs(w[1] - 8 / 9) < 1e-15 and abs(w[0] - 5 / 9) < 1e-15


@pytest.mark.parametrize("N", NS)
def test_lagrange_cardinal_and_exactness(N):
    xi, _ = oracle.gl_nodes(N)
    # cardinal property l_s(xi_a) = delta_sa
    for s in range(N):
        for a in range(N):
            assert abs(oracle.lagrange(N, xi, s, xi[a]) - (1.0 if s == a else 0.0)) < 1e-14
    # reproduces polynomials of degree <= p at arbitrary points, and their derivatives
    for x in (-1.0, -0.3, 0.77, 1.0):
        for m in range(N):
            v = sum(oracle.lagrange(N, xi, s, x) * xi[s] ** m for s in range(N))
            d = sum(oracle.lagrange_deriv(N, xi, s, x) * xi[s] ** m for s in range(N))
            assert abs(v - x ** m) < 1e-12
            assert abs(d - (m * x ** (m - 1) if m else 0.0)) < 1e-10


@pytest.mark.parametrize("N", NS)
def test_sbp_identity(N):
    # summation by parts with a Gauss rule: W D + D^T W = l(+1) l(+1)^T - l(-1) l(-1)^T,
    # D[a, s] = l_s'(xi_a), W = diag(w).  Exact because l_s l_r' has degree 2N-2 <= 2N-1.
    xi, w = oracle.gl_nodes(N)
    D = np.array([[oracle.lagrange_deriv(N, xi, s, xi[a]) for s in range(N)] for a in range(N)])
    lp = np.array([oracle.lagrange(N, xi, s, 1.0) for s in range(N)])
    lm = np.array([oracle.lagrange(N, xi, s, -1.0) for s in range(N)])
    W = np.diag(w)
    lhs = W @ D + D.T @ W
    rhs = np.outer(lp, lp) - np.outer(lm, lm)
    assert np.max(np.abs(lhs - rhs)) < 1e-12 * max(1.0, np.max(np.abs(D)))
    # partition of unity at the end points and zero row sums of D
    assert abs(lp.sum() - 1) < 1e-13 and abs(lm.sum() - 1) < 1e-13
    assert np.max(np.abs(D.sum(axis=1))) < 1e-11
