"""Pins for the oracle's GLL nodes, weights and derivative matrix (§2, Eq. 7-9)."""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle.gll import gll_nodes_weights, deriv_matrix, legendre
from oracle.dense import barycentric_deriv

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "gll_closed_forms.txt")


def _value(tok):
    tok = tok.strip()
    neg = tok.startswith("-")
    if neg:
        tok = tok[1:]
    if tok.startswith("sqrt(") and tok.endswith(")"):
        v = math.sqrt(float(Fraction(tok[5:-1])))
    else:
        v = float(Fraction(tok))
    return -v if neg else v


def _golden():
    table = {}
    with open(GOLDEN) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, rhs = line.split(":", 1)
            N = int(key.split()[0].split("=")[1])
            kind = key.split()[1]
            rows = [[_value(t) for t in row.split(",")] for row in rhs.split(";")]
            table[(N, kind)] = np.array(rows if kind == "D" else rows[0])
    return table


GOLD = _golden()


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_gll_closed_forms(N):
    xi, w = gll_nodes_weights(N)
    np.testing.assert_allclose(xi, GOLD[(N, "nodes")], rtol=0, atol=1e-15)
    np.testing.assert_allclose(w, GOLD[(N, "weights")], rtol=0, atol=1e-15)


@pytest.mark.parametrize("N", [1, 2])
def test_deriv_closed_forms(N):
    np.testing.assert_allclose(deriv_matrix(N), GOLD[(N, "D")], rtol=0, atol=1e-14)


@pytest.mark.parametrize("N", range(1, 13))
def test_quadrature_exact_to_2N_minus_1(N):
    xi, w = gll_nodes_weights(N)
    assert abs(w.sum() - 2.0) < 1e-14
    for k in range(0, 2 * N):
        exact = 2.0 / (k + 1) if k % 2 == 0 else 0.0
        assert abs(np.dot(w, xi ** k) - exact) < 1e-13, (N, k)
    # and not exact one degree further (even degree 2N)
    k = 2 * N
    assert abs(np.dot(w, xi ** k) - 2.0 / (k + 1)) > 1e-11


@pytest.mark.parametrize("N", range(2, 13))
def test_interior_nodes_are_roots_of_dLN(N):
    xi, _ = gll_nodes_weights(N)
    h = 1e-6
    dL = (legendre(N, xi[1:-1] + h) - legendre(N, xi[1:-1] - h)) / (2 * h)
    assert np.max(np.abs(dL)) < 1e-6 * N * N
    assert np.all(np.diff(xi) > 0)
    np.testing.assert_allclose(xi, -xi[::-1], atol=1e-15)


@pytest.mark.parametrize("N", range(1, 13))
def test_deriv_exact_on_monomials(N):
    xi, _ = gll_nodes_weights(N)
    D = deriv_matrix(N)
    np.testing.assert_allclose(D @ np.ones(N + 1), 0.0, atol=1e-12 * N * N)
    for k in range(1, N + 1):
        np.testing.assert_allclose(D @ xi ** k, k * xi ** (k - 1), atol=1e-12 * N ** 3)


@pytest.mark.parametrize("N", range(1, 13))
def test_deriv_matches_barycentric(N):
    xi, _ = gll_nodes_weights(N)
    np.testing.assert_allclose(deriv_matrix(N), barycentric_deriv(xi), atol=1e-12 * N ** 2)


@pytest.mark.parametrize("N", range(1, 11))
def test_deriv_antisymmetry(N):
    # GLL nodes are symmetric, so D[N-i, N-j] = -D[i, j]
    D = deriv_matrix(N)
    np.testing.assert_allclose(D[::-1, ::-1], -D, atol=1e-13 * N * N)
