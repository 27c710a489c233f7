"""GLL nodes, quadrature weights and the nodal derivative matrix (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

§2, Eq. 7-8: the element basis is the tensor product of the degree-N
Lagrange polynomials l_i on the N+1 Gauss-Lobatto-Legendre points.  The
printed Eq. 7 is garbled (its factor N(N+1) sits in the numerator and L'_N
is evaluated at xi_i); this oracle takes the reading that l_i is the unique
degree-N polynomial with l_i(xi_j) = delta_ij on the GLL nodes.
"""
import numpy as np
from numpy.polynomial import legendre as npleg


def legendre(N, x):
    """L_N(x), the Legendre polynomial of degree N (library evaluation)."""
    c = np.zeros(N + 1)
    c[N] = 1.0
    return npleg.legval(x, c)


def gll_nodes_weights(N):
    """GLL nodes xi_0 < ... < xi_N on [-1, 1] and their quadrature weights.

    The nodes are -1, +1 and the N-1 roots of L'_N (§2, "Gauss-Lobatto-
    Legendre (GLL) quadrature points"); the weights are
    w_i = 2 / (N (N+1) L_N(xi_i)^2).
    """
    if N < 1:
        raise ValueError("N must be >= 1")
    c = np.zeros(N + 1)
    c[N] = 1.0
    dc = npleg.legder(c)          # coefficients of L'_N
    d2c = npleg.legder(dc)        # coefficients of L''_N
    interior = np.sort(np.real(npleg.legroots(dc))) if N > 1 else np.zeros(0)
    # polish the interior roots with Newton on L'_N
    for _ in range(3):
        if N > 1:
            interior = interior - npleg.legval(interior, dc) / npleg.legval(interior, d2c)
    xi = np.concatenate(([-1.0], interior, [1.0]))
    w = 2.0 / (N * (N + 1) * legendre(N, xi) ** 2)
    return xi, w


def deriv_matrix(N):
    """D[i, j] = l_j'(xi_i): derivative at node i of the j-th GLL Lagrange
    polynomial (§2, Eq. 9, "the local derivatives of the operand at the GLL
    points").  Written from the closed form of l_j' at the GLL nodes:
    off-diagonal L_N(xi_i) / (L_N(xi_j) (xi_i - xi_j)); D[0,0] = -N(N+1)/4;
    D[N,N] = +N(N+1)/4; every other diagonal entry 0.
    """
    xi, _ = gll_nodes_weights(N)
    LN = legendre(N, xi)
    p = N + 1
    D = np.zeros((p, p))
    for i in range(p):
        for j in range(p):
            if i != j:
                D[i, j] = LN[i] / (LN[j] * (xi[i] - xi[j]))
    D[0, 0] = -N * (N + 1) / 4.0
    D[N, N] = N * (N + 1) / 4.0
    return D
