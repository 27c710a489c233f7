"""Brute-force dense element matrices and assembly for tiny meshes (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

§2, Eq. 3 and Eq. 9: A_ij = a(phi_j, phi_i) = integral of grad(phi_j).grad(phi_i),
evaluated with GLL quadrature.  This module builds every element matrix
entry by entry from explicit basis gradients -- the 1D derivative matrix
comes from the barycentric formula (not from the Legendre closed form used by
``gll.deriv_matrix``), the reference gradients from Kronecker products, and
the physical gradients from a 3x3 inverse Jacobian at each quadrature point
-- and assembles the global matrix with the global numbering.  It therefore
checks the sum-factorised apply and the geometric-factor definition by a
different route.  Cost grows as (N+1)^9 per element: tiny meshes only.
"""
import numpy as np

from .gll import gll_nodes_weights


def barycentric_deriv(xi):
    """D[i, j] = l_j'(xi_i) from barycentric weights lam_j = 1/prod_{k!=j}(xi_j - xi_k):
    D[i,j] = (lam_j / lam_i) / (xi_i - xi_j) for i != j, rows summing to zero."""
    n = len(xi)
    lam = np.array([1.0 / np.prod([xi[j] - xi[k] for k in range(n) if k != j])
                    for j in range(n)])
    D = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            if i != j:
                D[i, j] = (lam[j] / lam[i]) / (xi[i] - xi[j])
        D[i, i] = -np.sum(D[i, :])
    return D


def reference_gradient_matrices(N):
    """Dense (p^3 x p^3) matrices mapping nodal values to d/dr, d/ds, d/dt at the
    nodes, for local index i + p j + p^2 k (i fastest)."""
    xi, _ = gll_nodes_weights(N)
    D1 = barycentric_deriv(xi)
    I = np.eye(N + 1)
    Dr = np.kron(I, np.kron(I, D1))
    Ds = np.kron(I, np.kron(D1, I))
    Dt = np.kron(D1, np.kron(I, I))
    return Dr, Ds, Dt


def element_matrices(x, y, z, N):
    """Per-element stiffness K^e (p^3 x p^3) and diagonal mass m^e (p^3) from
    quadrature of explicit basis gradients.  x, y, z: (E,p,p,p)."""
    _, w = gll_nodes_weights(N)
    p = N + 1
    n = p ** 3
    Dr, Ds, Dt = reference_gradient_matrices(N)
    W = np.einsum('k,j,i->kji', w, w, w).ravel()
    E = x.shape[0]
    K = np.zeros((E, n, n))
    M = np.zeros((E, n))
    for e in range(E):
        X = np.stack([x[e].ravel(), y[e].ravel(), z[e].ravel()])   # (3, n)
        for q in range(n):
            J = np.array([[Dr[q] @ X[a], Ds[q] @ X[a], Dt[q] @ X[a]] for a in range(3)])
            detJ = np.linalg.det(J)
            JinvT = np.linalg.inv(J).T
            ref = np.stack([Dr[q], Ds[q], Dt[q]])       # (3, n): reference grads of all basis fns
            phys = JinvT @ ref                           # (3, n)
            K[e] += W[q] * detJ * (phys.T @ phys)
            M[e, q] = W[q] * detJ
    return K, M


def assemble(K, M, gid):
    """Global stiffness and mass from element matrices and the global numbering."""
    E = K.shape[0]
    g = gid.reshape(E, -1)
    ng = int(gid.max()) + 1
    A = np.zeros((ng, ng))
    Mg = np.zeros(ng)
    for e in range(E):
        A[np.ix_(g[e], g[e])] += K[e]
        np.add.at(Mg, g[e], M[e])
    return A, Mg
