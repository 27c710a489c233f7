"""Geometric factors G^e and lumped mass B (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

§2, Eq. 9: A^e = D^T G^e D where G^e holds "the geometric factors for mapping
to and from the reference element".  The paper gives no formula; the oracle
writes out the standard definition.  At each GLL point (quadrature point) of
an element, with J_ab = d x_a / d r_b the Jacobian of the isoparametric map
from the reference cube (r, s, t) in [-1,1]^3,

    G_bc = W detJ sum_a (d r_b / d x_a) (d r_c / d x_a),   W = w_i w_j w_k,

so that the element stiffness is the GLL quadrature of grad(u).grad(v).  The
six independent entries are returned in the order G11, G22, G33, G12, G13,
G23, and B = W detJ is the diagonal lumped mass.
"""
import numpy as np

from .gll import gll_nodes_weights, deriv_matrix


def ref_gradient(f, D):
    """Reference-cube derivatives (df/dr, df/ds, df/dt) of a local field.

    f has shape (E,p,p,p) indexed [e,k,j,i]; r varies with i, s with j, t with k.
    """
    fr = np.einsum('il,ekjl->ekji', D, f)
    fs = np.einsum('jl,ekli->ekji', D, f)
    ft = np.einsum('kl,elji->ekji', D, f)
    return fr, fs, ft


def geom_factors(x, y, z, N):
    """Return (G, B, detJ): G has shape (6, E, p, p, p), B and detJ (E, p, p, p)."""
    _, w = gll_nodes_weights(N)
    D = deriv_matrix(N)
    # J[..., a, b] = d x_a / d r_b
    J = np.stack([np.stack(ref_gradient(c, D), axis=-1) for c in (x, y, z)], axis=-2)
    detJ = np.linalg.det(J)
    if np.any(detJ <= 0.0):
        raise ValueError("element map is not orientation preserving (detJ <= 0)")
    Jinv = np.linalg.inv(J)                 # Jinv[..., b, a] = d r_b / d x_a
    M = np.einsum('...ba,...ca->...bc', Jinv, Jinv)
    W = w[None, :, None, None] * w[None, None, :, None] * w[None, None, None, :]
    scale = W * detJ
    G = np.stack([scale * M[..., 0, 0], scale * M[..., 1, 1], scale * M[..., 2, 2],
                  scale * M[..., 0, 1], scale * M[..., 0, 2], scale * M[..., 1, 2]])
    B = scale.copy()
    return G, B, detJ
