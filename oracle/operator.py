"""Matrix-free element operator and gather-scatter (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

§2, Eq. 9-10: the unassembled stiffness A_L = diag{A^1..A^E} with
A^e = D^T G^e D is applied element by element in sum-factorised form, and
continuity is restored by the gather-scatter QQ^T (w_L = QQ^T A_L u_L).
Helmholtz operators add the lumped mass: H_L = h1 A_L + h2 B_L, where a
variable h1 multiplies G at every GLL point.
"""
import numpy as np

from .geometry import ref_gradient


def ax_local(u, G, D, h1=1.0, h2=0.0, B=None, h1_field=None):
    """w_L = (h1 A_L + h2 B_L) u_L, element by element (§2, Eq. 9).

    u: (E,p,p,p); G: (6,E,p,p,p) in the order G11,G22,G33,G12,G13,G23;
    h1_field, if given, is a per-local-point coefficient that replaces h1.
    """
    ur, us, ut = ref_gradient(u, D)
    G11, G22, G33, G12, G13, G23 = G
    c = h1 if h1_field is None else h1_field
    wr = c * (G11 * ur + G12 * us + G13 * ut)
    ws = c * (G12 * ur + G22 * us + G23 * ut)
    wt = c * (G13 * ur + G23 * us + G33 * ut)
    # transposed contractions: w(i,j,k) = sum_l D_li wr(l,j,k) + D_lj ws(i,l,k) + D_lk wt(i,j,l)
    w = (np.einsum('li,ekjl->ekji', D, wr)
         + np.einsum('lj,ekli->ekji', D, ws)
         + np.einsum('lk,elji->ekji', D, wt))
    if h2 != 0.0:
        w = w + h2 * B * u
    return w


def dssum(w, gid):
    """QQ^T w_L: every local copy receives the sum over all copies that share
    its global number (§2, Eq. 10; §3.2).  The per-global-point sum runs in
    increasing local index (``np.bincount`` accumulates in input order)."""
    s = np.bincount(gid.ravel(), weights=w.ravel())
    return s[gid]


def apply_dirichlet(w, mask):
    """Zero the Dirichlet points (§2, Eq. 5: u = 0 on the boundary)."""
    return w * mask


def matvec(u, G, D, gid, mask, h1=1.0, h2=0.0, B=None, h1_field=None):
    """mask o QQ^T H_L u: the assembled, masked operator on L-vectors."""
    return apply_dirichlet(dssum(ax_local(u, G, D, h1, h2, B, h1_field), gid), mask)


def weighted_dot(a, b, mult):
    """<a, b> = sum_L a b / mult: for continuous L-vectors this counts every
    global degree of freedom once (the inner product on the unique space)."""
    return float(np.sum(a * b / mult))
