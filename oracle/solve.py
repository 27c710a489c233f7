"""Jacobi-preconditioned CG on the matrix-free operator (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

§2 (end): with a matrix-free product w_L = QQ^T A_L u_L, a matrix-free Krylov
method completes the SEM solver; §4 solves the velocity Helmholtz systems by
preconditioned CG.  The paper does not print the CG recurrences, the
preconditioner's formula, the right-hand side's discrete form or the stopping
rule; the oracle takes these readings:

* b_L = mask o QQ^T (B f)  (GLL-lumped mass times the nodal source);
* the preconditioner is point Jacobi: dinv = mask / QQ^T diag(H_L);
* x0 = 0, r = b, z = dinv r, p = z; each iteration
  w = mask o QQ^T H_L p, alpha = <r,z>/<p,w>, x += alpha p, r -= alpha w,
  stop when sqrt(<r,r>) <= tol sqrt(<b,b>), beta = <r_new,z_new>/<r,z>,
  p = z + beta p;
* <a,b> = sum_L a b / mult (the unique-dof inner product);
* <p,w> <= 0 is a breakdown; hitting maxit is non-convergence.
"""
import numpy as np

from .operator import ax_local, dssum, apply_dirichlet, weighted_dot


def rhs(f, B, gid, mask):
    """b_L = mask o QQ^T (B f) for a nodal source f."""
    return apply_dirichlet(dssum(B * f, gid), mask)


def local_diagonal(G, D, h1=1.0, h2=0.0, B=None, h1_field=None):
    """diag(H^e) at every local point, from A^e = D^T G D written out for a
    single basis function: the rr, ss and tt terms sum over the line through
    the point, the mixed terms only see the point itself."""
    c = h1 if h1_field is None else h1_field
    G11, G22, G33, G12, G13, G23 = (c * g for g in G)
    D2 = D * D
    dd = np.diag(D)
    p = D.shape[0]
    d = (np.einsum('li,ekjl->ekji', D2, G11)
         + np.einsum('lj,ekli->ekji', D2, G22)
         + np.einsum('lk,elji->ekji', D2, G33))
    di = dd[None, None, None, :]
    dj = dd[None, None, :, None]
    dk = dd[None, :, None, None]
    d = d + 2.0 * (di * dj * G12 + di * dk * G13 + dj * dk * G23)
    if h2 != 0.0:
        d = d + h2 * B
    assert d.shape[1:] == (p, p, p)
    return d


def jacobi_inverse(G, D, gid, mask, h1=1.0, h2=0.0, B=None, h1_field=None):
    """dinv = mask / QQ^T diag(H_L); masked points get 0."""
    dg = dssum(local_diagonal(G, D, h1, h2, B, h1_field), gid)
    out = np.zeros_like(dg)
    nz = mask != 0.0
    out[nz] = 1.0 / dg[nz]
    return out


class CGResult:
    def __init__(self, x, iters, rel_res, status, history):
        self.x = x
        self.iters = iters
        self.rel_res = rel_res
        self.status = status          # "ok", "noconv", "breakdown"
        self.history = history


def pcg(b, G, D, gid, mask, mult, h1=1.0, h2=0.0, B=None, h1_field=None,
        tol=1e-10, maxit=20000, x0=None):
    """Jacobi-PCG for mask o QQ^T H_L x = b, in the order stated above."""
    def op(v):
        return apply_dirichlet(dssum(ax_local(v, G, D, h1, h2, B, h1_field), gid), mask)

    dinv = jacobi_inverse(G, D, gid, mask, h1, h2, B, h1_field)
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b - op(x) if x0 is not None else b.copy()
    bnorm = np.sqrt(weighted_dot(b, b, mult))
    if bnorm == 0.0:
        return CGResult(x, 0, 0.0, "ok", [0.0])
    z = dinv * r
    p = z.copy()
    rz = weighted_dot(r, z, mult)
    hist = [np.sqrt(weighted_dot(r, r, mult)) / bnorm]
    if hist[0] <= tol:
        return CGResult(x, 0, hist[0], "ok", hist)
    for it in range(1, maxit + 1):
        w = op(p)
        pw = weighted_dot(p, w, mult)
        if not pw > 0.0:
            return CGResult(x, it, hist[-1], "breakdown", hist)
        alpha = rz / pw
        x = x + alpha * p
        r = r - alpha * w
        rel = np.sqrt(weighted_dot(r, r, mult)) / bnorm
        hist.append(rel)
        if rel <= tol:
            return CGResult(x, it, rel, "ok", hist)
        z = dinv * r
        rz_new = weighted_dot(r, z, mult)
        beta = rz_new / rz
        rz = rz_new
        p = z + beta * p
    return CGResult(x, maxit, hist[-1], "noconv", hist)


def residual(x, b, G, D, gid, mask, mult, h1=1.0, h2=0.0, B=None, h1_field=None):
    """Relative residual ||b - mask o QQ^T H_L x|| / ||b|| in the unique-dof norm."""
    r = b - apply_dirichlet(dssum(ax_local(x, G, D, h1, h2, B, h1_field), gid), mask)
    return np.sqrt(weighted_dot(r, r, mult)) / np.sqrt(weighted_dot(b, b, mult))
