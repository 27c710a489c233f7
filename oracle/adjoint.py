"""Gradient of a loss with respect to a per-point diffusion coefficient (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The operator H(h1) = D^T (h1 G) D + h2 B (§2, Eq. 9 with the coefficient
h1 multiplying G at every GLL point) is linear in each local value h1_p, and
d(v^T H u)/d h1_p = (D^ v)_p^T G_p (D^ u)_p, with D^ the reference gradient
(d/dr, d/ds, d/dt) at local point p.  For u = H^{-1} b and a loss L(u), the
adjoint lambda solves H lambda = mask o QQ^T (dL/du_L) and
dL/dh1_p = -(D^ lambda)_p^T G_p (D^ u)_p.
"""
import numpy as np

from .geometry import ref_gradient


def grad_h1(u, lam, G, D):
    """-(D^ lam)^T G (D^ u) at every local point, shape (E,p,p,p)."""
    ur, us, ut = ref_gradient(u, D)
    lr, ls, lt = ref_gradient(lam, D)
    G11, G22, G33, G12, G13, G23 = G
    gu_r = G11 * ur + G12 * us + G13 * ut
    gu_s = G12 * ur + G22 * us + G23 * ut
    gu_t = G13 * ur + G23 * us + G33 * ut
    return -(lr * gu_r + ls * gu_s + lt * gu_t)


def loss(u, u_target, mult):
    """L = ||u - u_target||^2 in the unique-dof norm (each global point once)."""
    d = u - u_target
    return float(np.sum(d * d / mult))


def loss_grad_u(u, u_target, mult):
    """dL/du_L for the loss above, taken per local entry (2 (u-u_t) / mult)."""
    return 2.0 * (u - u_target) / mult
