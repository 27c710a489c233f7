"""Projection onto previous solutions for successive right-hand sides (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

§4 and Table 2: Neko accelerates its pressure solves by keeping a space of
previous solutions (20 vectors) and starting each solve from the projection
onto it, after Nek5000; the paper gives no formulas.  Reading (the standard
form of the technique):

* the space is X = [x_1 .. x_l], kept H-orthonormal, <x_i, H x_j> = delta_ij
  in the unique-dof inner product, together with W = H X;
* for a new b: alpha_i = <x_i, b>, x_bar = X alpha (the best approximation of
  the solution in span X in the H-norm), r = b - W alpha;
* PCG solves H d = r from d = 0 to ||b - H(x_bar + d)|| <= tol ||b||, and
  x = x_bar + d;
* d is added to the space: w = H d, Gram-Schmidt in the H inner product
  (c_i = <x_i, w>, d -= X c, w -= W c), applied twice, then d and w are
  scaled by 1 / sqrt(<d, w>); a d whose remaining H-norm is below 1e-10 of
  the original is dropped;
* when the space holds m vectors it restarts from the latest solution alone
  (x and H x = W alpha + w, normalised).
"""
import numpy as np

from . import operator, solve


class Projection:
    """Space of at most m H-orthonormal previous solutions (L-vectors)."""

    def __init__(self, m):
        self.m = m
        self.X = []
        self.W = []

    def project(self, b, mult):
        """(x_bar, r, alpha) for right-hand side b."""
        alpha = [operator.weighted_dot(x, b, mult) for x in self.X]
        x_bar = np.zeros_like(b)
        r = b.copy()
        for a, x, w in zip(alpha, self.X, self.W):
            x_bar = x_bar + a * x
            r = r - a * w
        return x_bar, r, alpha

    def _orthonormal_add(self, d, w, mult):
        d0 = operator.weighted_dot(d, w, mult)
        for _ in range(2):
            c = [operator.weighted_dot(x, w, mult) for x in self.X]
            for ci, x, wx in zip(c, self.X, self.W):
                d = d - ci * x
                w = w - ci * wx
        nrm2 = operator.weighted_dot(d, w, mult)
        if not (nrm2 > 1e-20 * abs(d0)) or nrm2 <= 0.0:
            return False
        s = 1.0 / np.sqrt(nrm2)
        self.X.append(d * s)
        self.W.append(w * s)
        return True

    def update(self, x, hx, d, hd, mult):
        """Add the correction d (H d = hd) of the solve whose solution is x
        (H x = hx); restart from x alone when the space is full."""
        if self.m <= 0:
            return
        if len(self.X) >= self.m:
            self.X, self.W = [], []
            self._orthonormal_add(x, hx, mult)
        else:
            self._orthonormal_add(d, hd, mult)


def solve_projected(proj, b, matvec, pcg, mult, tol):
    """x for H x = b with the projection space proj (updated in place).

    matvec(v) = mask QQ^T H_L v; pcg(rhs, tol) -> CGResult.  Returns
    (x, x_bar, result of the correction solve)."""
    bnorm = np.sqrt(operator.weighted_dot(b, b, mult))
    x_bar, r, alpha = proj.project(b, mult)
    rnorm = np.sqrt(operator.weighted_dot(r, r, mult))
    if bnorm == 0.0 or rnorm <= tol * bnorm:
        d = np.zeros_like(b)
        res = solve.CGResult(d, 0, 0.0, "ok", [])
    else:
        res = pcg(r, tol * bnorm / rnorm)
        d = res.x
    x = x_bar + d
    hd = matvec(d)
    hx = b - r + hd                      # H x = W alpha + H d
    proj.update(x, hx, d, hd, mult)
    return x, x_bar, res
