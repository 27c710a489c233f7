"""Shared test helpers: oracle problem data and GPU handles on the same mesh."""
import math

import numpy as np

from oracle import mesh, geometry, operator, solve
from oracle.gll import deriv_matrix

TWO_PI = 2 * math.pi


class OracleProblem:
    """Everything the oracle needs for one box mesh."""

    def __init__(self, nel, N, x0=(0.0, 0.0, 0.0), length=(1.0, 1.0, 1.0), deform=0.0,
                 faces=mesh.ALL_FACES):
        self.nel, self.N = tuple(nel), N
        self.x, self.y, self.z = mesh.box_coords(*nel, N, x0, length, deform)
        self.G, self.B, self.detJ = geometry.geom_factors(self.x, self.y, self.z, N)
        self.D = deriv_matrix(N)
        self.gid = mesh.global_ids(*nel, N)
        self.mult = mesh.multiplicity(self.gid)
        self.mask = mesh.dirichlet_mask(*nel, N, faces)
        self.shape = self.gid.shape

    def ax(self, u, h1=1.0, h2=0.0, h1_field=None):
        return operator.ax_local(u, self.G, self.D, h1, h2, self.B, h1_field)

    def matvec(self, u, h1=1.0, h2=0.0, h1_field=None):
        return operator.apply_dirichlet(operator.dssum(self.ax(u, h1, h2, h1_field), self.gid),
                                        self.mask)

    def rhs(self, f):
        return solve.rhs(f, self.B, self.gid, self.mask)

    def pcg(self, b, **kw):
        return solve.pcg(b, self.G, self.D, self.gid, self.mask, self.mult, B=self.B, **kw)

    def residual(self, x, b, h1=1.0, h2=0.0, h1_field=None):
        return solve.residual(x, b, self.G, self.D, self.gid, self.mask, self.mult, h1, h2,
                              self.B, h1_field)


def rel_inf(a, b):
    """||a - b||_inf / ||b||_inf."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))
