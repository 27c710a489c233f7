"""One rank's compute for the partition tests on the CPU, done by the oracle:
the same interface as paper_2107_01243_gb300.partition.DeviceBackend, on
torch CPU tensors, so that the partition, the interface exchange and the
partitioned PCG of the package run unchanged on gloo ranks without a GPU."""
import numpy as np
import torch

from oracle import operator, solve
from tests.helpers import OracleProblem


class OracleBackend:
    def __init__(self, count, N, x0, length, deform, faces):
        self.o = OracleProblem(count, N, x0=x0, length=length, deform=deform, faces=faces)
        self.shape = self.o.shape
        self.n = int(np.prod(self.shape))
        self.mult = self.o.mult.astype(np.float64)

    def _a(self, v):
        return v.numpy().reshape(self.shape)

    def index(self, a):
        return torch.from_numpy(np.ascontiguousarray(a, dtype=np.int64))

    def empty(self, n):
        return torch.empty(n, dtype=torch.float64)

    def zeros(self):
        return torch.zeros(self.n, dtype=torch.float64)

    def copy(self, v):
        return v.clone()

    def fill(self, v, value):
        v.fill_(value)

    def scalars(self, values):
        return torch.tensor(values, dtype=torch.float64)

    def apply(self, u, w, h1, h2):
        w.copy_(torch.from_numpy(self.o.matvec(self._a(u), h1, h2).ravel()))

    def gather(self, v, idx):
        return v[idx].clone()

    def scatter_add(self, v, idx, pos, buf):
        v[idx] += buf[pos]

    def multiplicity(self):
        return torch.from_numpy(self.o.mult.astype(np.float64).ravel().copy())

    def set_multiplicity(self, mult):
        self.mult = mult.numpy().reshape(self.shape).copy()

    def wdot(self, a, b):
        return float(np.sum(self._a(a) * self._a(b) / self.mult))

    def jacobi_diag(self, h1, h2):
        d = solve.local_diagonal(self.o.G, self.o.D, h1, h2, self.o.B)
        return torch.from_numpy(operator.dssum(d, self.o.gid).ravel().copy())

    def jacobi_invert(self, d):
        dd = self._a(d)
        out = np.where(self.o.mask != 0, 1.0 / np.where(dd != 0, dd, 1.0), 0.0)
        return torch.from_numpy(out.ravel().copy())

    def cg_update(self, alpha, p, w, x, r, dinv, z):
        xa, ra, za = self._a(x), self._a(r), self._a(z)
        xa += alpha * self._a(p)
        ra -= alpha * self._a(w)
        za[...] = self._a(dinv) * ra
        return [float(np.sum(ra * za / self.mult)), float(np.sum(ra * ra / self.mult))]

    def cg_direction(self, beta, z, p):
        pa = self._a(p)
        pa[...] = self._a(z) + beta * pa
