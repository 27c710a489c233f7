"""Two-level additive overlapping Schwarz preconditioner (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

§4: Neko preconditions its pressure Poisson solves (GMRES) with a two-level
additive overlapping Schwarz method after Nek5000,

    M^-1 = R_0^T A_0^-1 R_0 + sum_k R_k^T A~_k^-1 R_k,

whose coarse level lives on linear elements and is solved only approximately
by a few (about 10) CG iterations.  The paper gives no subdomains, local
solver or coarse operator; the readings taken here (those of the Nek5000
method it cites) are:

* subdomain k is element e grown by one GLL point into each neighbour: the
  lattice points N e_d - 1 .. N e_d + N + 1 along each direction d, without
  points outside the box and without Dirichlet points.  N >= 2, so that the
  point taken from a neighbour lies inside that neighbour (for N = 1 it would
  be the neighbour's far vertex, shared with the next element);
* A~_e is separable, the Kronecker sum of one-dimensional operators on those
  points, h1 (Bz x By x Ax + Bz x Ay x Bx + Az x By x Bx) + h2 Bz x By x Bx,
  where Ad, Bd are the 1D spectral-element stiffness (2/L) D^T W D and lumped
  mass (L/2) W of the element and its two neighbours (undeformed length
  L = box length / elements along d), assembled and restricted to the
  subdomain's points.  On an undeformed box this is the assembled operator
  restricted to the subdomain;
* A~_e^-1 by fast diagonalisation: Ad S = Bd S Lambda with S^T Bd S = I in
  each direction, so A~_e^-1 = (Sz x Sy x Sx) (h1 (lx + ly + lz) + h2)^-1
  (Sz x Sy x Sx)^T;
* the local corrections are added where subdomains overlap (additive);
* the coarse space holds the trilinear functions on the element vertices:
  R_0^T interpolates vertex values to every GLL point, R_0 is its transpose
  in the unique-dof inner product, and A_0 = R_0 H R_0^T is assembled from
  the 8 x 8 element matrices Phi^T H_e Phi; vertices on Dirichlet faces are
  left out;
* A_0^-1 r_0 is approximated by a fixed number of Jacobi-preconditioned CG
  iterations from zero (10 by default).

Global (unique-dof) vectors are arrays of shape (gz, gy, gx) on the GLL
lattice; coarse vectors have shape (nelz + 1, nely + 1, nelx + 1).
"""
import numpy as np

from . import mesh
from .gll import gll_nodes_weights, deriv_matrix
from .operator import ax_local

NEIGHBOUR, DIRICHLET, FREE = 0, 1, 2


def side_kinds(e_d, nel_d, face_lo, face_hi, faces):
    """What lies beyond the low and high end of element e_d along one
    direction: a neighbour, a Dirichlet face or a free (natural) face."""
    lo = NEIGHBOUR if e_d > 0 else (DIRICHLET if faces & face_lo else FREE)
    hi = NEIGHBOUR if e_d < nel_d - 1 else (DIRICHLET if faces & face_hi else FREE)
    return lo, hi


def extended_1d(N, L, lo, hi):
    """1D stiffness and mass on the N + 3 points of a grown element.

    Position a = 0 .. N + 2 is the lattice point N e - 1 + a.  Returns (A, B,
    keep): A and B restricted to the kept points, every other position
    decoupled (unit diagonal in both), keep a boolean mask."""
    p = N + 1
    _, w = gll_nodes_weights(N)
    D = deriv_matrix(N)
    ae = (2.0 / L) * D.T @ np.diag(w) @ D
    be = (L / 2.0) * w
    n3 = 3 * N + 1                       # left neighbour, the element, right neighbour
    A3 = np.zeros((n3, n3))
    B3 = np.zeros(n3)
    for m in range(3):
        if (m == 0 and lo != NEIGHBOUR) or (m == 2 and hi != NEIGHBOUR):
            continue
        s = m * N
        A3[s:s + p, s:s + p] += ae
        B3[s:s + p] += be
    idx = np.arange(N - 1, 2 * N + 2)   # the grown element's points in the 3-element line
    keep = np.ones(N + 3, dtype=bool)
    if lo != NEIGHBOUR:
        keep[0] = False
        if lo == DIRICHLET:
            keep[1] = False
    if hi != NEIGHBOUR:
        keep[N + 2] = False
        if hi == DIRICHLET:
            keep[N + 1] = False
    A = A3[np.ix_(idx, idx)].copy()
    B = np.diag(B3[idx])
    for a in range(N + 3):
        if not keep[a]:
            A[a, :] = 0.0
            A[:, a] = 0.0
            B[a, :] = 0.0
            B[:, a] = 0.0
            A[a, a] = 1.0
            B[a, a] = 1.0
    return A, B, keep


def fdm_1d(A, B):
    """(S, lam) with A S = B S diag(lam) and S^T B S = I (B diagonal, positive)."""
    bh = 1.0 / np.sqrt(np.diag(B))
    C = bh[:, None] * A * bh[None, :]
    lam, Q = np.linalg.eigh(0.5 * (C + C.T))
    return bh[:, None] * Q, lam


def fdm_solve(r, Sx, Sy, Sz, lx, ly, lz, h1, h2):
    """A~^-1 r for r of shape (nz, ny, nx) indexed [c, b, a]."""
    t = np.einsum('xa,zyx->zya', Sx, r)          # S^T along x
    t = np.einsum('yb,zya->zba', Sy, t)          # S^T along y
    t = np.einsum('zc,zba->cba', Sz, t)          # S^T along z
    t = t / (h1 * (lx[None, None, :] + ly[None, :, None] + lz[:, None, None]) + h2)
    t = np.einsum('xa,cba->cbx', Sx, t)          # S along x
    t = np.einsum('yb,cbx->cyx', Sy, t)          # S along y
    return np.einsum('zc,cyx->zyx', Sz, t)       # S along z


class Schwarz:
    """Setup and application of the two-level preconditioner on one box mesh."""

    def __init__(self, nel, N, G, B, length=(1.0, 1.0, 1.0), faces=mesh.ALL_FACES, h1=1.0,
                 h2=0.0, coarse_iters=10):
        assert N >= 2, "the grown subdomains need N >= 2"
        self.nel = tuple(nel)
        self.N = N
        self.faces = faces
        self.h1, self.h2 = h1, h2
        self.coarse_iters = coarse_iters
        nelx, nely, nelz = self.nel
        self.gx, self.gy, self.gz = N * nelx + 1, N * nely + 1, N * nelz + 1
        self.gid = mesh.global_ids(nelx, nely, nelz, N)
        self.mult = mesh.multiplicity(self.gid)
        self.mask = mesh.dirichlet_mask(nelx, nely, nelz, N, faces)
        # per direction: the 1D factors of every element position
        self.fdm = []
        for d, (nd, lo_f, hi_f) in enumerate(((nelx, mesh.FACE_XMIN, mesh.FACE_XMAX),
                                              (nely, mesh.FACE_YMIN, mesh.FACE_YMAX),
                                              (nelz, mesh.FACE_ZMIN, mesh.FACE_ZMAX))):
            L = length[d] / nd
            per = []
            for e_d in range(nd):
                lo, hi = side_kinds(e_d, nd, lo_f, hi_f, faces)
                A, Bm, keep = extended_1d(N, L, lo, hi)
                S, lam = fdm_1d(A, Bm)
                per.append((S, lam, keep))
            self.fdm.append(per)
        # coarse level
        xi, _ = gll_nodes_weights(N)
        self.phi = np.stack([(1.0 - xi) / 2.0, (1.0 + xi) / 2.0])   # [a][i]
        self.K = self.coarse_element_matrices(G, B)
        self.cmask = self.coarse_mask()
        self.cdiag = self.coarse_diag()

    # ---------------------------------------------------------------- local level
    def local(self, rg):
        """sum_e R_e^T A~_e^-1 R_e rg for a global vector rg (gz, gy, gx)."""
        N = self.N
        nelx, nely, nelz = self.nel
        zg = np.zeros_like(rg)
        for ez in range(nelz):
            for ey in range(nely):
                for ex in range(nelx):
                    Sx, lx, kx = self.fdm[0][ex]
                    Sy, ly, ky = self.fdm[1][ey]
                    Sz, lz, kz = self.fdm[2][ez]
                    ix = N * ex - 1 + np.arange(N + 3)
                    iy = N * ey - 1 + np.arange(N + 3)
                    iz = N * ez - 1 + np.arange(N + 3)
                    keep = kz[:, None, None] & ky[None, :, None] & kx[None, None, :]
                    cz, cy, cx = (np.clip(iz, 0, self.gz - 1), np.clip(iy, 0, self.gy - 1),
                                  np.clip(ix, 0, self.gx - 1))
                    r = np.where(keep, rg[np.ix_(cz, cy, cx)], 0.0)
                    z = fdm_solve(r, Sx, Sy, Sz, lx, ly, lz, self.h1, self.h2)
                    z = np.where(keep, z, 0.0)
                    np.add.at(zg, np.ix_(cz, cy, cx), z)
        return zg

    # ---------------------------------------------------------------- coarse level
    def basis(self, a, b, c):
        """Trilinear vertex function (a, b, c) in {0, 1}^3 at the GLL points of
        an element, shape (p, p, p) indexed [k, j, i]."""
        return (self.phi[c][:, None, None] * self.phi[b][None, :, None] *
                self.phi[a][None, None, :])

    def coarse_element_matrices(self, G, B):
        """K[e, v', v] = Phi_v'^T H_e Phi_v for the 8 vertex functions,
        vertex v = a + 2 b + 4 c."""
        E = G[0].shape[0]
        K = np.zeros((E, 8, 8))
        fields = [self.basis(v & 1, (v >> 1) & 1, v >> 2) for v in range(8)]
        for v in range(8):
            u = np.broadcast_to(fields[v], G[0].shape).copy()
            hu = ax_local(u, G, deriv_matrix(self.N), self.h1, self.h2, B)
            for v2 in range(8):
                K[:, v2, v] = np.einsum('ekji,kji->e', hu, fields[v2])
        return K

    def element_vertices(self, e):
        nelx, nely, _ = self.nel
        ex, ey, ez = e % nelx, (e // nelx) % nely, e // (nelx * nely)
        return [(ez + (v >> 2), ey + ((v >> 1) & 1), ex + (v & 1)) for v in range(8)]

    def coarse_mask(self):
        nelx, nely, nelz = self.nel
        m = np.ones((nelz + 1, nely + 1, nelx + 1))
        f = self.faces
        if f & mesh.FACE_XMIN:
            m[:, :, 0] = 0.0
        if f & mesh.FACE_XMAX:
            m[:, :, nelx] = 0.0
        if f & mesh.FACE_YMIN:
            m[:, 0, :] = 0.0
        if f & mesh.FACE_YMAX:
            m[:, nely, :] = 0.0
        if f & mesh.FACE_ZMIN:
            m[0, :, :] = 0.0
        if f & mesh.FACE_ZMAX:
            m[nelz, :, :] = 0.0
        return m

    def coarse_matvec(self, c):
        """mask o A_0 c, assembled element by element."""
        out = np.zeros_like(c)
        for e in range(self.K.shape[0]):
            vs = self.element_vertices(e)
            ce = np.array([c[v] for v in vs])
            we = self.K[e] @ ce
            for v, val in zip(vs, we):
                out[v] += val
        return out * self.cmask

    def coarse_diag(self):
        d = np.zeros_like(self.cmask)
        for e in range(self.K.shape[0]):
            for q, v in enumerate(self.element_vertices(e)):
                d[v] += self.K[e, q, q]
        return d

    def prolong(self, c):
        """R_0^T c: trilinear interpolation of vertex values to every local point."""
        nelx, nely, nelz = self.nel
        E = nelx * nely * nelz
        p = self.N + 1
        u = np.zeros((E, p, p, p))
        for e in range(E):
            for v, (vz, vy, vx) in enumerate(self.element_vertices(e)):
                u[e] += c[vz, vy, vx] * self.basis(v & 1, (v >> 1) & 1, v >> 2)
        return u

    def restrict(self, r):
        """R_0 r for a continuous L-vector r: the transpose of prolong in the
        unique-dof inner product, sum over local points of phi_v r / mult."""
        rm = r / self.mult
        c = np.zeros_like(self.cmask)
        for e in range(rm.shape[0]):
            for v, vv in enumerate(self.element_vertices(e)):
                c[vv] += np.sum(rm[e] * self.basis(v & 1, (v >> 1) & 1, v >> 2))
        return c * self.cmask

    def coarse_solve(self, rc, iters=None):
        """A fixed number of Jacobi-PCG iterations on A_0 c = rc from c = 0."""
        iters = self.coarse_iters if iters is None else iters
        dinv = np.where(self.cmask != 0.0, 1.0 / np.where(self.cdiag != 0, self.cdiag, 1.0), 0.0)
        x = np.zeros_like(rc)
        r = rc * self.cmask
        z = dinv * r
        p = z.copy()
        rz = np.sum(r * z)
        for _ in range(iters):
            if rz == 0.0:
                break
            w = self.coarse_matvec(p)
            alpha = rz / np.sum(p * w)
            x = x + alpha * p
            r = r - alpha * w
            z = dinv * r
            rz_new = np.sum(r * z)
            p = z + (rz_new / rz) * p
            rz = rz_new
        return x

    # ---------------------------------------------------------------- both levels
    def to_global(self, r):
        """Global vector of a continuous L-vector (any copy of each point)."""
        g = np.zeros(self.gx * self.gy * self.gz)
        g[self.gid.reshape(-1)] = r.reshape(-1)
        return g.reshape(self.gz, self.gy, self.gx)

    def apply(self, r, coarse_exact=False):
        """M^-1 r for a continuous, masked L-vector r; the result is a
        continuous, masked L-vector.  coarse_exact: solve A_0 exactly instead
        of the fixed CG iterations (a linear, symmetric preconditioner)."""
        zl = self.local(self.to_global(r)).reshape(-1)[self.gid]
        rc = self.restrict(r)
        if coarse_exact:
            c = self.coarse_dense_solve(rc)
        else:
            c = self.coarse_solve(rc)
        return (zl + self.prolong(c)) * self.mask

    def coarse_dense_solve(self, rc):
        n = self.cmask.size
        free = self.cmask.reshape(-1) != 0.0
        A = np.zeros((n, n))
        for j in np.flatnonzero(free):
            ej = np.zeros(n)
            ej[j] = 1.0
            A[:, j] = self.coarse_matvec(ej.reshape(self.cmask.shape)).reshape(-1)
        Af = A[np.ix_(free, free)]
        out = np.zeros(n)
        out[free] = np.linalg.solve(Af, rc.reshape(-1)[free])
        return out.reshape(self.cmask.shape)
