"""Element partition across processes (arXiv 2107.01243 §3.2, Algorithm 1).

Neko distributes the elements over MPI ranks.  Each rank applies the element
operator to its own elements, sums the copies of a shared point that it holds
itself, then exchanges the partial sums of the points on its interfaces with
the neighbouring ranks and adds what they sent; the Krylov dots end in one
global reduction each.  This module is that scheme's host side on a
structured element box:

  grid_dims / split_box   processor grid (px, py, pz) with the least interface
                          area, and each rank's sub-box of elements
  SubBox                  offset and size of a rank's sub-box, its neighbours
                          across its six faces, the faces on the global boundary
  face_lists              index lists of one face plane of a sub-box: one local
                          copy per face point (to send) and every local copy
                          with its face point (to add what was received)
  Exchange                the interface sum over torch.distributed: direction
                          x, then y, then z, so that points on edges and corners
                          shared by 4 or 8 ranks are completed as well
  PartitionedOperator     w = mask o QQ^T H u over all ranks
  partitioned_pcg         Jacobi-PCG over all ranks, one all-reduce per dot
  DeviceBackend           the compute of one rank on its handle, in the CUDA
                          library (sem_apply, sem_gather, sem_scatter_add,
                          sem_dot, sem_cg_update, ...)

Numbering of a sub-box of (nx, ny, nz) elements of order N: element
e = ex + nx (ey + ny ez), local point e (N+1)^3 + (k (N+1) + j)(N+1) + i, lattice
point (ix, iy, iz) = (N ex + i, N ey + j, N ez + k).  Face f = 2 d + side lies at
lattice coordinate 0 (side 0) or N n_d (side 1) along direction d; its points
are numbered a + (N n_a + 1) b over the two other directions a < b.  Ranks
that share a face have the same extents along a and b, so both number the
face's points alike.

The operator, the multiplicities and the Jacobi diagonal are assembled the same
way: the rank's own gather-scatter first, then the exchange.  The mask of a
rank holds only the global box's Dirichlet faces that its sub-box touches, so
interface points are never masked before the exchange; points on a Dirichlet
face are zero on every rank that holds them, before and after it.
"""
import numpy as np

FACE_NAMES = ("xmin", "xmax", "ymin", "ymax", "zmin", "zmax")


# ---------------------------------------------------------------- decomposition
def grid_dims(nel, world):
    """(px, py, pz) with px py pz = world and p_d <= nel_d that minimises the
    interface area (element faces cut by the partition)."""
    best = None
    for px in range(1, world + 1):
        if world % px:
            continue
        for py in range(1, world // px + 1):
            if (world // px) % py:
                continue
            pz = world // (px * py)
            p = (px, py, pz)
            if any(p[d] > nel[d] for d in range(3)):
                continue
            cost = ((px - 1) * nel[1] * nel[2] + (py - 1) * nel[0] * nel[2] +
                    (pz - 1) * nel[0] * nel[1])
            if best is None or cost < best[0]:
                best = (cost, p)
    if best is None:
        raise ValueError(f"{world} ranks cannot split a {nel} element box")
    return best[1]


def _blocks(n, p):
    """Offsets and sizes of n items in p contiguous blocks (sizes differ by <= 1)."""
    sizes = [n // p + (1 if c < n % p else 0) for c in range(p)]
    offs = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(int).tolist()
    return offs, sizes


class SubBox:
    """Rank `rank`'s elements of a (nelx, nely, nelz) box on a processor grid
    `dims`: rank = cx + px (cy + py cz)."""

    def __init__(self, nel, dims, rank):
        self.nel_global = tuple(int(v) for v in nel)
        self.dims = tuple(int(v) for v in dims)
        px, py, pz = self.dims
        self.rank = rank
        self.coord = (rank % px, (rank // px) % py, rank // (px * py))
        self.offset, self.count = [], []
        for d in range(3):
            offs, sizes = _blocks(self.nel_global[d], self.dims[d])
            self.offset.append(offs[self.coord[d]])
            self.count.append(sizes[self.coord[d]])
        self.offset, self.count = tuple(self.offset), tuple(self.count)
        # neighbour rank across each face (None on the global boundary)
        self.neighbours = []
        for f in range(6):
            d, side = divmod(f, 2)
            c = list(self.coord)
            c[d] += 1 if side else -1
            if 0 <= c[d] < self.dims[d]:
                self.neighbours.append(c[0] + px * (c[1] + py * c[2]))
            else:
                self.neighbours.append(None)
        self.neighbours = tuple(self.neighbours)
        # bits of the global faces this sub-box lies on
        self.boundary = sum(1 << f for f in range(6) if self.neighbours[f] is None)

    def local_faces(self, dirichlet_faces):
        """Dirichlet faces of the rank's handle: the global ones it touches."""
        return int(dirichlet_faces) & self.boundary

    def local_mesh(self, x0, length):
        """(x0, len) of the sub-box with the global box's element size."""
        h = [length[d] / self.nel_global[d] for d in range(3)]
        return (tuple(x0[d] + self.offset[d] * h[d] for d in range(3)),
                tuple(self.count[d] * h[d] for d in range(3)))


def split_box(nel, world, rank, dims=None):
    return SubBox(nel, dims or grid_dims(nel, world), rank)


# ---------------------------------------------------------------- face index lists
def face_lists(count, N, face):
    """Index lists of face `face` of a sub-box of `count` elements, order N.

    pack[m]:  a local point that is a copy of face point m (after the rank's own
              gather-scatter every copy holds the same value);
    add_idx:  every local point on the face, add_pos its face point m.
    """
    P = N + 1
    d, side = divmod(face, 2)
    a, b = [x for x in range(3) if x != d]
    na, nb = count[a], count[b]
    ga = N * na + 1
    npts = ga * (N * nb + 1)
    e_d = count[d] - 1 if side else 0
    l_d = N if side else 0
    strides = (1, count[0], count[0] * count[1])     # element index per direction
    lstr = (1, P, P * P)                              # local index inside an element
    # every local copy on the face: elements (ea, eb), nodes (la, lb)
    ea, eb, la, lb = np.meshgrid(np.arange(na), np.arange(nb), np.arange(P), np.arange(P),
                                 indexing="ij")
    e = e_d * strides[d] + ea * strides[a] + eb * strides[b]
    q = e * P ** 3 + l_d * lstr[d] + la * lstr[a] + lb * lstr[b]
    m = (N * ea + la) + ga * (N * eb + lb)
    add_idx = q.ravel().astype(np.int64)
    add_pos = m.ravel().astype(np.int64)
    pack = np.full(npts, -1, dtype=np.int64)
    pack[add_pos] = add_idx                           # any copy will do
    assert (pack >= 0).all()
    return pack, add_idx, add_pos


# ---------------------------------------------------------------- exchange
class Exchange:
    """In-place interface sum of an L-vector over the ranks of the default
    torch.distributed group: x faces, then y, then z.  Buffers travel as the
    backend's tensors; with `host_staged` (gloo with CUDA vectors) they are
    copied to host memory for the transfer."""

    def __init__(self, backend, sub, N, host_staged=False):
        import torch.distributed as dist
        self.dist = dist
        self.be = backend
        self.sub = sub
        self.staged = host_staged
        self.lists = {}
        for f in range(6):
            if sub.neighbours[f] is None:
                continue
            pack, add_idx, add_pos = face_lists(sub.count, N, f)
            self.lists[f] = (backend.index(pack), backend.index(add_idx), backend.index(add_pos),
                             len(pack))

    def __call__(self, v):
        dist = self.dist
        for d in range(3):
            pending = []
            for side in (0, 1):
                f = 2 * d + side
                if f not in self.lists:
                    continue
                pack, _, _, npts = self.lists[f]
                send = self.be.gather(v, pack)
                recv = self.be.empty(npts)
                if self.staged:
                    send_c = send.cpu()
                    recv_c = send_c.new_empty(npts)
                else:
                    send_c, recv_c = send, recv
                nb = self.sub.neighbours[f]
                reqs = [dist.isend(send_c, nb), dist.irecv(recv_c, nb)]
                pending.append((f, reqs, send_c, recv, recv_c))
            for f, reqs, _, recv, recv_c in pending:
                for r in reqs:
                    r.wait()
                if self.staged:
                    recv.copy_(recv_c)
                _, add_idx, add_pos, _ = self.lists[f]
                self.be.scatter_add(v, add_idx, add_pos, recv)
        return v

    def allreduce(self, values):
        """Sum of host floats over the ranks (one collective for all of them)."""
        t = self.be.scalars(values)
        self.dist.all_reduce(t)
        return [float(x) for x in t.cpu()]


# ---------------------------------------------------------------- operator and PCG
class PartitionedOperator:
    """mask o QQ^T (h1 A + h2 B) over all ranks: each rank's operator on its
    sub-box, then the interface exchange.  Setting it up also gives the
    backend the global multiplicities (its dots then return this rank's share
    of the unique-dof inner product)."""

    def __init__(self, backend, sub, N, host_staged=False):
        self.be = backend
        self.sub = sub
        self.exchange = Exchange(backend, sub, N, host_staged)
        mult = backend.multiplicity()
        self.exchange(mult)
        backend.set_multiplicity(mult)

    def apply(self, u, w, h1=1.0, h2=0.0):
        self.be.apply(u, w, h1, h2)
        return self.exchange(w)

    def dot(self, a, b):
        return self.exchange.allreduce([self.be.wdot(a, b)])[0]


def partitioned_pcg(op, b, x, h1=1.0, h2=0.0, tol=1e-8, maxit=20000):
    """Jacobi-PCG for the partitioned operator, in the order of the library's
    sem_cg_solve: x0 = 0, r = b, z = dinv r, p = z; each iteration w = H p
    (with the exchange), alpha = <r,z>/<p,w>, x += alpha p, r -= alpha w, stop
    when <r,r> <= tol^2 <b,b>, beta, p = z + beta p.  Every dot is the sum over
    the ranks of their shares.  Returns (iterations, relative residual,
    status) with status "ok", "breakdown" or "noconv"."""
    be, ex = op.be, op.exchange
    d = be.jacobi_diag(h1, h2)
    ex(d)
    dinv = be.jacobi_invert(d)
    r, z, p, w = be.copy(b), be.zeros(), be.zeros(), be.zeros()
    be.fill(x, 0.0)
    rz, rr = ex.allreduce(be.cg_update(0.0, r, r, x, r, dinv, z))
    bb = rr
    if bb == 0.0:
        return 0, 0.0, "ok"
    tol2 = tol * tol * bb
    if rr <= tol2:
        return 0, float(np.sqrt(rr / bb)), "ok"
    be.cg_direction(0.0, z, p)
    for it in range(1, maxit + 1):
        op.apply(p, w, h1, h2)
        (pw,) = ex.allreduce([be.wdot(p, w)])
        if not pw > 0.0:
            return it, float(np.sqrt(rr / bb)), "breakdown"
        alpha = rz / pw
        rz_new, rr = ex.allreduce(be.cg_update(alpha, p, w, x, r, dinv, z))
        if not (rr == rr):
            return it, float("nan"), "breakdown"
        if rr <= tol2:
            return it, float(np.sqrt(rr / bb)), "ok"
        beta = rz_new / rz
        rz = rz_new
        be.cg_direction(beta, z, p)
    return maxit, float(np.sqrt(rr / bb)), "noconv"


# ---------------------------------------------------------------- CUDA backend
class DeviceBackend:
    """A rank's compute in the CUDA library, on the handle of its sub-box.
    Vectors are CUDA float64 tensors of the handle's n_L values."""

    def __init__(self, h, device="cuda"):
        import torch
        from . import api
        self.torch = torch
        self.api = api
        self.h = h
        self.dev = torch.device(device)
        self.n = h.n_local
        self._dot = torch.empty(1, dtype=torch.float64, device=self.dev)
        self._dots = torch.empty(2, dtype=torch.float64, device=self.dev)

    # vectors and index arrays
    def index(self, a):
        return self.torch.from_numpy(np.ascontiguousarray(a, dtype=np.int64)).to(self.dev)

    def empty(self, n):
        return self.torch.empty(n, dtype=self.torch.float64, device=self.dev)

    def zeros(self):
        return self.torch.zeros(self.n, dtype=self.torch.float64, device=self.dev)

    def copy(self, v):
        return v.clone()

    def fill(self, v, value):
        v.fill_(value)

    def scalars(self, values):
        return self.torch.tensor(values, dtype=self.torch.float64, device=self.dev)

    # compute
    def apply(self, u, w, h1, h2):
        self.api.sem_apply(self.h, u, w, h1, h2)

    def gather(self, v, idx):
        return self.api.sem_gather(self.h, v, idx, self.empty(idx.numel()))

    def scatter_add(self, v, idx, pos, buf):
        self.api.sem_scatter_add(self.h, v, idx, pos, buf)

    def multiplicity(self):
        m = self.empty(self.n)
        self.api.sem_get_field(self.h, 5, m)          # SEM_FIELD_MULT
        return m

    def set_multiplicity(self, mult):
        self.api.sem_set_multiplicity(self.h, mult)

    def wdot(self, a, b):
        self.api.sem_dot(self.h, a, b, self._dot)
        return float(self._dot.item())

    def jacobi_diag(self, h1, h2):
        return self.api.sem_jacobi_diag(self.h, self.empty(self.n), h1, h2)

    def jacobi_invert(self, d):
        return self.api.sem_jacobi_invert(self.h, d, self.empty(self.n))

    def cg_update(self, alpha, p, w, x, r, dinv, z):
        self.api.sem_cg_update(self.h, alpha, p, w, x, r, dinv, z, self._dots)
        return [float(v) for v in self._dots.cpu()]

    def cg_direction(self, beta, z, p):
        self.api.sem_cg_direction(self.h, beta, z, p)


def setup_rank(nel, N, world, rank, x0=(0.0, 0.0, 0.0), length=(1.0, 1.0, 1.0), deform=0.0,
               faces=63, dims=None, host_staged=False, device="cuda"):
    """Handle, backend and operator of one rank (the default torch.distributed
    group must be initialised)."""
    from . import api
    sub = split_box(nel, world, rank, dims)
    lx0, llen = sub.local_mesh(x0, length)
    h = api.sem_setup(sub.count, N, x0=lx0, length=llen, deform=deform,
                      faces=sub.local_faces(faces))
    be = DeviceBackend(h, device)
    return sub, h, be, PartitionedOperator(be, sub, N, host_staged)


__all__ = ["FACE_NAMES", "grid_dims", "SubBox", "split_box", "face_lists", "Exchange",
           "PartitionedOperator", "partitioned_pcg", "DeviceBackend", "setup_rank"]
