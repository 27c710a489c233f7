"""Structured hexahedral box mesh on GLL nodes (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

§2 (after Eq. 6): Omega is split into E non-overlapping hexahedra; every
local GLL point u^e_ijk of every element carries a value, and every degree of
freedom gets one unique global number.  The Boolean gather Q^T maps local to
global numbers (Eq. 10).  The oracle builds a structured nelx x nely x nelz box
with element index e = ex + nelx (ey + nely ez) and local index [e, k, j, i].

Readings where the paper is silent:
* the global number of the point with lattice index (ix, iy, iz), ix = N ex + i,
  is ix + (N nelx + 1) (iy + (N nely + 1) iz);
* "deformed" boxes apply x' = x + a sin(y) sin(z), y' = y + a sin(z) sin(x),
  z' = z + a sin(x) sin(y) at every GLL node, evaluated at the undeformed
  coordinates (an isoparametric degree-N map);
* homogeneous Dirichlet data (§2, Eq. 5) is imposed by a 0/1 mask on every
  global point of the selected box faces.
"""
import numpy as np

from .gll import gll_nodes_weights

# bit of each box face in a Dirichlet face mask
FACE_XMIN, FACE_XMAX, FACE_YMIN, FACE_YMAX, FACE_ZMIN, FACE_ZMAX = 1, 2, 4, 8, 16, 32
ALL_FACES = 63


def lattice_indices(nelx, nely, nelz, N):
    """Global lattice indices (ix, iy, iz) of every local point, each (E,p,p,p)."""
    p = N + 1
    E = nelx * nely * nelz
    e = np.arange(E)
    ex = e % nelx
    ey = (e // nelx) % nely
    ez = e // (nelx * nely)
    i = np.arange(p)
    ix = N * ex[:, None, None, None] + i[None, None, None, :]
    iy = N * ey[:, None, None, None] + i[None, None, :, None]
    iz = N * ez[:, None, None, None] + i[None, :, None, None]
    shape = (E, p, p, p)
    return (np.broadcast_to(ix, shape), np.broadcast_to(iy, shape),
            np.broadcast_to(iz, shape))


def box_coords(nelx, nely, nelz, N, x0=(0.0, 0.0, 0.0), length=(1.0, 1.0, 1.0),
               deform_amp=0.0):
    """Physical coordinates (x, y, z) of every local GLL point, each (E,p,p,p)."""
    xi, _ = gll_nodes_weights(N)
    p = N + 1
    E = nelx * nely * nelz
    e = np.arange(E)
    ex = e % nelx
    ey = (e // nelx) % nely
    ez = e // (nelx * nely)
    hx, hy, hz = length[0] / nelx, length[1] / nely, length[2] / nelz
    t = (xi + 1.0) / 2.0
    x = x0[0] + (ex[:, None, None, None] + t[None, None, None, :]) * hx
    y = x0[1] + (ey[:, None, None, None] + t[None, None, :, None]) * hy
    z = x0[2] + (ez[:, None, None, None] + t[None, :, None, None]) * hz
    shape = (E, p, p, p)
    x, y, z = (np.broadcast_to(x, shape).copy(), np.broadcast_to(y, shape).copy(),
               np.broadcast_to(z, shape).copy())
    if deform_amp != 0.0:
        a = deform_amp
        xd = x + a * np.sin(y) * np.sin(z)
        yd = y + a * np.sin(z) * np.sin(x)
        zd = z + a * np.sin(x) * np.sin(y)
        x, y, z = xd, yd, zd
    return x, y, z


def global_ids(nelx, nely, nelz, N):
    """Unique global number of every local point (the action of Q^T), (E,p,p,p)."""
    ix, iy, iz = lattice_indices(nelx, nely, nelz, N)
    gx = N * nelx + 1
    gy = N * nely + 1
    return (ix + gx * (iy + gy * iz)).astype(np.int64)


def dirichlet_mask(nelx, nely, nelz, N, faces=ALL_FACES):
    """0 on local points whose global point lies on a selected box face, else 1."""
    ix, iy, iz = lattice_indices(nelx, nely, nelz, N)
    m = np.ones(ix.shape)
    if faces & FACE_XMIN:
        m[ix == 0] = 0.0
    if faces & FACE_XMAX:
        m[ix == N * nelx] = 0.0
    if faces & FACE_YMIN:
        m[iy == 0] = 0.0
    if faces & FACE_YMAX:
        m[iy == N * nely] = 0.0
    if faces & FACE_ZMIN:
        m[iz == 0] = 0.0
    if faces & FACE_ZMAX:
        m[iz == N * nelz] = 0.0
    return m


def multiplicity(gid):
    """Number of local copies of each local point's global point, (E,p,p,p)."""
    counts = np.bincount(gid.ravel())
    return counts[gid].astype(np.float64)
