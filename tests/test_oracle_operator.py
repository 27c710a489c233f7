"""Pins for the oracle's mesh, geometric factors, element operator and
gather-scatter (§2, Eq. 9-10; §3.2)."""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import mesh, geometry, operator, dense
from oracle.gll import gll_nodes_weights, deriv_matrix
import seeded_inputs as si

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "poisson_closed_forms.txt")
TWO_PI = 2 * math.pi


def build(nel, N, x0=(0, 0, 0), length=(1, 1, 1), deform=0.0):
    x, y, z = mesh.box_coords(*nel, N, x0, length, deform)
    G, B, detJ = geometry.geom_factors(x, y, z, N)
    gid = mesh.global_ids(*nel, N)
    return dict(x=x, y=y, z=z, G=G, B=B, D=deriv_matrix(N), gid=gid,
                mult=mesh.multiplicity(gid))


# ---------------------------------------------------------------- geometry
@pytest.mark.parametrize("N", [2, 5, 7])
def test_undeformed_geometric_factors(N):
    h = 0.25
    m = build((2, 3, 2), N, length=(2 * h, 3 * h, 2 * h))
    _, w = gll_nodes_weights(N)
    W = np.einsum('k,j,i->kji', w, w, w)[None]
    G = m["G"]
    for c in range(3):
        np.testing.assert_allclose(G[c], np.broadcast_to(W * h / 2, G[c].shape), rtol=1e-13)
    for c in range(3, 6):
        np.testing.assert_allclose(G[c], 0.0, atol=1e-15)
    np.testing.assert_allclose(m["B"], np.broadcast_to(W * h ** 3 / 8, m["B"].shape), rtol=1e-13)
    assert abs(m["B"].sum() - 12 * h ** 3) < 1e-13


def test_deformation_structure():
    """Structure of the deformed-box reading: the displacement of each
    coordinate depends only on the other two, and the map commutes with the
    cyclic permutation of the axes (x, y, z) -> (y, z, x), so on a cube mesh
    the point with lattice index (ix, iy, iz) lands, permuted, where the point
    (iy, iz, ix) does."""
    nel, N, a = 3, 4, 0.1
    x0, y0, z0 = mesh.box_coords(nel, nel, nel, N, (0, 0, 0), (TWO_PI,) * 3, 0.0)
    x, y, z = mesh.box_coords(nel, nel, nel, N, (0, 0, 0), (TWO_PI,) * 3, a)
    dx, dy, dz = x - x0, y - y0, z - z0
    ix, iy, iz = mesh.lattice_indices(nel, nel, nel, N)
    n = N * nel + 1

    def on_lattice(f):
        out = np.full((n, n, n), np.nan)
        out[iz.ravel(), iy.ravel(), ix.ravel()] = f.ravel()
        return out                                   # out[iz, iy, ix]

    DX, DY, DZ = on_lattice(dx), on_lattice(dy), on_lattice(dz)
    assert not np.isnan(DX).any()
    # dx is constant along x, dy along y, dz along z
    assert np.abs(DX - DX[:, :, :1]).max() < 1e-15
    assert np.abs(DY - DY[:, :1, :]).max() < 1e-15
    assert np.abs(DZ - DZ[:1, :, :]).max() < 1e-15
    assert np.abs(DX).max() > 0.05 and np.abs(DY).max() > 0.05 and np.abs(DZ).max() > 0.05
    # cyclic symmetry: dy at lattice (ix, iy, iz) equals dx at (iy, iz, ix), and
    # so on round the cycle; with arrays indexed [iz, iy, ix] the value at
    # (iy, iz, ix) is F[ix, iz, iy]
    cyc = lambda F: np.einsum('abc->bca', F)
    assert np.abs(DY - cyc(DX)).max() < 1e-15
    assert np.abs(DZ - cyc(DY)).max() < 1e-15
    assert np.abs(DX - cyc(DZ)).max() < 1e-15


def test_deformed_volume():
    # the sine deformation's det(grad) perturbation terms integrate to zero
    # over a period, so the deformed box keeps the volume (2 pi)^3
    for N in (3, 5, 7, 9):
        x, y, z = mesh.box_coords(2, 2, 2, N, (0, 0, 0), (TWO_PI,) * 3, 0.1)
        _, B, detJ = geometry.geom_factors(x, y, z, N)
        assert np.all(detJ > 0)
        assert abs(B.sum() - TWO_PI ** 3) < 1e-13 * TWO_PI ** 3
    # a map with polynomial Jacobian: x' = x (1 + c y) has det = 1 + c y,
    # so the unit cube maps to volume 1 + c/2 (exact for N >= 2)
    c = 0.4
    for N in (2, 4, 7):
        x, y, z = mesh.box_coords(3, 2, 2, N)
        _, B, detJ = geometry.geom_factors(x * (1 + c * y), y, z, N)
        assert abs(B.sum() - (1 + c / 2)) < 1e-14
        # reference-to-element scaling (hx hy hz) / 8 with h = (1/3, 1/2, 1/2)
        np.testing.assert_allclose(detJ, (1 + c * y) * (1.0 / 12) / 8, rtol=1e-13)


def test_global_ids_and_multiplicity_pattern():
    N = 3
    nel = (3, 2, 2)
    gid = mesh.global_ids(*nel, N)
    ng = (3 * N + 1) * (2 * N + 1) * (2 * N + 1)
    assert gid.max() + 1 == ng and len(np.unique(gid)) == ng
    mult = mesh.multiplicity(gid)
    # independent formula: a lattice index on an interior element interface
    # doubles the count in that direction
    ix, iy, iz = mesh.lattice_indices(*nel, N)

    def f(ind, nl):
        return np.where((ind % N == 0) & (ind > 0) & (ind < N * nl), 2, 1)
    expect = f(ix, nel[0]) * f(iy, nel[1]) * f(iz, nel[2])
    np.testing.assert_array_equal(mult, expect)
    assert set(np.unique(mult)) == {1, 2, 4, 8}
    # dssum(1) is the multiplicity
    np.testing.assert_array_equal(operator.dssum(np.ones(gid.shape), gid), mult)


def test_dirichlet_mask_faces():
    N = 2
    nel = (2, 2, 2)
    ix, iy, iz = mesh.lattice_indices(*nel, N)
    m = mesh.dirichlet_mask(*nel, N)
    on = (ix == 0) | (ix == 4) | (iy == 0) | (iy == 4) | (iz == 0) | (iz == 4)
    np.testing.assert_array_equal(m == 0, on)
    m2 = mesh.dirichlet_mask(*nel, N, faces=mesh.FACE_XMIN)
    np.testing.assert_array_equal(m2 == 0, ix == 0)


# ---------------------------------------------------------------- dssum
def test_dssum_symmetric_and_projection():
    m = build((3, 2, 2), 4, deform=0.0)
    gid, mult = m["gid"], m["mult"]
    a = si.uniform(gid.shape, 1)
    b = si.uniform(gid.shape, 2)
    lhs = np.sum(a * operator.dssum(b, gid))
    rhs = np.sum(operator.dssum(a, gid) * b)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    # continuous field: dssum(u / mult) == u
    ug = si.uniform(int(gid.max()) + 1, 3)
    u = ug[gid]
    np.testing.assert_allclose(operator.dssum(u / mult, gid), u, rtol=1e-14)


def test_dssum_explicit_loop():
    # brute force: walk every pair of local points
    m = build((2, 2, 1), 2)
    gid = m["gid"].ravel()
    w = si.uniform(gid.shape, 5)
    out = np.zeros_like(w)
    for a in range(len(w)):
        out[a] = sum(w[b] for b in range(len(w)) if gid[b] == gid[a])
    np.testing.assert_allclose(operator.dssum(w.reshape(m["gid"].shape), m["gid"]).ravel(),
                               out, rtol=1e-15)


# ---------------------------------------------------------------- Ax
@pytest.mark.parametrize("N", [1, 3, 7])
def test_ax_annihilates_constants(N):
    m = build((2, 2, 2), N, length=(TWO_PI,) * 3, deform=0.1)
    w = operator.ax_local(np.ones(m["gid"].shape), m["G"], m["D"])
    scale = np.abs(m["G"]).max() * N * N
    assert np.abs(w).max() < 1e-12 * scale


def _golden_energies():
    rows = []
    with open(GOLDEN) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                f, v = line.split("|")
                rows.append((f.strip(), float(Fraction(v.strip()))))
    return rows


@pytest.mark.parametrize("N", [2, 4, 7])
@pytest.mark.parametrize("field,energy", _golden_energies())
def test_energy_closed_forms_affine(N, field, energy):
    m = build((2, 3, 2), N)
    x, y, z = m["x"], m["y"], m["z"]
    u = eval(field, {}, dict(x=x, y=y, z=z))
    e = np.sum(u * operator.ax_local(u, m["G"], m["D"]))
    assert abs(e - energy) < 1e-12


def test_energy_sheared_affine_element():
    # affine but non-rectangular element: x' = x + 0.3 y, u = x' -> energy = volume
    N = 3
    x, y, z = mesh.box_coords(2, 2, 2, N)
    xs = x + 0.3 * y
    G, B, _ = geometry.geom_factors(xs, y, z, N)
    u = xs
    e = np.sum(u * operator.ax_local(u, G, deriv_matrix(N)))
    assert abs(e - 1.0) < 1e-12
    # cross term: a(u, v) for u = x', v = y: integral of grad x' . grad y = 0
    assert abs(np.sum(y * operator.ax_local(u, G, deriv_matrix(N)))) < 1e-12


@pytest.mark.parametrize("nel,N", [((1, 1, 1), 2), ((2, 1, 1), 3), ((2, 2, 2), 2), ((2, 2, 1), 4)])
def test_ax_matches_dense_assembly(nel, N):
    m = build(nel, N, length=(TWO_PI,) * 3, deform=0.1)
    K, M = dense.element_matrices(m["x"], m["y"], m["z"], N)
    A, Mg = dense.assemble(K, M, m["gid"])
    ug = si.uniform(A.shape[0], 11)
    uL = ug[m["gid"]]
    h2 = 0.7
    wL = operator.dssum(operator.ax_local(uL, m["G"], m["D"], 1.0, h2, m["B"]), m["gid"])
    wg = A @ ug + h2 * Mg * ug
    np.testing.assert_allclose(wL, wg[m["gid"]], rtol=0, atol=1e-12 * np.abs(wg).max())
    # element by element, unassembled, on a discontinuous random field
    uL2 = si.uniform(m["gid"].shape, 12)
    w2 = operator.ax_local(uL2, m["G"], m["D"])
    E = uL2.shape[0]
    ref = np.einsum('epq,eq->ep', K, uL2.reshape(E, -1)).reshape(uL2.shape)
    np.testing.assert_allclose(w2, ref, rtol=0, atol=1e-12 * np.abs(ref).max())


def test_variable_coefficient_matches_dense():
    N = 2
    nel = (2, 1, 1)
    m = build(nel, N, length=(TWO_PI,) * 3, deform=0.1)
    h1 = 1.0 + 0.5 * si.uniform(m["gid"].shape, 21)
    # dense: scale every quadrature point's contribution by h1 at that point
    _, w = gll_nodes_weights(N)
    Dr, Ds, Dt = dense.reference_gradient_matrices(N)
    W = np.einsum('k,j,i->kji', w, w, w).ravel()
    E = m["x"].shape[0]
    n = (N + 1) ** 3
    u = si.uniform(m["gid"].shape, 22)
    for e in range(E):
        X = np.stack([m["x"][e].ravel(), m["y"][e].ravel(), m["z"][e].ravel()])
        K = np.zeros((n, n))
        for q in range(n):
            J = np.array([[Dr[q] @ X[a], Ds[q] @ X[a], Dt[q] @ X[a]] for a in range(3)])
            phys = np.linalg.inv(J).T @ np.stack([Dr[q], Ds[q], Dt[q]])
            K += h1[e].ravel()[q] * W[q] * np.linalg.det(J) * (phys.T @ phys)
        got = operator.ax_local(u, m["G"], m["D"], h1_field=h1)[e].ravel()
        np.testing.assert_allclose(got, K @ u[e].ravel(), atol=1e-12 * np.abs(K).max())


@pytest.mark.parametrize("nel,N", [((2, 2, 2), 2), ((3, 2, 1), 3)])
def test_assembled_masked_operator_spd(nel, N):
    m = build(nel, N, length=(TWO_PI,) * 3, deform=0.1)
    K, M = dense.element_matrices(m["x"], m["y"], m["z"], N)
    A, _ = dense.assemble(K, M, m["gid"])
    mask = mesh.dirichlet_mask(*nel, N)
    interior = np.zeros(A.shape[0], bool)
    interior[m["gid"][mask == 1]] = True
    Ai = A[np.ix_(interior, interior)]
    np.testing.assert_allclose(Ai, Ai.T, atol=1e-13 * np.abs(Ai).max())
    np.linalg.cholesky(Ai)      # raises if not positive definite
    # the matrix-free operator, probed column by column, is this matrix
    gi = np.nonzero(interior)[0]
    for col in gi[:: max(1, len(gi) // 7)]:
        eg = np.zeros(A.shape[0])
        eg[col] = 1.0
        wL = operator.matvec(eg[m["gid"]], m["G"], m["D"], m["gid"], mask)
        expect = (A[:, col] * interior)[m["gid"]]
        np.testing.assert_allclose(wL, expect, atol=1e-12 * np.abs(A).max())


@pytest.mark.parametrize("h2", [0.0, 1.7])
def test_energy_from_local_products(h2):
    """<p, mask QQ^T H_L p> on unique dofs equals sum_L p_L (H_L p)_L when p is
    continuous and zero on Dirichlet points (the identity the element kernels
    use to form <p, w> of CG without the gather-scatter)."""
    m = build((3, 2, 3), 5, length=(2 * math.pi,) * 3, deform=0.1)
    gid, mult = m["gid"], m["mult"]
    mask = mesh.dirichlet_mask(3, 2, 3, 5)
    pg = si.uniform(int(gid.max()) + 1, 9)
    p = pg[gid] * mask                      # continuous, zero on the boundary
    w = operator.matvec(p, m["G"], m["D"], gid, mask, 1.0, h2, m["B"])
    lhs = operator.weighted_dot(p, w, mult)
    rhs = float(np.sum(p * operator.ax_local(p, m["G"], m["D"], 1.0, h2, m["B"])))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    # a p that is not continuous breaks it: the identity is not a tautology
    q = p + 1e-3 * si.uniform(p.shape, 10) * mask
    wq = operator.matvec(q, m["G"], m["D"], gid, mask, 1.0, h2, m["B"])
    assert abs(operator.weighted_dot(q, wq, mult) -
               float(np.sum(q * operator.ax_local(q, m["G"], m["D"], 1.0, h2, m["B"])))) > 1e-9
