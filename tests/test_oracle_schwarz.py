"""Pins of the two-level Schwarz preconditioner and of flexible GMRES in the
oracle against independent constructions: the assembled operator applied to
unit vectors, dense Kronecker matrices and dense solves, trilinear fields,
the Galerkin identity through the matrix-free operator, and the least-squares
minimum over an explicit Krylov basis."""
import numpy as np
import pytest

import seeded_inputs as si
from oracle import mesh, operator, solve, schwarz, gmres
from oracle.schwarz import Schwarz
from tests.helpers import OracleProblem, TWO_PI


def dense_separable(S1, h1, h2):
    """Kronecker-sum matrix h1 (Bz x By x Ax + Bz x Ay x Bx + Az x By x Bx) + h2 Bz x By x Bx
    from per-direction (A, B) pairs; index order [c, b, a] flattened, a fastest."""
    (Ax, Bx), (Ay, By), (Az, Bz) = S1
    k = np.kron
    return (h1 * (k(Bz, k(By, Ax)) + k(Bz, k(Ay, Bx)) + k(Az, k(By, Bx)))
            + h2 * k(Bz, k(By, Bx)))


def assembled_column(o, g, h1, h2):
    """Column g of the assembled, masked operator on the lattice."""
    ng = o.gid.max() + 1
    eg = np.zeros(ng)
    eg[g] = 1.0
    w = o.matvec(eg[o.gid], h1, h2)
    out = np.zeros(ng)
    out[o.gid.reshape(-1)] = w.reshape(-1)
    return out


@pytest.mark.parametrize("faces", [mesh.ALL_FACES, mesh.FACE_XMIN | mesh.FACE_YMAX | mesh.FACE_ZMIN])
@pytest.mark.parametrize("elem", [(1, 1, 1), (0, 0, 0), (2, 1, 0), (0, 2, 1)])
@pytest.mark.parametrize("N", [2, 3, 6])
def test_separable_operator_is_the_restricted_assembled_operator(faces, elem, N):
    """Undeformed box: the Kronecker sum of the grown element's 1D operators
    equals the assembled operator restricted to the subdomain's points."""
    nel, length, h1, h2 = (3, 3, 2), (1.5, 1.0, 0.8), 0.7, 1.3
    o = OracleProblem(nel, N, length=length, faces=faces)
    ex, ey, ez = elem
    ez = min(ez, nel[2] - 1)
    one = []
    keeps = []
    for d, (e_d, nd, lo_f, hi_f) in enumerate(((ex, nel[0], mesh.FACE_XMIN, mesh.FACE_XMAX),
                                               (ey, nel[1], mesh.FACE_YMIN, mesh.FACE_YMAX),
                                               (ez, nel[2], mesh.FACE_ZMIN, mesh.FACE_ZMAX))):
        lo, hi = schwarz.side_kinds(e_d, nd, lo_f, hi_f, faces)
        A, B, keep = schwarz.extended_1d(N, length[d] / nd, lo, hi)
        one.append((A, B))
        keeps.append(keep)
    At = dense_separable(one, h1, h2)
    kx, ky, kz = keeps
    keep = (kz[:, None, None] & ky[None, :, None] & kx[None, None, :]).reshape(-1)
    gx, gy = N * nel[0] + 1, N * nel[1] + 1
    a = np.arange(N + 3) - 1
    ix, iy, iz = N * ex + a, N * ey + a, N * ez + a
    lat = (ix[None, None, :] + gx * (iy[None, :, None] + gy * iz[:, None, None])).reshape(-1)
    sel = np.flatnonzero(keep)
    ref = np.zeros((sel.size, sel.size))
    for q, s in enumerate(sel):
        ref[:, q] = assembled_column(o, lat[s], h1, h2)[lat[sel]]
    got = At[np.ix_(sel, sel)]
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("kinds", [(schwarz.NEIGHBOUR, schwarz.NEIGHBOUR),
                                   (schwarz.DIRICHLET, schwarz.NEIGHBOUR),
                                   (schwarz.NEIGHBOUR, schwarz.FREE),
                                   (schwarz.FREE, schwarz.DIRICHLET)])
@pytest.mark.parametrize("N", [2, 5, 7])
def test_fast_diagonalisation_inverts_the_separable_operator(kinds, N):
    A, B, keep = schwarz.extended_1d(N, 0.4, *kinds)
    S, lam = schwarz.fdm_1d(A, B)
    assert np.allclose(S.T @ B @ S, np.eye(N + 3), atol=1e-12)
    assert np.allclose(S.T @ A @ S, np.diag(lam), atol=1e-10 * np.abs(lam).max())
    A2, B2, _ = schwarz.extended_1d(N, 0.9, schwarz.NEIGHBOUR, schwarz.NEIGHBOUR)
    S2, l2 = schwarz.fdm_1d(A2, B2)
    h1, h2 = 1.7, 0.6
    At = dense_separable([(A, B), (A2, B2), (A, B)], h1, h2)
    v = si.uniform(((N + 3) ** 3,), 90)
    got = schwarz.fdm_solve((At @ v).reshape(N + 3, N + 3, N + 3), S, S2, S, lam, l2, lam, h1, h2)
    assert np.abs(got.reshape(-1) - v).max() <= 1e-10


def test_single_element_local_solve_is_exact():
    """One undeformed element, Dirichlet on every face: the local solve is
    the exact inverse of the operator on the interior points."""
    N = 5
    o = OracleProblem((1, 1, 1), N, length=(1.0, 2.0, 0.5))
    sw = Schwarz((1, 1, 1), N, o.G, o.B, length=(1.0, 2.0, 0.5), h1=1.0, h2=0.3)
    x = si.uniform(o.shape, 91) * o.mask
    r = o.matvec(x, 1.0, 0.3)
    z = sw.local(sw.to_global(r)).reshape(-1)[o.gid]
    assert np.abs(z - x).max() <= 1e-11 * np.abs(x).max()


def test_prolongation_reproduces_trilinear_fields():
    nel, N, length = (3, 2, 2), 4, (1.0, 1.5, 2.0)
    o = OracleProblem(nel, N, length=length, faces=0)
    sw = Schwarz(nel, N, o.G, o.B, length=length, faces=0)
    f = lambda x, y, z: 1.0 + 2.0 * x - y + 3.0 * z + x * y - 0.5 * x * y * z + y * z
    vz, vy, vx = np.meshgrid(np.arange(nel[2] + 1) * length[2] / nel[2],
                             np.arange(nel[1] + 1) * length[1] / nel[1],
                             np.arange(nel[0] + 1) * length[0] / nel[0], indexing="ij")
    got = sw.prolong(f(vx, vy, vz))
    assert np.abs(got - f(o.x, o.y, o.z)).max() <= 1e-13
    # continuous: every copy of a point holds the same value
    assert np.abs(operator.dssum(got / o.mult, o.gid) - got).max() <= 1e-13


def test_restriction_is_the_transpose_of_prolongation():
    nel, N = (2, 3, 2), 3
    o = OracleProblem(nel, N, length=(TWO_PI,) * 3, deform=0.1, faces=mesh.FACE_XMIN | mesh.FACE_ZMAX)
    sw = Schwarz(nel, N, o.G, o.B, length=(TWO_PI,) * 3, faces=mesh.FACE_XMIN | mesh.FACE_ZMAX)
    r = si.uniform((o.gid.max() + 1,), 92)[o.gid] * o.mask
    c = si.uniform(sw.cmask.shape, 93) * sw.cmask
    lhs = np.sum(sw.restrict(r) * c)
    rhs = operator.weighted_dot(r, sw.prolong(c), o.mult)
    assert abs(lhs - rhs) <= 1e-12 * abs(rhs)


def test_coarse_matrix_is_galerkin():
    nel, N, h1, h2 = (3, 2, 2), 4, 0.8, 2.0
    o = OracleProblem(nel, N, length=(TWO_PI,) * 3, deform=0.1)
    sw = Schwarz(nel, N, o.G, o.B, length=(TWO_PI,) * 3, h1=h1, h2=h2)
    c1 = si.uniform(sw.cmask.shape, 94) * sw.cmask
    c2 = si.uniform(sw.cmask.shape, 95) * sw.cmask
    lhs = np.sum(c1 * sw.coarse_matvec(c2))
    rhs = operator.weighted_dot(sw.prolong(c1), o.matvec(sw.prolong(c2), h1, h2), o.mult)
    assert abs(lhs - rhs) <= 1e-12 * abs(rhs)


def test_coarse_cg_reaches_the_dense_solve():
    nel, N = (4, 3, 3), 3
    o = OracleProblem(nel, N, length=(TWO_PI,) * 3, deform=0.1)
    sw = Schwarz(nel, N, o.G, o.B, length=(TWO_PI,) * 3)
    rc = si.uniform(sw.cmask.shape, 96) * sw.cmask
    exact = sw.coarse_dense_solve(rc)
    got = sw.coarse_solve(rc, iters=200)
    assert np.abs(got - exact).max() <= 1e-10 * np.abs(exact).max()


def test_preconditioner_symmetric_positive_with_exact_coarse_solve():
    nel, N = (3, 2, 2), 3
    faces = mesh.FACE_XMIN | mesh.FACE_XMAX | mesh.FACE_YMIN | mesh.FACE_ZMAX
    o = OracleProblem(nel, N, length=(TWO_PI,) * 3, deform=0.1, faces=faces)
    sw = Schwarz(nel, N, o.G, o.B, length=(TWO_PI,) * 3, faces=faces, h2=0.5)
    ng = o.gid.max() + 1
    a = si.uniform((ng,), 97)[o.gid] * o.mask
    b = si.uniform((ng,), 98)[o.gid] * o.mask
    ma, mb = sw.apply(a, coarse_exact=True), sw.apply(b, coarse_exact=True)
    lhs = operator.weighted_dot(ma, b, o.mult)
    rhs = operator.weighted_dot(a, mb, o.mult)
    assert abs(lhs - rhs) <= 1e-12 * abs(rhs)
    assert operator.weighted_dot(ma, a, o.mult) > 0.0
    # the output is continuous and masked
    assert np.abs(operator.dssum(ma / o.mult, o.gid) - ma).max() <= 1e-12 * np.abs(ma).max()
    assert np.all(ma[o.mask == 0] == 0.0)


def test_gmres_minimises_the_residual_over_the_krylov_space():
    nel, N = (2, 2, 1), 3
    o = OracleProblem(nel, N, length=(TWO_PI,) * 3, deform=0.1)
    b = o.rhs(si.eval_fourier(si.fourier_modes(99), o.x, o.y, o.z))
    H = lambda v: o.matvec(v, 1.0, 0.4)
    wts = np.sqrt(1.0 / o.mult).reshape(-1)
    bnorm = np.sqrt(operator.weighted_dot(b, b, o.mult))
    for k in (1, 3, 6, 10):
        res = gmres.fgmres(b, H, lambda v: v, o.mult, tol=1e-30, m=50, maxit=k)
        assert res.iters == k
        basis = [b]
        for _ in range(k - 1):
            basis.append(H(basis[-1]))
        K = np.stack([v.reshape(-1) for v in basis], axis=1)
        HK = np.stack([H(v).reshape(-1) for v in basis], axis=1)
        # weighted least squares: the unique-dof norm of b - H K y
        scale = np.abs(HK).max(axis=0)
        y, *_ = np.linalg.lstsq(HK * wts[:, None] / scale, b.reshape(-1) * wts, rcond=None)
        best = np.sqrt(operator.weighted_dot(b.reshape(-1) - HK @ (y / scale),
                                             b.reshape(-1) - HK @ (y / scale),
                                             o.mult.reshape(-1))) / bnorm
        got = np.sqrt(operator.weighted_dot(b - H(res.x), b - H(res.x), o.mult)) / bnorm
        assert abs(got - best) <= 1e-7 * best + 1e-14, (k, got, best)


@pytest.mark.parametrize("nel,N", [((2, 2, 1), 3), ((2, 2, 2), 4)])
def test_arnoldi_basis_stays_orthonormal(nel, N):
    """Classical Gram-Schmidt applied twice keeps the Arnoldi vectors
    orthonormal in the unique-dof inner product to rounding over a long cycle
    (32 and 61 vectors, run to 1e-14); a single pass loses orthogonality to
    about 3e-3 on these problems."""
    o = OracleProblem(nel, N, length=(TWO_PI,) * 3, deform=0.1)
    b = o.rhs(si.eval_fourier(si.fourier_modes(99), o.x, o.y, o.z))
    cycles = []
    res = gmres.fgmres(b, lambda v: o.matvec(v, 1.0, 0.0), lambda v: v, o.mult, tol=1e-14,
                       m=1000, maxit=1000, basis=cycles)
    assert res.status == "ok" and len(cycles) == 1
    V = cycles[0]
    assert len(V) >= 30
    M = np.array([[operator.weighted_dot(a, c, o.mult) for c in V] for a in V])
    assert np.abs(M - np.eye(len(V))).max() < 1e-13


@pytest.mark.parametrize("m", [40, 4])
def test_fgmres_with_schwarz_reaches_the_solution(m):
    nel, N, h2 = (3, 3, 2), 4, 0.7
    o = OracleProblem(nel, N, length=(TWO_PI,) * 3, deform=0.1)
    sw = Schwarz(nel, N, o.G, o.B, length=(TWO_PI,) * 3, h2=h2)
    b = o.rhs(si.eval_fourier(si.fourier_modes(100), o.x, o.y, o.z))
    H = lambda v: o.matvec(v, 1.0, h2)
    res = gmres.fgmres(b, H, sw.apply, o.mult, tol=1e-10, m=m, maxit=500)
    assert res.status == "ok"
    assert o.residual(res.x, b, 1.0, h2) <= 1.0001e-10
    ref = o.pcg(b, h2=h2, tol=1e-13)
    assert np.abs(res.x - ref.x).max() <= 1e-8 * np.abs(ref.x).max()
    # the preconditioner pays: fewer iterations than Jacobi-PCG takes
    assert res.iters < ref.iters


def test_fgmres_zero_rhs():
    o = OracleProblem((1, 1, 1), 2)
    res = gmres.fgmres(np.zeros(o.shape), lambda v: o.matvec(v), lambda v: v, o.mult)
    assert res.iters == 0 and np.all(res.x == 0.0)
