"""Pins for the oracle's Jacobi preconditioner and PCG (§2 end, §4), the
manufactured-solution spectral convergence, and Helmholtz special cases."""
import math

import numpy as np
import pytest

from oracle import mesh, geometry, operator, solve, dense
from oracle.gll import deriv_matrix
import seeded_inputs as si

TWO_PI = 2 * math.pi


def build(nel, N, x0=(0, 0, 0), length=(1, 1, 1), deform=0.0, faces=mesh.ALL_FACES):
    x, y, z = mesh.box_coords(*nel, N, x0, length, deform)
    G, B, _ = geometry.geom_factors(x, y, z, N)
    gid = mesh.global_ids(*nel, N)
    return dict(x=x, y=y, z=z, G=G, B=B, D=deriv_matrix(N), gid=gid,
                mult=mesh.multiplicity(gid), mask=mesh.dirichlet_mask(*nel, N, faces))


@pytest.mark.parametrize("h1,h2", [(1.0, 0.0), (1.0, 2.5)])
def test_jacobi_diagonal_matches_dense(h1, h2):
    nel, N = (2, 2, 1), 3
    m = build(nel, N, length=(TWO_PI,) * 3, deform=0.1)
    K, M = dense.element_matrices(m["x"], m["y"], m["z"], N)
    E = K.shape[0]
    dl = solve.local_diagonal(m["G"], m["D"], h1, h2, m["B"])
    expect = (h1 * np.einsum('epp->ep', K) + h2 * M).reshape(dl.shape)
    np.testing.assert_allclose(dl, expect, rtol=1e-12)
    assert E == 4


@pytest.mark.parametrize("h2", [0.0, 3.0])
def test_pcg_matches_dense_cholesky(h2):
    nel, N = (2, 2, 2), 3
    m = build(nel, N, length=(TWO_PI,) * 3, deform=0.1)
    K, M = dense.element_matrices(m["x"], m["y"], m["z"], N)
    A, Mg = dense.assemble(K, M, m["gid"])
    H = A + h2 * np.diag(Mg)
    f = si.eval_fourier(si.fourier_modes(5), m["x"], m["y"], m["z"])
    b = solve.rhs(f, m["B"], m["gid"], m["mask"])
    res = solve.pcg(b, m["G"], m["D"], m["gid"], m["mask"], m["mult"], 1.0, h2, m["B"],
                    tol=1e-13)
    assert res.status == "ok"
    interior = np.zeros(A.shape[0], bool)
    interior[m["gid"][m["mask"] == 1]] = True
    bg = np.zeros(A.shape[0])
    bg[m["gid"]] = b                    # b is continuous: every copy holds the sum
    L = np.linalg.cholesky(H[np.ix_(interior, interior)])
    xi = np.linalg.solve(L.T, np.linalg.solve(L, bg[interior]))
    xg = np.zeros(A.shape[0])
    xg[interior] = xi
    np.testing.assert_allclose(res.x, xg[m["gid"]], atol=1e-10 * np.abs(xi).max())
    # residual helper agrees
    assert solve.residual(res.x, b, m["G"], m["D"], m["gid"], m["mask"], m["mult"],
                          1.0, h2, m["B"]) < 1e-12


def test_pcg_energy_error_decreases_monotonically():
    nel, N = (2, 2, 2), 4
    m = build(nel, N, length=(TWO_PI,) * 3, deform=0.1)
    f = si.eval_fourier(si.fourier_modes(6), m["x"], m["y"], m["z"])
    b = solve.rhs(f, m["B"], m["gid"], m["mask"])
    xs = solve.pcg(b, m["G"], m["D"], m["gid"], m["mask"], m["mult"], tol=1e-14).x

    def energy_err(x):
        e = x - xs
        return solve.weighted_dot(e, operator.matvec(e, m["G"], m["D"], m["gid"], m["mask"]),
                                  m["mult"])
    errs = []
    for k in range(1, 25):
        x = solve.pcg(b, m["G"], m["D"], m["gid"], m["mask"], m["mult"], tol=0.0, maxit=k).x
        errs.append(energy_err(x))
    assert all(b_ <= a_ * (1 + 1e-9) for a_, b_ in zip(errs, errs[1:]))
    assert errs[-1] < 1e-6 * errs[0]


def test_spectral_convergence_manufactured():
    """-lap u = 3 pi^2 u, u = sin(pi x) sin(pi y) sin(pi z), 4^3 elements on the
    unit cube: the max nodal error falls exponentially in N."""
    errs = {}
    for N in range(2, 11):
        m = build((4, 4, 4), N)
        f = si.manufactured_f(m["x"], m["y"], m["z"])
        b = solve.rhs(f, m["B"], m["gid"], m["mask"])
        res = solve.pcg(b, m["G"], m["D"], m["gid"], m["mask"], m["mult"], tol=1e-13)
        assert res.status == "ok"
        errs[N] = np.abs(res.x - si.manufactured_u(m["x"], m["y"], m["z"])).max()
    # exponential decay: log10(err) drops by more than 0.8 per unit N over N=2..8
    slope = (math.log10(errs[8]) - math.log10(errs[2])) / 6
    assert slope < -0.8, errs
    for N in range(2, 9):
        assert errs[N + 1] < errs[N], errs
    assert errs[7] < 1e-6
    assert errs[10] < 1e-9


def test_helmholtz_mass_only_is_one_iteration():
    nel, N = (2, 2, 2), 5
    m = build(nel, N, length=(TWO_PI,) * 3, deform=0.1)
    f = si.eval_fourier(si.fourier_modes(7), m["x"], m["y"], m["z"])
    b = solve.rhs(f, m["B"], m["gid"], m["mask"])
    res = solve.pcg(b, m["G"], m["D"], m["gid"], m["mask"], m["mult"], 0.0, 2.0, m["B"],
                    tol=1e-12)
    assert res.status == "ok" and res.iters == 1
    Bg = operator.dssum(m["B"], m["gid"])
    np.testing.assert_allclose(res.x, m["mask"] * b / (2.0 * Bg), rtol=1e-12, atol=1e-15)


def test_breakdown_and_noconv_status():
    nel, N = (2, 2, 2), 3
    m = build(nel, N, length=(TWO_PI,) * 3, deform=0.1)
    f = si.eval_fourier(si.fourier_modes(8), m["x"], m["y"], m["z"])
    b = solve.rhs(f, m["B"], m["gid"], m["mask"])
    bad = solve.pcg(b, m["G"], m["D"], m["gid"], m["mask"], m["mult"], -1.0, 0.0, m["B"])
    assert bad.status == "breakdown"
    slow = solve.pcg(b, m["G"], m["D"], m["gid"], m["mask"], m["mult"], tol=1e-14, maxit=3)
    assert slow.status == "noconv" and slow.iters == 3
