"""Pins of the oracle's projection onto previous solutions (CPU): the space
stays H-orthonormal, the projected start satisfies the Galerkin condition,
a repeated right-hand side needs no iterations, solutions equal plain PCG's,
and the space restarts when full."""
import numpy as np

import seeded_inputs as si
from oracle import operator, projection
from tests.helpers import OracleProblem, TWO_PI

NEL, N = (3, 2, 2), 5


def setup(h2=0.5):
    o = OracleProblem(NEL, N, length=(TWO_PI,) * 3, deform=0.1)
    rhs = [o.rhs(si.eval_fourier(si.fourier_modes(300 + k), o.x, o.y, o.z)) for k in range(6)]

    def mv(v):
        return o.matvec(v, 1.0, h2)

    def pcg(b, tol):
        return o.pcg(b, h2=h2, tol=tol)
    return o, rhs, mv, pcg


def test_space_is_h_orthonormal_and_galerkin():
    o, rhs, mv, pcg = setup()
    proj = projection.Projection(4)
    for b in rhs[:4]:
        projection.solve_projected(proj, b, mv, pcg, o.mult, 1e-11)
    l = len(proj.X)
    assert l == 4
    gram = np.array([[operator.weighted_dot(xi, mv(xj), o.mult) for xj in proj.X]
                     for xi in proj.X])
    assert np.abs(gram - np.eye(l)).max() < 1e-9
    # W holds H X
    for x, w in zip(proj.X, proj.W):
        assert np.abs(mv(x) - w).max() < 1e-9 * np.abs(w).max()
    # Galerkin: the residual of the projected start is orthogonal to the space
    b = rhs[4]
    x_bar, r, _ = proj.project(b, o.mult)
    for x in proj.X:
        assert abs(operator.weighted_dot(x, r, o.mult)) < 1e-10 * np.sqrt(
            operator.weighted_dot(b, b, o.mult))
    assert np.abs(b - mv(x_bar) - r).max() < 1e-10 * np.abs(b).max()


def test_repeated_rhs_needs_no_iterations_and_matches_plain_pcg():
    o, rhs, mv, pcg = setup()
    proj = projection.Projection(20)
    x1, _, res1 = projection.solve_projected(proj, rhs[0], mv, pcg, o.mult, 1e-10)
    ref = pcg(rhs[0], 1e-10)
    assert res1.iters == ref.iters
    assert np.abs(x1 - ref.x).max() < 1e-12 * np.abs(ref.x).max()
    x2, x_bar, res2 = projection.solve_projected(proj, rhs[0], mv, pcg, o.mult, 1e-10)
    assert res2.iters <= 1
    assert o.residual(x2, rhs[0], 1.0, 0.5) <= 1.05e-10
    # a new right-hand side: fewer iterations than from zero, same tolerance
    x3, _, res3 = projection.solve_projected(proj, rhs[1], mv, pcg, o.mult, 1e-10)
    assert o.residual(x3, rhs[1], 1.0, 0.5) <= 1.05e-10


def test_restart_when_full():
    o, rhs, mv, pcg = setup()
    proj = projection.Projection(2)
    sizes = []
    for b in rhs[:5]:
        x, _, _ = projection.solve_projected(proj, b, mv, pcg, o.mult, 1e-10)
        sizes.append(len(proj.X))
        assert o.residual(x, b, 1.0, 0.5) <= 1.05e-10
    assert sizes == [1, 2, 1, 2, 1]
