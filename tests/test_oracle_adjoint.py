"""Pins for the oracle's adjoint gradient dL/dh1 (structure of §2, Eq. 9):
central finite differences and the uniform-scaling closed form."""
import math

import numpy as np

from oracle import mesh, geometry, operator, solve, adjoint
from oracle.gll import deriv_matrix
import seeded_inputs as si

TWO_PI = 2 * math.pi


def build(nel, N):
    x, y, z = mesh.box_coords(*nel, N, (0, 0, 0), (TWO_PI,) * 3, 0.1)
    G, B, _ = geometry.geom_factors(x, y, z, N)
    gid = mesh.global_ids(*nel, N)
    return dict(x=x, y=y, z=z, G=G, B=B, D=deriv_matrix(N), gid=gid,
                mult=mesh.multiplicity(gid), mask=mesh.dirichlet_mask(*nel, N))


def forward(m, h1, h2, b, tol=1e-14):
    r = solve.pcg(b, m["G"], m["D"], m["gid"], m["mask"], m["mult"], 1.0, h2, m["B"],
                  h1_field=h1, tol=tol, maxit=5000)
    assert r.status == "ok"
    return r.x


def gradient(m, h1, h2, b, ut):
    u = forward(m, h1, h2, b)
    gL = adjoint.loss_grad_u(u, ut, m["mult"])
    rhs_adj = operator.apply_dirichlet(operator.dssum(gL, m["gid"]), m["mask"])
    lam = forward(m, h1, h2, rhs_adj)
    return u, adjoint.grad_h1(u, lam, m["G"], m["D"])


def test_gradient_matches_central_differences():
    m = build((2, 2, 2), 3)
    h1 = si.smooth_coefficient(m["x"], m["y"], m["z"], seed=77)
    ut = si.eval_fourier(si.fourier_modes(78), m["x"], m["y"], m["z"]) * 0.01
    f = si.eval_fourier(si.fourier_modes(79), m["x"], m["y"], m["z"])
    b = solve.rhs(f, m["B"], m["gid"], m["mask"])
    h2 = 1.0
    u, g = gradient(m, h1, h2, b, ut)

    def L(h):
        return adjoint.loss(forward(m, h, h2, b), ut, m["mult"])
    # smooth direction
    d = si.eval_fourier(si.fourier_modes(80), m["x"], m["y"], m["z"])
    # central differences: truncation error ~ eps^2 (1e-6 relative at eps = 1e-4)
    eps = 1e-5 * np.abs(h1).max()
    fd = (L(h1 + eps * d) - L(h1 - eps * d)) / (2 * eps)
    assert abs(fd - np.sum(g * d)) < 1e-6 * abs(fd)
    # 16 single points
    rng = np.random.default_rng(81)
    flat = rng.choice(h1.size, 16, replace=False)
    for q in flat:
        e = np.zeros(h1.size)
        e[q] = 1.0
        e = e.reshape(h1.shape)
        fdq = (L(h1 + eps * e) - L(h1 - eps * e)) / (2 * eps)
        gq = g.ravel()[q]
        assert abs(fdq - gq) < 1e-6 * max(abs(gq), 1e-3 * np.abs(g).max()), (q, fdq, gq)


def test_gradient_uniform_scaling_closed_form():
    # h2 = 0, h1 = c everywhere: u = u1 / c, so dL/dc = -2 <u1/c - ut, u1> / c^2,
    # which must equal the sum of the per-point gradient.
    m = build((2, 2, 1), 4)
    f = si.eval_fourier(si.fourier_modes(90), m["x"], m["y"], m["z"])
    b = solve.rhs(f, m["B"], m["gid"], m["mask"])
    ut = si.eval_fourier(si.fourier_modes(91), m["x"], m["y"], m["z"]) * 0.1
    c = 1.7
    u1 = forward(m, np.ones(m["gid"].shape), 0.0, b)
    u, g = gradient(m, c * np.ones(m["gid"].shape), 0.0, b, ut)
    np.testing.assert_allclose(u, u1 / c, atol=1e-12 * np.abs(u1).max())
    expect = -2.0 * solve.weighted_dot(u1 / c - ut, u1, m["mult"]) / c ** 2
    assert abs(np.sum(g) - expect) < 1e-9 * abs(expect)
