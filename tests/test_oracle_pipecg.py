"""Pins of the pipelined PCG oracle: its iterates follow standard PCG (the
oracle's own recurrence of a different form) for the early iterations, it
converges to the dense solution, and a zero right-hand side stops at once."""
import numpy as np

import seeded_inputs as si
from oracle import pipecg, solve
from tests.helpers import OracleProblem, TWO_PI


def _problem(nel=(3, 2, 2), N=4, h2=0.5):
    o = OracleProblem(nel, N, length=(TWO_PI,) * 3, deform=0.1)
    b = o.rhs(si.eval_fourier(si.fourier_modes(120), o.x, o.y, o.z))
    dinv = solve.jacobi_inverse(o.G, o.D, o.gid, o.mask, 1.0, h2, o.B)
    return o, b, dinv, (lambda v: o.matvec(v, 1.0, h2))


def test_iterates_follow_standard_pcg():
    o, b, dinv, H = _problem()
    hist = []
    pipecg.pipecg(b, H, dinv, o.mult, tol=1e-30, maxit=12, max_restarts=0, history=hist)
    for k in (1, 4, 8, 12):
        ref = solve.pcg(b, o.G, o.D, o.gid, o.mask, o.mult, h2=0.5, B=o.B, tol=1e-30, maxit=k)
        assert np.abs(hist[k - 1] - ref.x).max() <= 1e-9 * np.abs(ref.x).max(), k


def test_converges_to_the_solution():
    o, b, dinv, H = _problem()
    res = pipecg.pipecg(b, H, dinv, o.mult, tol=1e-10)
    assert res.status == "ok"
    ref = solve.pcg(b, o.G, o.D, o.gid, o.mask, o.mult, h2=0.5, B=o.B, tol=1e-13)
    assert np.abs(res.x - ref.x).max() <= 1e-8 * np.abs(ref.x).max()
    assert o.residual(res.x, b, 1.0, 0.5) <= 1.0001e-10
    # the same number of iterations as standard PCG, give or take rounding
    ref10 = solve.pcg(b, o.G, o.D, o.gid, o.mask, o.mult, h2=0.5, B=o.B, tol=1e-10)
    assert abs(res.iters - ref10.iters) <= 2


def test_zero_rhs():
    o, b, dinv, H = _problem((1, 1, 1), 2)
    res = pipecg.pipecg(np.zeros_like(b), H, dinv, o.mult)
    assert res.iters == 0 and np.all(res.x == 0.0)
