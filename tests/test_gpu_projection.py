"""Projection onto previous solutions (sem_proj_*) against the oracle's
projection: a sequence of right-hand sides solved with the same space on
both sides (iterations and solutions), the restart of a full space, a
repeated right-hand side, and mixed-precision corrections judged by the
oracle's residual."""
import numpy as np
import pytest
import torch

import paper_2107_01243_gb300 as sem
import seeded_inputs as si
from oracle import projection
from tests.helpers import OracleProblem, rel_inf, TWO_PI

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def setup(nel=(3, 2, 2), N=5, h2=0.5, nrhs=6):
    h = sem.sem_setup(nel, N, length=(TWO_PI,) * 3, deform=0.1)
    o = OracleProblem(nel, N, length=(TWO_PI,) * 3, deform=0.1)
    rhs = [o.rhs(si.eval_fourier(si.fourier_modes(300 + k), o.x, o.y, o.z))
           for k in range(nrhs)]
    return h, o, rhs


@pytest.mark.parametrize("m", [20, 2])
def test_projected_sequence_matches_oracle(m):
    h2, tol = 0.5, 1e-10
    h, o, rhs = setup(h2=h2)
    p = sem.sem_proj_create(h, m)
    proj = projection.Projection(m)
    mv = lambda v: o.matvec(v, 1.0, h2)
    pcg = lambda b, t: o.pcg(b, h2=h2, tol=t)
    for k, b_ref in enumerate(rhs + [rhs[0]]):
        b = torch.from_numpy(b_ref).to(DEV).view(-1)
        x = torch.empty_like(b)
        info = sem.sem_proj_solve(p, b, x, h2=h2, tol=tol)
        x_ref, _, res = projection.solve_projected(proj, b_ref, mv, pcg, o.mult, tol)
        assert info["status"] == "SEM_OK"
        assert abs(info["iters"] - res.iters) <= 1, (k, info, res.iters)
        xg = x.cpu().numpy().reshape(o.shape)
        assert rel_inf(xg, x_ref) < 1e-8, k
        assert o.residual(xg, b_ref, 1.0, h2) <= 1.05 * tol
        assert abs(info["rel_res"] - o.residual(xg, b_ref, 1.0, h2)) < 1e-12
        assert sem.sem_proj_size(p) == len(proj.X), k
    # with room for every solution, the repeated right-hand side (last)
    # needed no correction iterations
    if m >= len(rhs):
        assert info["iters"] <= 1


def test_projected_mixed_precision():
    h2, tol = 0.5, 1e-9
    h, o, rhs = setup(nel=(4, 3, 3), N=7, h2=h2, nrhs=5)
    p = sem.sem_proj_create(h, 20)
    iters = []
    for b_ref in rhs:
        b = torch.from_numpy(b_ref).to(DEV).view(-1)
        x = torch.empty_like(b)
        info = sem.sem_proj_solve(p, b, x, h2=h2, tol=tol, precision=sem.SEM_SOLVE_MIXED)
        assert info["status"] == "SEM_OK"
        assert o.residual(x.cpu().numpy().reshape(o.shape), b_ref, 1.0, h2) <= 1.05 * tol
        iters.append(info["iters"])
    sem.sem_proj_reset(p)
    assert sem.sem_proj_size(p) == 0


def test_projection_rejects_bad_arguments():
    h, o, rhs = setup()
    with pytest.raises(sem.SemError):
        sem.sem_proj_create(h, 65)
