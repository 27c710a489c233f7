"""GPU parity of the pipelined FP64 PCG (sem_set_cg_variant) against the
oracle's pipelined PCG: iteration counts, the oracle's residual of the
returned x, and agreement with the standard PCG solution."""
import numpy as np
import pytest
import torch

import paper_2107_01243_gb300 as sem
import seeded_inputs as si
from oracle import mesh, pipecg, solve
from tests.helpers import OracleProblem, rel_inf, TWO_PI

pytestmark = pytest.mark.gpu
DEV = "cuda:0"

CASES = [((3, 3, 2), 5, 0.0, mesh.ALL_FACES), ((4, 3, 3), 7, 1.0, mesh.ALL_FACES),
         ((2, 3, 2), 4, 0.3, mesh.FACE_XMIN | mesh.FACE_YMAX), ((5, 2, 2), 3, 2.0, 63),
         ((1, 1, 1), 7, 0.0, 63)]


@pytest.mark.parametrize("nel,N,h2,faces", CASES)
@pytest.mark.parametrize("use_graph", [True, False])
def test_pipelined_cg_matches_oracle(nel, N, h2, faces, use_graph):
    h = sem.sem_setup(nel, N, length=(TWO_PI,) * 3, deform=0.1, faces=faces)
    o = OracleProblem(nel, N, length=(TWO_PI,) * 3, deform=0.1, faces=faces)
    b = o.rhs(si.eval_fourier(si.fourier_modes(5000 + N), o.x, o.y, o.z))
    bd = torch.from_numpy(b).to(DEV).view(-1)
    sem.sem_set_cg_variant(h, sem.SEM_CG_PIPELINED)
    x = torch.empty_like(bd)
    info = sem.sem_cg_solve(h, bd, x, h2=h2, tol=1e-9, use_graph=use_graph, check_every=5)
    assert info["status"] == "SEM_OK", info
    res = o.residual(x.cpu().numpy().reshape(o.shape), b, 1.0, h2)
    assert res <= 1.0001e-9
    assert abs(res - info["rel_res"]) < 1e-12
    dinv = solve.jacobi_inverse(o.G, o.D, o.gid, o.mask, 1.0, h2, o.B)
    ref = pipecg.pipecg(b, lambda v: o.matvec(v, 1.0, h2), dinv, o.mult, tol=1e-9)
    assert ref.status == "ok"
    assert abs(info["iters"] - ref.iters) <= 2, (info, ref.iters)
    # the standard recurrences reach the same solution
    sem.sem_set_cg_variant(h, sem.SEM_CG_STANDARD)
    xs = torch.empty_like(bd)
    info_s = sem.sem_cg_solve(h, bd, xs, h2=h2, tol=1e-9)
    assert abs(info_s["iters"] - info["iters"]) <= 3, (info_s, info)
    assert rel_inf(x.cpu().numpy(), xs.cpu().numpy()) < 1e-6


def test_pipelined_cg_with_h1_field_and_errors():
    nel, N = (3, 2, 2), 5
    h = sem.sem_setup(nel, N, length=(TWO_PI,) * 3, deform=0.1)
    o = OracleProblem(nel, N, length=(TWO_PI,) * 3, deform=0.1)
    b = o.rhs(si.eval_fourier(si.fourier_modes(5100), o.x, o.y, o.z))
    h1f = 1.0 + 0.5 * si.uniform(o.shape, 121)
    sem.sem_set_cg_variant(h, sem.SEM_CG_PIPELINED)
    bd = torch.from_numpy(b).to(DEV).view(-1)
    x = torch.empty_like(bd)
    info = sem.sem_cg_solve(h, bd, x, h1_field=torch.from_numpy(h1f).to(DEV).view(-1), tol=1e-9)
    assert info["status"] == "SEM_OK", info
    assert o.residual(x.cpu().numpy().reshape(o.shape), b, h1_field=h1f) <= 1.0001e-9
    with pytest.raises(sem.SemError):
        sem.sem_set_cg_variant(h, 5)
    # a zero right-hand side returns x = 0 without iterating
    z = torch.zeros_like(bd)
    info0 = sem.sem_cg_solve(h, z, x)
    assert info0["iters"] == 0 and float(x.abs().max()) == 0.0
