"""GPU parity of the two-level Schwarz preconditioner (each level and both)
and of flexible GMRES (Jacobi or Schwarz preconditioned) against the oracle.

The preconditioner runs in FP32 (FP64 in and out): its output is compared
with the FP64 oracle to 2e-5 of its largest value for the local level (six
FP32 contractions of length N + 3 and a diagonal scaling) and to 1e-4 for
the coarse level, whose ten CG iterations are a nonlinear function of an
FP32-rounded restriction; with the coarse CG run to convergence both sides
reach A_0^-1 R_0 r and agree to 2e-5."""
import numpy as np
import pytest
import torch

import paper_2107_01243_gb300 as sem
import seeded_inputs as si
from oracle import mesh, solve, gmres
from oracle.schwarz import Schwarz
from tests.helpers import OracleProblem, rel_inf, TWO_PI

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
L = (TWO_PI,) * 3

CASES = [((3, 2, 2), 3, mesh.ALL_FACES), ((2, 3, 2), 5, mesh.ALL_FACES),
         ((3, 3, 2), 7, mesh.FACE_XMIN | mesh.FACE_YMAX | mesh.FACE_ZMIN), ((1, 1, 1), 7, 63),
         ((4, 1, 2), 9, mesh.ALL_FACES), ((2, 2, 3), 4, 0), ((5, 4, 3), 7, mesh.ALL_FACES),
         ((2, 1, 1), 2, mesh.FACE_XMIN), ((3, 2, 2), 9, mesh.ALL_FACES),
         ((2, 2, 2), 10, mesh.FACE_YMIN | mesh.FACE_ZMAX)]


def make(nel, N, faces, h1=1.0, h2=0.0, coarse_iters=10):
    h = sem.sem_setup(nel, N, length=L, deform=0.1, faces=faces)
    o = OracleProblem(nel, N, length=L, deform=0.1, faces=faces)
    sw = Schwarz(nel, N, o.G, o.B, length=L, faces=faces, h1=h1, h2=h2,
                 coarse_iters=coarse_iters)
    return h, o, sw


def residual_vector(o, seed):
    ng = o.gid.max() + 1
    return si.uniform((ng,), seed)[o.gid] * o.mask


def gpu_apply(h, r, levels, h1=1.0, h2=0.0, coarse_iters=10):
    pre = sem.sem_schwarz_create(h, h1, h2, levels=levels, coarse_iters=coarse_iters)
    rd = torch.from_numpy(np.ascontiguousarray(r)).to(DEV).view(-1)
    z = torch.full_like(rd, float("nan"))
    sem.sem_schwarz_apply(pre, rd, z)
    sem.sem_sync(h)
    return z.cpu().numpy().reshape(r.shape)


@pytest.mark.parametrize("nel,N,faces", CASES)
@pytest.mark.parametrize("h2", [0.0, 1.5])
def test_local_level_matches_oracle(nel, N, faces, h2):
    h, o, sw = make(nel, N, faces, h2=h2)
    r = residual_vector(o, 110)
    ref = sw.local(sw.to_global(r)).reshape(-1)[o.gid] * o.mask
    got = gpu_apply(h, r, sem.SEM_SCHWARZ_LOCAL, h2=h2)
    assert rel_inf(got, ref) < 2e-5


@pytest.mark.parametrize("nel,N,faces", CASES)
def test_coarse_level_matches_oracle(nel, N, faces):
    h, o, sw = make(nel, N, faces, h2=0.4)
    r = residual_vector(o, 111)
    ref = sw.prolong(sw.coarse_solve(sw.restrict(r))) * o.mask
    got = gpu_apply(h, r, sem.SEM_SCHWARZ_COARSE, h2=0.4)
    if np.abs(ref).max() == 0.0:          # no free vertex: the coarse level is empty
        assert np.abs(got).max() == 0.0
        return
    assert rel_inf(got, ref) < 1e-4


@pytest.mark.parametrize("nel,N,faces", [((3, 3, 2), 5, mesh.ALL_FACES), ((4, 2, 3), 3, 0)])
def test_coarse_level_converged_matches_dense_solve(nel, N, faces):
    h, o, sw = make(nel, N, faces, h2=0.4)
    r = residual_vector(o, 112)
    ref = sw.prolong(sw.coarse_dense_solve(sw.restrict(r))) * o.mask
    got = gpu_apply(h, r, sem.SEM_SCHWARZ_COARSE, h2=0.4, coarse_iters=300)
    assert rel_inf(got, ref) < 2e-5


@pytest.mark.parametrize("nel,N,faces", CASES[:5])
def test_both_levels_match_oracle(nel, N, faces):
    h, o, sw = make(nel, N, faces, h2=0.8)
    r = residual_vector(o, 113)
    got = gpu_apply(h, r, sem.SEM_SCHWARZ_BOTH, h2=0.8)
    assert rel_inf(got, sw.apply(r)) < 1e-4
    assert np.all(got[o.mask == 0] == 0.0)


def test_schwarz_rejects_bad_arguments():
    h = sem.sem_setup((2, 2, 2), 3)
    with pytest.raises(sem.SemError):
        sem.sem_schwarz_create(h, 1.0, 0.0, levels=0)
    with pytest.raises(sem.SemError):
        sem.sem_schwarz_create(h, 0.0, 1.0)
    with pytest.raises(sem.SemError):               # N = 1: the growth reaches the next vertex
        sem.sem_schwarz_create(sem.sem_setup((2, 2, 2), 1))
    pre = sem.sem_schwarz_create(h)
    v = torch.zeros(h.n_local, dtype=torch.float64, device=DEV)
    with pytest.raises(sem.SemError):
        sem.sem_schwarz_apply(pre, v, v)


# N = 9, 10: grown boxes of 12^2, 13^2 columns (more than 128 threads per CTA)
SOLVES = [((3, 3, 2), 5, 0.0, mesh.ALL_FACES), ((4, 3, 3), 7, 1.0, mesh.ALL_FACES),
          ((2, 2, 4), 3, 0.0, mesh.FACE_XMIN | mesh.FACE_ZMAX),
          ((5, 2, 3), 9, 0.2, mesh.FACE_XMIN | mesh.FACE_ZMAX)]


@pytest.mark.parametrize("nel,N,h2,faces", SOLVES)
@pytest.mark.parametrize("restart", [30, 6])
def test_gmres_schwarz_matches_oracle(nel, N, h2, faces, restart):
    h, o, sw = make(nel, N, faces, h2=h2)
    b = o.rhs(si.eval_fourier(si.fourier_modes(4000 + N), o.x, o.y, o.z))
    bd = torch.from_numpy(b).to(DEV).view(-1)
    x = torch.empty_like(bd)
    pre = sem.sem_schwarz_create(h, 1.0, h2)
    info = sem.sem_gmres_solve(h, bd, x, h2=h2, tol=1e-9, restart=restart, precond=pre)
    assert info["status"] == "SEM_OK", info
    res = o.residual(x.cpu().numpy().reshape(o.shape), b, 1.0, h2)
    assert res <= 1.0001e-9
    assert abs(res - info["rel_res"]) < 1e-12
    ref = gmres.fgmres(b, lambda v: o.matvec(v, 1.0, h2), sw.apply, o.mult, tol=1e-9, m=restart,
                       maxit=2000)
    assert ref.status == "ok"
    # the FP32 preconditioner changes the Krylov space slightly
    assert abs(info["iters"] - ref.iters) <= max(2, ref.iters // 10), (info, ref.iters)
    assert rel_inf(x.cpu().numpy().reshape(o.shape), ref.x) < 1e-6


@pytest.mark.parametrize("nel,N,h2", [((3, 2, 2), 5, 0.0), ((2, 3, 3), 7, 2.0)])
def test_gmres_jacobi_matches_oracle(nel, N, h2):
    h, o, _ = make(nel, N, mesh.ALL_FACES, h2=h2)
    b = o.rhs(si.eval_fourier(si.fourier_modes(4100 + N), o.x, o.y, o.z))
    bd = torch.from_numpy(b).to(DEV).view(-1)
    x = torch.empty_like(bd)
    info = sem.sem_gmres_solve(h, bd, x, h2=h2, tol=1e-9, restart=20)
    assert info["status"] == "SEM_OK", info
    dinv = solve.jacobi_inverse(o.G, o.D, o.gid, o.mask, 1.0, h2, o.B)
    ref = gmres.fgmres(b, lambda v: o.matvec(v, 1.0, h2), lambda v: dinv * v, o.mult, tol=1e-9,
                       m=20, maxit=5000)
    assert abs(info["iters"] - ref.iters) <= 1, (info, ref.iters)
    assert o.residual(x.cpu().numpy().reshape(o.shape), b, 1.0, h2) <= 1.0001e-9


def test_gmres_zero_rhs_and_errors():
    h, o, _ = make((2, 2, 2), 3, mesh.ALL_FACES)
    b = torch.zeros(h.n_local, dtype=torch.float64, device=DEV)
    x = torch.full_like(b, 3.0)
    info = sem.sem_gmres_solve(h, b, x)
    assert info["status"] == "SEM_OK" and info["iters"] == 0
    assert float(x.abs().max()) == 0.0
    with pytest.raises(sem.SemError):
        sem.sem_gmres_solve(h, b, x, restart=0)
    h2 = sem.sem_setup((2, 2, 2), 3)
    other = sem.sem_schwarz_create(h2)
    with pytest.raises(sem.SemError):
        sem.sem_gmres_solve(h, b, x, precond=other)


@pytest.mark.parametrize("nel,N,h2,faces", [((3, 3, 2), 5, 0.0, mesh.ALL_FACES),
                                            ((4, 3, 3), 7, 1.0, mesh.ALL_FACES),
                                            ((5, 2, 3), 9, 0.2, mesh.FACE_XMIN | mesh.FACE_ZMAX),
                                            ((4, 4, 4), 3, 0.0, mesh.ALL_FACES)])
def test_gmres_mixed_precision(nel, N, h2, faces):
    """FP32 inner FGMRES on global vectors with the Schwarz preconditioner inside
    FP64 refinement: the oracle's FP64 residual reaches the tolerance and the
    solution matches the FP64 GMRES solution."""
    h, o, _ = make(nel, N, faces, h2=h2)
    b = o.rhs(si.eval_fourier(si.fourier_modes(4200 + N), o.x, o.y, o.z))
    bd = torch.from_numpy(b).to(DEV).view(-1)
    pre = sem.sem_schwarz_create(h, 1.0, h2)
    x = torch.empty_like(bd)
    info = sem.sem_gmres_solve(h, bd, x, h2=h2, tol=1e-9, restart=10, precond=pre,
                               precision=sem.SEM_SOLVE_MIXED)
    assert info["status"] == "SEM_OK", info
    assert info["outer_iters"] >= 1
    res = o.residual(x.cpu().numpy().reshape(o.shape), b, 1.0, h2)
    assert res <= 1.0001e-9
    assert abs(res - info["rel_res"]) < 1e-12
    x64 = torch.empty_like(bd)
    sem.sem_gmres_solve(h, bd, x64, h2=h2, tol=1e-9, restart=10, precond=pre)
    assert rel_inf(x.cpu().numpy(), x64.cpu().numpy()) < 1e-6
