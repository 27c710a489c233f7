"""GPU solves through the C ABI, judged by the oracle: FP64 PCG against the
oracle's PCG (iteration count and solution), mixed-precision refinement
by the oracle's FP64 residual, Jacobi diagonal, status codes, and the
adjoint gradient against the oracle and finite differences."""
import math

import numpy as np
import pytest
import torch

import paper_2107_01243_gb300 as sem
import seeded_inputs as si
from tests.helpers import OracleProblem, rel_inf, TWO_PI

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV, torch.float64).view(-1)


def to_np(t, shape):
    return t.detach().double().cpu().numpy().reshape(shape)


def test_manufactured_poisson_fp64():
    """Unit cube, 4^3 undeformed elements, N=7, PCG to 1e-10 (the manufactured case)."""
    cfg = si.MANUFACTURED
    h = sem.sem_setup(cfg["nel"], cfg["N"], length=cfg["length"], deform=cfg["deform"])
    o = OracleProblem(cfg["nel"], cfg["N"], length=cfg["length"], deform=cfg["deform"])
    f = si.manufactured_f(o.x, o.y, o.z)
    b_ref = o.rhs(f)
    b = torch.empty(h.n_local, dtype=torch.float64, device=DEV)
    sem.sem_rhs(h, to_dev(f), b)
    x = torch.empty_like(b)
    info = sem.sem_cg_solve(h, b, x, tol=cfg["tol"])
    ref = o.pcg(b_ref, tol=cfg["tol"])
    xg = to_np(x, o.shape)
    assert info["status"] == "SEM_OK"
    assert abs(info["iters"] - ref.iters) <= 1
    assert o.residual(xg, b_ref) <= 1.05 * cfg["tol"]
    assert rel_inf(xg, ref.x) < 1e-8
    # discretisation error against the exact solution (spectral accuracy at N=7)
    assert np.abs(xg - si.manufactured_u(o.x, o.y, o.z)).max() < 1e-6
    # the Jacobi inverse diagonal used by the solve
    from oracle import solve
    d = torch.empty_like(b)
    sem.sem_get_field(h, sem.SEM_FIELD_DINV, d)
    dref = solve.jacobi_inverse(o.G, o.D, o.gid, o.mask, B=o.B)
    assert rel_inf(to_np(d, o.shape), dref) < 1e-12


@pytest.mark.parametrize("use_graph", [True, False])
@pytest.mark.parametrize("h2", [0.0, 3.0])
def test_deformed_fp64_matches_oracle_iterates(use_graph, h2):
    nel, N = (3, 3, 2), 5
    h = sem.sem_setup(nel, N, length=(TWO_PI,) * 3, deform=0.1)
    o = OracleProblem(nel, N, length=(TWO_PI,) * 3, deform=0.1)
    f = si.eval_fourier(si.fourier_modes(1234), o.x, o.y, o.z)
    b_ref = o.rhs(f)
    b = to_dev(b_ref)
    x = torch.empty_like(b)
    info = sem.sem_cg_solve(h, b, x, h2=h2, tol=1e-8, use_graph=use_graph, check_every=7)
    ref = o.pcg(b_ref, h2=h2, tol=1e-8)
    assert abs(info["iters"] - ref.iters) <= 1
    xg = to_np(x, o.shape)
    assert o.residual(xg, b_ref, h2=h2) <= 1.05e-8
    assert abs(info["rel_res"] - o.residual(xg, b_ref, h2=h2)) < 1e-12


@pytest.mark.parametrize("nel,N", [((4, 3, 3), 7), ((3, 2, 2), 9), ((4, 4, 2), 5)])
def test_mixed_precision_refinement(nel, N):
    h = sem.sem_setup(nel, N, length=(TWO_PI,) * 3, deform=0.1)
    o = OracleProblem(nel, N, length=(TWO_PI,) * 3, deform=0.1)
    f = si.eval_fourier(si.fourier_modes(1234), o.x, o.y, o.z)
    b_ref = o.rhs(f)
    b = to_dev(b_ref)
    x = torch.empty_like(b)
    info = sem.sem_cg_solve(h, b, x, tol=1e-8, precision=sem.SEM_SOLVE_MIXED, inner_tol=1e-4)
    assert info["status"] == "SEM_OK" and info["outer_iters"] >= 2
    xg = to_np(x, o.shape)
    res = o.residual(xg, b_ref)
    assert res <= 1.05e-8
    assert abs(res - info["rel_res"]) < 1e-12
    ref = o.pcg(b_ref, tol=1e-12)
    assert rel_inf(xg, ref.x) < 1e-6


@pytest.mark.parametrize("precision", [sem.SEM_SOLVE_F64, sem.SEM_SOLVE_MIXED])
@pytest.mark.parametrize("side_stream", [False, True])
def test_initial_guess(precision, side_stream):
    """A solve started from a given x0 (continuous, zero on Dirichlet points):
    the FP64 iterates follow the oracle's PCG started from the same x0, both
    precisions reach the tolerance by the oracle's residual, and on a side
    stream the copy of x0 into x is ordered before the solve (x starts as NaN)."""
    nel, N, tol = (3, 2, 2), 7, 1e-9
    h = sem.sem_setup(nel, N, length=(TWO_PI,) * 3, deform=0.1)
    o = OracleProblem(nel, N, length=(TWO_PI,) * 3, deform=0.1)
    b_ref = o.rhs(si.eval_fourier(si.fourier_modes(1240), o.x, o.y, o.z))
    x0 = si.uniform((int(o.gid.max()) + 1,), 1241)[o.gid] * o.mask
    b, x0d = to_dev(b_ref), to_dev(x0)
    x = torch.full_like(b, float("nan"))
    stream = torch.cuda.Stream() if side_stream else None
    info = sem.sem_cg_solve(h, b, x, tol=tol, precision=precision, x0=x0d, stream=stream)
    torch.cuda.synchronize()
    xg = to_np(x, o.shape)
    assert info["status"] == "SEM_OK", info
    res = o.residual(xg, b_ref)
    assert res <= 1.05 * tol and abs(res - info["rel_res"]) < 1e-12
    if precision == sem.SEM_SOLVE_F64:
        ref = o.pcg(b_ref, tol=tol, x0=x0)
        assert abs(info["iters"] - ref.iters) <= 1, (info, ref.iters)
        assert rel_inf(xg, ref.x) < 1e-7


def test_helmholtz_mass_only_converges_in_one_iteration():
    nel, N = (3, 2, 2), 5
    h = sem.sem_setup(nel, N, length=(TWO_PI,) * 3, deform=0.1)
    o = OracleProblem(nel, N, length=(TWO_PI,) * 3, deform=0.1)
    f = si.eval_fourier(si.fourier_modes(5), o.x, o.y, o.z)
    b = to_dev(o.rhs(f))
    x = torch.empty_like(b)
    info = sem.sem_cg_solve(h, b, x, h1=0.0, h2=2.0, tol=1e-12)
    assert info["iters"] == 1


def test_status_codes():
    nel, N = (2, 2, 2), 3
    h = sem.sem_setup(nel, N, length=(TWO_PI,) * 3, deform=0.1)
    o = OracleProblem(nel, N, length=(TWO_PI,) * 3, deform=0.1)
    b = to_dev(o.rhs(si.eval_fourier(si.fourier_modes(9), o.x, o.y, o.z)))
    x = torch.empty_like(b)
    info = sem.sem_cg_solve(h, b, x, h1=-1.0, raise_on_fail=False)
    assert info["status"] == "SEM_ERR_BREAKDOWN"
    info = sem.sem_cg_solve(h, b, x, tol=1e-14, maxit=3, raise_on_fail=False)
    assert info["status"] == "SEM_ERR_NOCONV" and info["iters"] == 3
    with pytest.raises(sem.SemError):
        sem.sem_cg_solve(h, b, x, tol=1e-14, maxit=3)
    with pytest.raises(sem.SemError) as e:
        sem.sem_setup((2, 2, 2), 11)
    assert e.value.status == 1
    with pytest.raises(sem.SemError):
        sem.sem_ax(h, b, b)                         # aliasing input and output
    with pytest.raises(sem.SemError):
        sem.sem_ax(h, b[:-1], x[:-1])               # wrong size
    # the handle still works after the errors
    sem.sem_cg_solve(h, b, x, tol=1e-10)


def test_zero_rhs_returns_zero():
    h = sem.sem_setup((2, 2, 1), 4)
    b = torch.zeros(h.n_local, dtype=torch.float64, device=DEV)
    x = torch.full_like(b, 3.0)
    info = sem.sem_cg_solve(h, b, x)
    assert info["iters"] == 0 and float(x.abs().max()) == 0.0


def _adjoint_setup(nel, N):
    h = sem.sem_setup(nel, N, length=(TWO_PI,) * 3, deform=0.1)
    o = OracleProblem(nel, N, length=(TWO_PI,) * 3, deform=0.1)
    h1 = si.smooth_coefficient(o.x, o.y, o.z, 77)
    ut = si.eval_fourier(si.fourier_modes(78), o.x, o.y, o.z) * 0.01
    f = si.eval_fourier(si.fourier_modes(79), o.x, o.y, o.z)
    return h, o, h1, ut, o.rhs(f)


def test_adjoint_gradient_matches_oracle():
    from oracle import adjoint, operator
    h, o, h1, ut, b_ref = _adjoint_setup((3, 2, 2), 5)
    h1_t = to_dev(h1).requires_grad_(True)
    x = sem.helmholtz_solve(h1_t, to_dev(b_ref), h, h2=1.0, tol=1e-13)
    mult = to_dev(o.mult)
    loss = (((x - to_dev(ut)) ** 2) / mult).sum()
    loss.backward()
    g = to_np(h1_t.grad, o.shape)
    # oracle: forward solve, adjoint solve, per-point gradient
    u = o.pcg(b_ref, h1_field=h1, h2=1.0, tol=1e-14).x
    rhs_adj = operator.apply_dirichlet(operator.dssum(adjoint.loss_grad_u(u, ut, o.mult), o.gid),
                                       o.mask)
    lam = o.pcg(rhs_adj, h1_field=h1, h2=1.0, tol=1e-14).x
    gref = adjoint.grad_h1(u, lam, o.G, o.D)
    assert rel_inf(g, gref) < 1e-9


def test_adjoint_gradient_finite_differences():
    h, o, h1, ut, b_ref = _adjoint_setup((2, 2, 2), 4)
    b = to_dev(b_ref)
    mult = to_dev(o.mult)
    utd = to_dev(ut)

    def L(h1v):
        x = torch.empty_like(b)
        sem.sem_cg_solve(h, b, x, h1_field=h1v, h2=1.0, tol=1e-14)
        return float((((x - utd) ** 2) / mult).sum())

    h1_t = to_dev(h1).requires_grad_(True)
    x = sem.helmholtz_solve(h1_t, b, h, h2=1.0, tol=1e-14)
    (((x - utd) ** 2) / mult).sum().backward()
    g = h1_t.grad.detach()
    d = to_dev(si.eval_fourier(si.fourier_modes(80), o.x, o.y, o.z))
    eps = 1e-5 * float(np.abs(h1).max())
    base = to_dev(h1)
    fd = (L(base + eps * d) - L(base - eps * d)) / (2 * eps)
    assert abs(fd - float((g * d).sum())) < 1e-6 * abs(fd)


def test_bounded_wait_times_out_and_context_survives():
    """A bulk-copy barrier that can never complete: the kernel gives up after
    the limit, records SEM_ERR_TIMEOUT and returns; the handle keeps working."""
    h = sem.sem_setup((4, 3, 2), 7, length=(TWO_PI,) * 3, deform=0.1)
    assert sem.sem_selftest_timeout(h, 20.0) == "SEM_ERR_TIMEOUT"
    sem.sem_sync(h)                       # the record was cleared
    o = OracleProblem((4, 3, 2), 7, length=(TWO_PI,) * 3, deform=0.1)
    u = si.uniform(o.shape, 3)
    w = torch.empty(h.n_local, dtype=torch.float32, device=DEV)
    sem.sem_ax(h, torch.from_numpy(u).to(DEV, torch.float32), w)
    sem.sem_sync(h)
    ref = o.ax(u.astype(np.float32).astype(np.float64))
    assert rel_inf(w.double().cpu().numpy().reshape(o.shape), ref) < 2e-5
