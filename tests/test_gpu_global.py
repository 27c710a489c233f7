"""GPU parity of the operator on global (unique-dof) vectors, sem_apply_global
(the element kernel gathers u_g and assembles w_g by atomics), of the
L-vector to global conversion, and of mixed-precision solves whose FP32 inner
PCG runs on global vectors, all against the oracle."""
import numpy as np
import pytest
import torch

import paper_2107_01243_gb300 as sem
import seeded_inputs as si
from oracle import mesh
from tests.helpers import OracleProblem, rel_inf, TWO_PI

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
TOL32 = 2e-5

# one element, single-element rows, meshes one element thick, n_G not a
# multiple of 4 (padded vectors), more elements than resident CTAs
CASES = [((5, 3, 3), 7), ((2, 3, 2), 5), ((3, 3, 1), 9), ((1, 2, 2), 9), ((4, 1, 1), 1),
         ((1, 1, 1), 7), ((7, 1, 5), 3), ((2, 2, 2), 7), ((30, 20, 6), 7)]


def make(nel, N, faces=mesh.ALL_FACES):
    h = sem.sem_setup(nel, N, length=(TWO_PI,) * 3, deform=0.1, faces=faces)
    o = OracleProblem(nel, N, length=(TWO_PI,) * 3, deform=0.1, faces=faces)
    return h, o


def apply_global(h, ug, h1, h2):
    ud = torch.from_numpy(np.ascontiguousarray(ug, dtype=np.float32)).to(DEV)
    w = torch.full_like(ud, float("nan"))      # the call clears w_g itself
    sem.sem_apply_global(h, ud, w, h1, h2)
    sem.sem_sync(h)
    return w.double().cpu().numpy()


@pytest.mark.parametrize("nel,N", CASES)
@pytest.mark.parametrize("h1,h2", [(1.0, 0.0), (0.8, 2.5)])
def test_apply_global_matches_oracle(nel, N, h1, h2):
    h, o = make(nel, N)
    ng = sem.sem_get_sizes(h)["n_global"]
    ug = si.uniform((ng,), 71).astype(np.float32).astype(np.float64)
    wg = apply_global(h, ug, h1, h2)
    ref = o.matvec(ug[o.gid], h1, h2)           # continuous L-vector
    # every local copy of g holds the assembled value w_g[g]
    assert rel_inf(wg[o.gid], ref) < TOL32


@pytest.mark.parametrize("faces", [0, mesh.FACE_XMIN | mesh.FACE_ZMAX,
                                   mesh.FACE_YMIN | mesh.FACE_YMAX | mesh.FACE_XMAX])
def test_apply_global_dirichlet_faces(faces):
    h, o = make((3, 2, 4), 7, faces)
    ng = sem.sem_get_sizes(h)["n_global"]
    ug = si.uniform((ng,), 72).astype(np.float32).astype(np.float64)
    wg = apply_global(h, ug, 1.0, 0.3)
    assert rel_inf(wg[o.gid], o.matvec(ug[o.gid], 1.0, 0.3)) < TOL32


def test_apply_global_masked_points_zero():
    h, o = make((3, 3, 2), 5)
    ng = sem.sem_get_sizes(h)["n_global"]
    wg = apply_global(h, si.uniform((ng,), 73), 1.0, 1.0)
    assert np.all(wg[o.gid][o.mask == 0] == 0.0)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("nel,N", [((3, 2, 2), 5), ((4, 1, 3), 7), ((1, 1, 1), 3)])
def test_to_global_takes_a_copy(nel, N, dtype):
    h, o = make(nel, N)
    ng = sem.sem_get_sizes(h)["n_global"]
    ug = si.uniform((ng,), 74)
    u = torch.from_numpy(ug[o.gid]).to(DEV, dtype).view(-1)
    out = torch.full((ng,), float("nan"), dtype=torch.float32, device=DEV)
    sem.sem_to_global(h, u, out)
    sem.sem_sync(h)
    assert np.array_equal(out.cpu().numpy(), ug.astype(np.float32 if dtype == torch.float32
                                                       else np.float64).astype(np.float32))


def test_apply_global_rejects_bad_arguments():
    h, _ = make((2, 2, 2), 4)                   # even N: odd P, no bulk copies
    ng = sem.sem_get_sizes(h)["n_global"]
    u = torch.zeros(ng, dtype=torch.float32, device=DEV)
    w = torch.zeros_like(u)
    with pytest.raises(sem.SemError):
        sem.sem_apply_global(h, u, w)
    h, _ = make((2, 2, 2), 5)
    ng = sem.sem_get_sizes(h)["n_global"]
    u = torch.zeros(ng, dtype=torch.float32, device=DEV)
    with pytest.raises(sem.SemError):
        sem.sem_apply_global(h, u, u)


# mixed-precision solves: global inner vectors against the oracle's residual
SOLVES = [((4, 3, 3), 7, 0.0, mesh.ALL_FACES), ((3, 3, 2), 5, 2.0, mesh.ALL_FACES),
          ((2, 2, 5), 9, 0.5, mesh.FACE_XMIN | mesh.FACE_YMAX), ((6, 5, 4), 3, 1.0, mesh.ALL_FACES),
          ((5, 4, 3), 7, 3.0, mesh.FACE_ZMIN)]


@pytest.mark.parametrize("nel,N,lam,faces", SOLVES)
@pytest.mark.parametrize("use_graph", [True, False])
def test_mixed_solve_global_inner(nel, N, lam, faces, use_graph):
    h, o = make(nel, N, faces)
    sem.sem_set_inner_vectors(h, sem.SEM_INNER_GLOBAL)
    f = si.eval_fourier(si.fourier_modes(3000 + N), o.x, o.y, o.z)
    b = o.rhs(f)
    bd = torch.from_numpy(b).to(DEV).view(-1)
    x = torch.empty_like(bd)
    info = sem.sem_cg_solve(h, bd, x, h1=1.0, h2=lam, tol=1e-8, precision=sem.SEM_SOLVE_MIXED,
                            use_graph=use_graph, check_every=7)
    assert info["status"] == "SEM_OK", info
    res = o.residual(x.cpu().numpy().reshape(o.shape), b, 1.0, lam)
    assert res <= 1.05e-8, res
    assert abs(res - info["rel_res"]) < 1e-12
    # the same problem with local inner vectors converges to the same solution
    sem.sem_set_inner_vectors(h, sem.SEM_INNER_LOCAL)
    xl = torch.empty_like(bd)
    info_l = sem.sem_cg_solve(h, bd, xl, h1=1.0, h2=lam, tol=1e-8,
                              precision=sem.SEM_SOLVE_MIXED)
    assert info_l["status"] == "SEM_OK"
    assert rel_inf(x.cpu().numpy(), xl.cpu().numpy()) < 1e-5
    # both take about the same number of iterations (same arithmetic up to FP32 rounding)
    assert abs(info["iters"] - info_l["iters"]) <= max(3, info_l["iters"] // 10), (info, info_l)


def test_mixed_solve_global_falls_back_with_h1_field():
    h, o = make((3, 2, 2), 5)
    sem.sem_set_inner_vectors(h, sem.SEM_INNER_GLOBAL)
    f = si.eval_fourier(si.fourier_modes(3100), o.x, o.y, o.z)
    b = o.rhs(f)
    h1f = 1.0 + 0.5 * si.uniform(o.shape, 75)
    bd = torch.from_numpy(b).to(DEV).view(-1)
    x = torch.empty_like(bd)
    info = sem.sem_cg_solve(h, bd, x, h1_field=torch.from_numpy(h1f).to(DEV).view(-1), tol=1e-8,
                            precision=sem.SEM_SOLVE_MIXED)
    assert info["status"] == "SEM_OK", info
    assert o.residual(x.cpu().numpy().reshape(o.shape), b, h1_field=h1f) <= 1.05e-8


def test_inner_vectors_rejects_unknown_kind():
    h, _ = make((1, 1, 1), 3)
    with pytest.raises(sem.SemError):
        sem.sem_set_inner_vectors(h, 7)
