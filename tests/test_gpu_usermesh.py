"""Meshes from user GLL coordinates (sem_mesh_desc.xyz_gll): a box topology
with a map the library does not generate (a twisted, graded box).  The
oracle computes geometry, operator and solve from the same coordinates."""
import numpy as np
import pytest
import torch

import paper_2107_01243_gb300 as sem
import seeded_inputs as si
from oracle import mesh, geometry, operator, solve
from oracle.gll import deriv_matrix
from tests.helpers import rel_inf

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def twisted(nel, N):
    """Graded unit box, twisted about z and bulged: a smooth map with
    non-constant Jacobian that keeps det J > 0."""
    x, y, z = mesh.box_coords(*nel, N, (0.0, 0.0, 0.0), (1.0, 1.0, 1.0), 0.0)
    xg = x + 0.2 * x * (1.0 - x)                 # grading in x
    th = 0.4 * z
    xc, yc = xg - 0.5, y - 0.5
    X = 0.5 + np.cos(th) * xc - np.sin(th) * yc
    Y = 0.5 + np.sin(th) * xc + np.cos(th) * yc
    Z = z + 0.05 * np.sin(np.pi * xg) * np.sin(np.pi * y)
    return X, Y, Z


@pytest.mark.parametrize("nel,N", [((4, 3, 2), 7), ((3, 2, 3), 5), ((2, 2, 2), 4)])
def test_user_coordinates_geometry_and_operator(nel, N):
    X, Y, Z = twisted(nel, N)
    xyz = np.concatenate([X.ravel(), Y.ravel(), Z.ravel()])
    h = sem.sem_setup(nel, N, xyz=xyz)
    G, B, _ = geometry.geom_factors(X, Y, Z, N)
    D = deriv_matrix(N)
    gid = mesh.global_ids(*nel, N)
    mask = mesh.dirichlet_mask(*nel, N)
    n = h.n_local
    g = torch.empty(6 * n, dtype=torch.float64, device=DEV)
    sem.sem_get_field(h, sem.SEM_FIELD_G, g)
    gg = g.cpu().numpy().reshape(gid.shape[0], 6, *gid.shape[1:]).transpose(1, 0, 2, 3, 4)
    assert rel_inf(gg, G) < 1e-12
    u = si.uniform(gid.shape, 31)
    ud = torch.from_numpy(u).to(DEV).view(-1)
    w = torch.empty_like(ud)
    sem.sem_apply(h, ud, w, 1.0, 0.6)
    ref = operator.matvec(u, G, D, gid, mask, 1.0, 0.6, B)
    assert rel_inf(w.cpu().numpy().reshape(gid.shape), ref) < 1e-12


def test_user_coordinates_solve():
    nel, N = (4, 3, 3), 7
    X, Y, Z = twisted(nel, N)
    xyz = np.concatenate([X.ravel(), Y.ravel(), Z.ravel()])
    h = sem.sem_setup(nel, N, xyz=xyz)
    G, B, _ = geometry.geom_factors(X, Y, Z, N)
    D = deriv_matrix(N)
    gid = mesh.global_ids(*nel, N)
    mask = mesh.dirichlet_mask(*nel, N)
    mult = mesh.multiplicity(gid)
    f = si.eval_fourier(si.fourier_modes(41), X, Y, Z)
    b_ref = solve.rhs(f, B, gid, mask)
    b = torch.from_numpy(b_ref).to(DEV).view(-1)
    for prec in (sem.SEM_SOLVE_F64, sem.SEM_SOLVE_MIXED):
        x = torch.empty_like(b)
        info = sem.sem_cg_solve(h, b, x, h2=0.5, tol=1e-9, precision=prec)
        assert info["status"] == "SEM_OK"
        res = solve.residual(x.cpu().numpy().reshape(gid.shape), b_ref, G, D, gid, mask, mult,
                             1.0, 0.5, B)
        assert res <= 1.05e-9


def _user_problem(nel, N):
    X, Y, Z = twisted(nel, N)
    xyz = np.concatenate([X.ravel(), Y.ravel(), Z.ravel()])
    h = sem.sem_setup(nel, N, xyz=xyz)
    G, B, _ = geometry.geom_factors(X, Y, Z, N)
    gid = mesh.global_ids(*nel, N)
    return h, (X, Y, Z), G, B, deriv_matrix(N), gid, mesh.dirichlet_mask(*nel, N), \
        mesh.multiplicity(gid)


def test_user_coordinates_global_operator():
    nel, N = (3, 4, 2), 7
    h, _, G, B, D, gid, mask, _ = _user_problem(nel, N)
    ug = si.uniform((int(gid.max()) + 1,), 32).astype(np.float32).astype(np.float64)
    ud = torch.from_numpy(ug).to(DEV, torch.float32)
    w = torch.empty_like(ud)
    sem.sem_apply_global(h, ud, w, 1.0, 0.6)
    ref = operator.matvec(ug[gid], G, D, gid, mask, 1.0, 0.6, B)
    assert rel_inf(w.double().cpu().numpy()[gid], ref) < 2e-5


def test_user_coordinates_pressure_and_pipelined_solvers():
    """GMRES with the Schwarz preconditioner (whose local solves use the box
    spacing of the mesh description, here the unit box) and the pipelined
    PCG on the twisted mesh, against the oracle."""
    from oracle import gmres
    from oracle.schwarz import Schwarz
    nel, N, h2 = (4, 3, 3), 5, 0.5
    h, (X, Y, Z), G, B, D, gid, mask, mult = _user_problem(nel, N)
    f = si.eval_fourier(si.fourier_modes(42), X, Y, Z)
    b_ref = solve.rhs(f, B, gid, mask)
    b = torch.from_numpy(b_ref).to(DEV).view(-1)
    H = lambda v: operator.matvec(v, G, D, gid, mask, 1.0, h2, B)
    pre = sem.sem_schwarz_create(h, 1.0, h2)
    x = torch.empty_like(b)
    info = sem.sem_gmres_solve(h, b, x, h2=h2, tol=1e-9, restart=10, precond=pre)
    assert info["status"] == "SEM_OK", info
    res = solve.residual(x.cpu().numpy().reshape(gid.shape), b_ref, G, D, gid, mask, mult, 1.0,
                         h2, B)
    assert res <= 1.0001e-9
    sw = Schwarz(nel, N, G, B, length=(1.0, 1.0, 1.0), h2=h2)
    ref = gmres.fgmres(b_ref, H, sw.apply, mult, tol=1e-9, m=10, maxit=2000)
    assert abs(info["iters"] - ref.iters) <= max(2, ref.iters // 10), (info, ref.iters)
    sem.sem_set_cg_variant(h, sem.SEM_CG_PIPELINED)
    xp = torch.empty_like(b)
    info_p = sem.sem_cg_solve(h, b, xp, h2=h2, tol=1e-9)
    assert info_p["status"] == "SEM_OK", info_p
    assert solve.residual(xp.cpu().numpy().reshape(gid.shape), b_ref, G, D, gid, mask, mult, 1.0,
                          h2, B) <= 1.0001e-9
