"""Full-size parity, in the launch configuration the benchmark times
(autotuned tiles): the throughput mesh (32^3 deformed elements, N=7), the
solve mesh (48^3, N=7, Fourier-mode right-hand side, PCG to 1e-8) and the
adjoint mesh (16^3, N=7).

The oracle cannot hold these meshes, so it works on samples:
  * Ax on sampled elements, each built by the oracle as a one-element box
    placed where the element sits (the deformation is a function of the
    physical position, so this reproduces the element's coordinates);
  * dssum on the whole mesh (a bincount over 16.7M local points);
  * the assembled operator (sem_apply) at every point of the elements that
    3x3x3 patches of elements fully cover (all copies of such a point lie in
    the patch);
  * the solve's assembled residual at the covered points of such patches,
    checked against |r_g| <= ||r|| <= tol ||b||;
  * the dL/dh1 kernel on sampled elements with seeded fields;
  * the adjoint gradient against central finite differences of the loss.
"""
import numpy as np
import pytest
import torch

import paper_2107_01243_gb300 as sem
import seeded_inputs as si
from oracle import adjoint, mesh, operator
from tests.helpers import OracleProblem, rel_inf

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def element_oracle(cfg, e, faces=0):
    """One-element oracle problem at element e of the box mesh cfg."""
    nx, ny, nz = cfg["nel"]
    ex, ey, ez = e % nx, (e // nx) % ny, e // (nx * ny)
    h = [cfg["length"][a] / cfg["nel"][a] for a in range(3)]
    x0 = (ex * h[0], ey * h[1], ez * h[2])
    return OracleProblem((1, 1, 1), cfg["N"], x0=x0, length=tuple(h), deform=cfg["deform"],
                         faces=faces)


def sample_elements(nel, count, seed):
    E = nel[0] * nel[1] * nel[2]
    rng = np.random.default_rng(seed)
    fixed = [0, nel[0] - 1, E - 1, E // 2, nel[0] * nel[1] + nel[0] + 1]
    return sorted(set(fixed) | set(rng.choice(E, count, replace=False).tolist()))


@pytest.fixture(scope="module")
def throughput_handle():
    cfg = si.THROUGHPUT
    h = sem.sem_setup(cfg["nel"], cfg["N"], length=cfg["length"], deform=cfg["deform"])
    sem.sem_autotune(h)
    yield h
    sem.sem_destroy(h)


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-12), (torch.float32, 2e-5)])
def test_ax_sampled_elements_fullsize(throughput_handle, dtype, tol):
    cfg = si.THROUGHPUT
    h = throughput_handle
    p = cfg["N"] + 1
    u = si.uniform((h.E, p, p, p), cfg["seed"])
    if dtype == torch.float32:
        u = u.astype(np.float32).astype(np.float64)
    ud = torch.from_numpy(u).to(DEV, dtype).view(-1)
    w = torch.empty_like(ud)
    sem.sem_ax(h, ud, w)
    sem.sem_sync(h)
    wv = w.view(h.E, p, p, p)
    for e in sample_elements(cfg["nel"], 48, 5):
        o = element_oracle(cfg, e)
        ref = o.ax(u[e:e + 1])
        got = wv[e:e + 1].double().cpu().numpy()
        assert rel_inf(got, ref) < tol, e


def test_dssum_whole_mesh_fullsize(throughput_handle):
    """Box gather-scatter on 16.7M local points: bit-equal to the oracle's
    bincount (both sum the copies of a point in local-index order)."""
    cfg = si.THROUGHPUT
    h = throughput_handle
    N, nel = cfg["N"], cfg["nel"]
    p = N + 1
    w = si.uniform((h.E, p, p, p), 7)
    gid = mesh.global_ids(*nel, N)
    ref = operator.apply_dirichlet(operator.dssum(w, gid), mesh.dirichlet_mask(*nel, N))
    wd = torch.from_numpy(w).to(DEV).view(-1)
    sem.sem_dssum(h, wd, apply_mask=True)
    np.testing.assert_array_equal(wd.cpu().numpy().reshape(w.shape), ref)


def _covered(start, nel):
    """Per axis, the offsets (0..2) of the patch elements whose every
    neighbour in the mesh lies in the 3-element patch starting at start."""
    out = []
    for s, n in zip(start, nel):
        out.append([a for a in range(3)
                    if (s + a - 1 < 0 or a >= 1) and (s + a + 1 >= n or a <= 1)])
    return out


def _patch_oracle(cfg, start):
    """Oracle problem of the 3x3x3 element patch at start, the patch's
    elements in the full mesh (patch order) and the covered ones."""
    nx, ny, nz = cfg["nel"]
    hs = [cfg["length"][a] / cfg["nel"][a] for a in range(3)]
    faces = 0
    faces |= mesh.FACE_XMIN if start[0] == 0 else 0
    faces |= mesh.FACE_XMAX if start[0] + 3 == nx else 0
    faces |= mesh.FACE_YMIN if start[1] == 0 else 0
    faces |= mesh.FACE_YMAX if start[1] + 3 == ny else 0
    faces |= mesh.FACE_ZMIN if start[2] == 0 else 0
    faces |= mesh.FACE_ZMAX if start[2] + 3 == nz else 0
    x0 = tuple(start[a] * hs[a] for a in range(3))
    o = OracleProblem((3, 3, 3), cfg["N"], x0=x0, length=tuple(3 * v for v in hs),
                      deform=cfg["deform"], faces=faces)
    full = [(start[0] + a) + nx * ((start[1] + b) + ny * (start[2] + c))
            for c in range(3) for b in range(3) for a in range(3)]
    cov = _covered(start, cfg["nel"])
    sel = [a + 3 * (b + 3 * c) for c in cov[2] for b in cov[1] for a in cov[0]]
    return o, full, sel


def _patch_residual(cfg, start, x_dev, b_dev, h1=1.0, h2=0.0):
    """Oracle residual b - mask QQ^T A x at every point of the covered
    elements of a 3x3x3 patch; also returns the oracle's b there and the
    GPU's b at the same points."""
    p = cfg["N"] + 1
    o, full, sel = _patch_oracle(cfg, start)
    idx = torch.tensor(full, device=DEV)
    xp = x_dev.view(-1, p, p, p)[idx].cpu().numpy()
    bp_gpu = b_dev.view(-1, p, p, p)[idx].cpu().numpy()
    f = si.eval_fourier(si.fourier_modes(cfg["seed"]), o.x, o.y, o.z)
    bp = o.rhs(f)
    r = bp - o.matvec(xp, h1, h2)
    return r[sel], bp[sel], bp_gpu[sel]


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-12), (torch.float32, 2e-5)])
def test_apply_patches_fullsize(throughput_handle, dtype, tol):
    """The assembled operator (fused element kernel + split gather-scatter)
    on the whole 32^3 mesh, checked by the oracle's assembled operator at
    every point of the elements covered by 3x3x3 patches."""
    cfg = si.THROUGHPUT
    h = throughput_handle
    p = cfg["N"] + 1
    u = si.uniform((h.E, p, p, p), cfg["seed"])
    if dtype == torch.float32:
        u = u.astype(np.float32).astype(np.float64)
    ud = torch.from_numpy(u).to(DEV, dtype).view(-1)
    w = torch.empty_like(ud)
    sem.sem_apply(h, ud, w)
    sem.sem_sync(h)
    wv = w.view(h.E, p, p, p)
    for start in [(0, 0, 0), (13, 7, 21), (29, 29, 29), (0, 15, 29), (30 - 1, 0, 12)]:
        o, full, sel = _patch_oracle(cfg, start)
        ref = o.matvec(u[full])[sel]
        got = wv[torch.tensor(full, device=DEV)].double().cpu().numpy()[sel]
        assert rel_inf(got, ref) < tol, start


@pytest.fixture(scope="module")
def solve_case():
    cfg = si.SOLVE
    h = sem.sem_setup(cfg["nel"], cfg["N"], length=cfg["length"], deform=cfg["deform"])
    sem.sem_autotune(h)
    n = h.n_local
    xyz = [torch.empty(n, dtype=torch.float64, device=DEV) for _ in range(3)]
    for t, which in zip(xyz, (sem.SEM_FIELD_X, sem.SEM_FIELD_Y, sem.SEM_FIELD_Z)):
        sem.sem_get_field(h, which, t)
    X, Y, Z = (t.cpu().numpy() for t in xyz)
    del xyz
    f = torch.from_numpy(si.eval_fourier(si.fourier_modes(cfg["seed"]), X, Y, Z)).to(DEV)
    del X, Y, Z
    b = torch.empty_like(f)
    sem.sem_rhs(h, f, b)
    del f
    yield cfg, h, b
    sem.sem_destroy(h)


PATCHES = [(0, 0, 0), (22, 17, 30), (45, 45, 45), (0, 23, 45)]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_solve_fullsize_patch_residual(solve_case, precision):
    cfg, h, b = solve_case
    prec = sem.SEM_SOLVE_F64 if precision == "fp64" else sem.SEM_SOLVE_MIXED
    x = torch.empty_like(b)
    info = sem.sem_cg_solve(h, b, x, tol=cfg["tol"], precision=prec)
    assert info["status"] == "SEM_OK"
    assert info["rel_res"] <= cfg["tol"]
    # |r_g| <= ||r||_unique <= tol ||b||_unique <= tol sqrt(sum_L b_L^2)
    bound = cfg["tol"] * float(torch.sqrt((b * b).sum()))
    for start in PATCHES:
        r, bref, bgpu = _patch_residual(cfg, start, x, b)
        assert rel_inf(bgpu, bref) < 1e-12, start
        assert np.abs(r).max() <= bound, (start, np.abs(r).max(), bound)


def test_grad_kernel_sampled_elements_fullsize():
    cfg = si.ADJOINT
    h = sem.sem_setup(cfg["nel"], cfg["N"], length=cfg["length"], deform=cfg["deform"])
    p = cfg["N"] + 1
    u = si.uniform((h.E, p, p, p), 11)
    lam = si.uniform((h.E, p, p, p), 12)
    g = torch.empty(h.n_local, dtype=torch.float64, device=DEV)
    sem.sem_helmholtz_grad(h, torch.from_numpy(u).to(DEV).view(-1),
                           torch.from_numpy(lam).to(DEV).view(-1), g)
    gv = g.view(h.E, p, p, p)
    for e in sample_elements(cfg["nel"], 24, 6):
        o = element_oracle(cfg, e)
        ref = adjoint.grad_h1(u[e:e + 1], lam[e:e + 1], o.G, o.D)
        assert rel_inf(gv[e:e + 1].cpu().numpy(), ref) < 1e-12, e
    sem.sem_destroy(h)


def test_adjoint_gradient_fd_fullsize():
    """16^3 deformed elements, N=7, h1 = 1 + 0.5 tanh(smooth field): the
    autograd gradient of ||u - u_target||^2 (unique-dof norm) along a smooth
    direction against central differences, to 1e-6 relative."""
    cfg = si.ADJOINT
    h = sem.sem_setup(cfg["nel"], cfg["N"], length=cfg["length"], deform=cfg["deform"])
    n = h.n_local
    xyz = [torch.empty(n, dtype=torch.float64, device=DEV) for _ in range(3)]
    for t, which in zip(xyz, (sem.SEM_FIELD_X, sem.SEM_FIELD_Y, sem.SEM_FIELD_Z)):
        sem.sem_get_field(h, which, t)
    X, Y, Z = (t.cpu().numpy() for t in xyz)
    h1 = torch.from_numpy(si.smooth_coefficient(X, Y, Z, cfg["h1_seed"])).to(DEV)
    ut = torch.from_numpy(0.01 * si.eval_fourier(si.fourier_modes(cfg["target_seed"]),
                                                 X, Y, Z)).to(DEV)
    f = torch.from_numpy(si.eval_fourier(si.fourier_modes(cfg["rhs_seed"]), X, Y, Z)).to(DEV)
    d = torch.from_numpy(si.eval_fourier(si.fourier_modes(80), X, Y, Z)).to(DEV)
    b = torch.empty_like(f)
    sem.sem_rhs(h, f, b)
    mult = torch.empty_like(b)
    sem.sem_get_field(h, sem.SEM_FIELD_MULT, mult)

    def L(h1v):
        x = torch.empty_like(b)
        sem.sem_cg_solve(h, b, x, h1_field=h1v, h2=1.0, tol=1e-14)
        return float((((x - ut) ** 2) / mult).sum())

    h1_t = h1.clone().requires_grad_(True)
    x = sem.helmholtz_solve(h1_t, b, h, h2=1.0, tol=1e-14)
    (((x - ut) ** 2) / mult).sum().backward()
    gd = float((h1_t.grad * d).sum())
    eps = 1e-5 * float(h1.abs().max())
    fd = (L(h1 + eps * d) - L(h1 - eps * d)) / (2 * eps)
    assert abs(fd - gd) < 1e-6 * abs(fd)
    sem.sem_destroy(h)
