"""GPU parity of the assembled operator sem_apply (element kernel with the
x-neighbour sums fused, then the split gather-scatter passes) against the
oracle's mask o QQ^T A_L u, on meshes where the CTA element ranges hold one
element, several whole x-rows, or cut x-rows in the middle."""
import numpy as np
import pytest
import torch

import paper_2107_01243_gb300 as sem
import seeded_inputs as si
from oracle import mesh
from tests.helpers import OracleProblem, rel_inf, TWO_PI

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
TOL64 = 1e-12
TOL32 = 2e-5

# small meshes (one element per CTA), one larger than the FP64 grid (several
# elements per CTA, ranges cutting x-rows), odd orders (fallback path)
CASES = [((5, 3, 3), 7), ((3, 2, 1), 2), ((2, 3, 2), 5), ((3, 3, 1), 9), ((1, 2, 2), 9),
         ((4, 1, 1), 1), ((2, 2, 2), 4), ((1, 1, 1), 7), ((7, 1, 5), 3), ((12, 10, 9), 7)]


def make(nel, N, faces=63):
    h = sem.sem_setup(nel, N, length=(TWO_PI,) * 3, deform=0.1, faces=faces)
    o = OracleProblem(nel, N, length=(TWO_PI,) * 3, deform=0.1, faces=faces)
    return h, o


def run(h, u, dtype, h1=1.0, h2=0.0, h1_field=None, phase="full"):
    ud = torch.from_numpy(np.ascontiguousarray(u)).to(DEV, dtype).view(-1)
    w = torch.empty_like(ud)
    f = (torch.from_numpy(np.ascontiguousarray(h1_field)).to(DEV, dtype).view(-1)
         if h1_field is not None else None)
    if phase == "full":
        sem.sem_apply(h, ud, w, h1, h2, h1_field=f)
    else:
        sem.sem_apply(h, ud, w, h1, h2, h1_field=f, phase=sem.SEM_APPLY_LOCAL)
        sem.sem_apply(h, ud, w, h1, h2, h1_field=f, phase=sem.SEM_APPLY_FINISH)
    sem.sem_sync(h)
    return w.double().cpu().numpy()


@pytest.mark.parametrize("nel,N", CASES)
@pytest.mark.parametrize("h1,h2", [(1.0, 0.0), (0.8, 2.5)])
def test_apply_fp64(nel, N, h1, h2):
    h, o = make(nel, N)
    u = si.uniform(o.shape, 61)
    got = run(h, u, torch.float64, h1, h2).reshape(o.shape)
    assert rel_inf(got, o.matvec(u, h1, h2)) < TOL64


@pytest.mark.parametrize("nel,N", CASES)
def test_apply_fp32(nel, N):
    h, o = make(nel, N)
    u = si.uniform(o.shape, 62).astype(np.float32).astype(np.float64)
    got = run(h, u, torch.float32, 1.0, 1.5).reshape(o.shape)
    assert rel_inf(got, o.matvec(u, 1.0, 1.5)) < TOL32


@pytest.mark.parametrize("faces", [0, mesh.FACE_XMIN | mesh.FACE_YMAX, mesh.FACE_ZMIN | mesh.FACE_XMAX])
def test_apply_face_subsets(faces):
    h, o = make((6, 4, 5), 7, faces=faces)
    u = si.uniform(o.shape, 63)
    assert rel_inf(run(h, u, torch.float64).reshape(o.shape), o.matvec(u)) < TOL64
    u32 = u.astype(np.float32).astype(np.float64)
    assert rel_inf(run(h, u32, torch.float32).reshape(o.shape), o.matvec(u32)) < TOL32


def test_apply_split_phases_equal_full():
    h, o = make((12, 10, 9), 7)
    u = si.uniform(o.shape, 64)
    for dtype in (torch.float64, torch.float32):
        a = run(h, u, dtype)
        b = run(h, u, dtype, phase="split")
        np.testing.assert_array_equal(a, b)


def test_apply_variable_coefficient_fp32_and_native_fp64():
    """FP32 with a per-point h1 (fused kernel) and FP64 with a per-point h1
    or the native kernel (the unfused fallback)."""
    h, o = make((9, 4, 3), 7)
    u = si.uniform(o.shape, 65)
    h1 = si.smooth_coefficient(o.x, o.y, o.z, 77)
    u32 = u.astype(np.float32).astype(np.float64)
    h1_32 = h1.astype(np.float32).astype(np.float64)
    got = run(h, u32, torch.float32, 0.0, 1.0, h1_field=h1_32).reshape(o.shape)
    assert rel_inf(got, o.matvec(u32, 0.0, 1.0, h1_32)) < TOL32
    got = run(h, u, torch.float64, 0.0, 1.0, h1_field=h1).reshape(o.shape)
    assert rel_inf(got, o.matvec(u, 0.0, 1.0, h1)) < TOL64
    sem.sem_set_f64_kernel(h, sem.SEM_F64_KERNEL_NATIVE)
    got = run(h, u, torch.float64, 1.0, 0.5).reshape(o.shape)
    assert rel_inf(got, o.matvec(u, 1.0, 0.5)) < TOL64


def test_apply_rejects_bad_phase_and_aliasing():
    h, o = make((2, 2, 2), 7)
    u = torch.zeros(h.n_local, dtype=torch.float64, device=DEV)
    w = torch.empty_like(u)
    with pytest.raises(sem.SemError):
        sem.sem_apply(h, u, w, phase=0)
    with pytest.raises(sem.SemError):
        sem.sem_apply(h, u, u)
