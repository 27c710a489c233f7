"""GPU parity: the CUDA path against the oracle, element by element, through
the C ABI, on meshes that span several CTAs and end in a ragged tail."""
import numpy as np
import pytest
import torch

import paper_2107_01243_gb300 as sem
import seeded_inputs as si
from tests.helpers import OracleProblem, rel_inf, TWO_PI

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
TOL64 = 1e-12          # FP64 Ax / dssum / geometry: relative to the max norm
TOL32 = 2e-5           # FP32 Ax against the FP64 oracle (24-bit significand, ~3P-term sums)


def to_dev(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV, dtype)


def to_np(t):
    return t.detach().double().cpu().numpy()


def make(nel, N, deform=0.1, length=(TWO_PI,) * 3, faces=63):
    h = sem.sem_setup(nel, N, length=length, deform=deform, faces=faces)
    o = OracleProblem(nel, N, length=length, deform=deform, faces=faces)
    return h, o


CASES = [((5, 3, 3), 7), ((3, 2, 1), 2), ((2, 3, 2), 5), ((3, 3, 1), 9), ((1, 2, 2), 10),
         ((4, 1, 1), 1), ((2, 2, 2), 4), ((1, 1, 1), 7)]


@pytest.mark.parametrize("nel,N", CASES)
def test_geometry(nel, N):
    h, o = make(nel, N)
    n = h.n_local
    for which, ref in ((sem.SEM_FIELD_X, o.x), (sem.SEM_FIELD_Y, o.y), (sem.SEM_FIELD_Z, o.z),
                       (sem.SEM_FIELD_B, o.B)):
        t = torch.empty(n, dtype=torch.float64, device=DEV)
        sem.sem_get_field(h, which, t)
        assert rel_inf(to_np(t).reshape(o.shape), ref) < TOL64
    g = torch.empty(6 * n, dtype=torch.float64, device=DEV)
    sem.sem_get_field(h, sem.SEM_FIELD_G, g)
    gg = to_np(g).reshape(o.shape[0], 6, *o.shape[1:]).transpose(1, 0, 2, 3, 4)
    assert rel_inf(gg, o.G) < TOL64
    gid = torch.empty(n, dtype=torch.int64, device=DEV)
    sem.sem_get_field(h, sem.SEM_FIELD_GID, gid)
    np.testing.assert_array_equal(gid.cpu().numpy().reshape(o.shape), o.gid)
    m = torch.empty(n, dtype=torch.float64, device=DEV)
    sem.sem_get_field(h, sem.SEM_FIELD_MULT, m)
    np.testing.assert_array_equal(to_np(m).reshape(o.shape), o.mult)
    sem.sem_get_field(h, sem.SEM_FIELD_MASK, m)
    np.testing.assert_array_equal(to_np(m).reshape(o.shape), o.mask)


@pytest.mark.parametrize("nel,N", CASES)
@pytest.mark.parametrize("h1,h2", [(1.0, 0.0), (0.8, 2.5)])
def test_ax_fp64(nel, N, h1, h2):
    h, o = make(nel, N)
    u = si.uniform(o.shape, 42)
    w = torch.empty(h.n_local, dtype=torch.float64, device=DEV)
    sem.sem_ax(h, to_dev(u).view(-1), w, h1, h2)
    torch.cuda.synchronize()
    assert rel_inf(to_np(w).reshape(o.shape), o.ax(u, h1, h2)) < TOL64


@pytest.mark.parametrize("nel,N", [((5, 3, 3), 7), ((2, 3, 2), 5), ((3, 3, 1), 9)])
def test_ax_variable_coefficient(nel, N):
    h, o = make(nel, N)
    u = si.uniform(o.shape, 7)
    h1 = si.smooth_coefficient(o.x, o.y, o.z, 77)
    for dtype, tol in ((torch.float64, TOL64), (torch.float32, TOL32)):
        w = torch.empty(h.n_local, dtype=dtype, device=DEV)
        sem.sem_ax(h, to_dev(u, dtype).view(-1), w, 0.0, 1.0, h1_field=to_dev(h1, dtype).view(-1))
        assert rel_inf(to_np(w).reshape(o.shape), o.ax(u, 0.0, 1.0, h1)) < tol


@pytest.mark.parametrize("nel,N", CASES)
def test_ax_fp32(nel, N):
    h, o = make(nel, N)
    u = si.uniform(o.shape, 43)
    w = torch.empty(h.n_local, dtype=torch.float32, device=DEV)
    sem.sem_ax(h, to_dev(u, torch.float32).view(-1), w)
    # the oracle sees the same FP32-rounded input
    ref = o.ax(u.astype(np.float32).astype(np.float64))
    assert rel_inf(to_np(w).reshape(o.shape), ref) < TOL32


@pytest.mark.parametrize("nel,N", CASES)
@pytest.mark.parametrize("apply_mask", [False, True])
@pytest.mark.parametrize("kind", ["box", "segments"])
def test_dssum_fp64_bitexact(nel, N, apply_mask, kind):
    from oracle import operator
    h, o = make(nel, N)
    sem.sem_set_dssum_kernel(h, sem.SEM_DSSUM_BOX if kind == "box" else sem.SEM_DSSUM_SEGMENTS)
    w0 = si.uniform(o.shape, 44)
    w = to_dev(w0).view(-1).clone()
    sem.sem_dssum(h, w, apply_mask=apply_mask)
    ref = operator.dssum(w0, o.gid)
    if apply_mask:
        ref = operator.apply_dirichlet(ref, o.mask)
    # same summation order (increasing local index) on both sides: bitwise equal
    np.testing.assert_array_equal(to_np(w).reshape(o.shape), ref)


@pytest.mark.parametrize("nel,N", [((5, 3, 3), 7), ((3, 3, 1), 9)])
def test_dssum_fp32(nel, N):
    from oracle import operator
    h, o = make(nel, N)
    w0 = si.uniform(o.shape, 45).astype(np.float32)
    w = to_dev(w0, torch.float32).view(-1).clone()
    sem.sem_dssum(h, w, apply_mask=True)
    ref = operator.apply_dirichlet(operator.dssum(w0.astype(np.float64), o.gid), o.mask)
    assert rel_inf(to_np(w).reshape(o.shape), ref) < 1e-6


def test_dirichlet_faces_subset():
    from oracle import operator
    faces = 1 | 8 | 32
    h, o = make((3, 2, 2), 3, faces=faces)
    w0 = si.uniform(o.shape, 46)
    w = to_dev(w0).view(-1).clone()
    sem.sem_dssum(h, w, apply_mask=True)
    ref = operator.apply_dirichlet(operator.dssum(w0, o.gid), o.mask)
    np.testing.assert_array_equal(to_np(w).reshape(o.shape), ref)


@pytest.mark.parametrize("nel,N", [((5, 3, 3), 7), ((2, 2, 3), 4)])
def test_rhs(nel, N):
    h, o = make(nel, N)
    f = si.eval_fourier(si.fourier_modes(3), o.x, o.y, o.z)
    b = torch.empty(h.n_local, dtype=torch.float64, device=DEV)
    sem.sem_rhs(h, to_dev(f).view(-1), b)
    assert rel_inf(to_np(b).reshape(o.shape), o.rhs(f)) < TOL64


@pytest.mark.parametrize("nel,N", [((5, 3, 3), 7), ((3, 3, 1), 9), ((2, 2, 3), 3)])
def test_gradient_kernel(nel, N):
    from oracle import adjoint
    h, o = make(nel, N)
    u = si.uniform(o.shape, 47)
    lam = si.uniform(o.shape, 48)
    g = torch.empty(h.n_local, dtype=torch.float64, device=DEV)
    sem.sem_helmholtz_grad(h, to_dev(u).view(-1), to_dev(lam).view(-1), g)
    assert rel_inf(to_np(g).reshape(o.shape), adjoint.grad_h1(u, lam, o.G, o.D)) < TOL64


def test_apply_host_matches_device():
    h, o = make((5, 3, 3), 7)
    u = si.uniform(o.shape, 49)
    for dtype, tol in ((torch.float64, TOL64), (torch.float32, TOL32)):
        uh = torch.from_numpy(u.astype(np.float64)).to(dtype).view(-1).pin_memory()
        wh = torch.empty_like(uh).pin_memory()
        sem.sem_apply_host(h, uh, wh)
        ref = o.matvec(uh.double().numpy().reshape(o.shape))
        assert rel_inf(wh.double().numpy().reshape(o.shape), ref) < tol


@pytest.mark.parametrize("nel,N", [((5, 3, 9), 7), ((3, 3, 2), 5), ((7, 2, 11), 9), ((4, 4, 1), 7),
                                   ((2, 3, 4), 4)])
def test_apply_host_pipelined_equals_device(nel, N):
    """FP64 with host buffers: the copies overlap the work slab by slab of
    element planes; every pair sum is the unsplit operator's, so the result
    equals the device call bit for bit (odd N falls back to the plain path)."""
    h, o = make(nel, N)
    u = si.uniform(o.shape, 54)
    uh = torch.from_numpy(u).view(-1).pin_memory()
    wh = torch.empty_like(uh).pin_memory()
    sem.sem_apply_host(h, uh, wh)
    wd = torch.empty(h.n_local, dtype=torch.float64, device=DEV)
    sem.sem_apply(h, uh.to(DEV), wd)
    sem.sem_sync(h)
    assert torch.equal(wh, wd.cpu())
    assert rel_inf(wh.numpy().reshape(o.shape), o.matvec(u)) < TOL64


@pytest.mark.parametrize("nel,N", [((5, 3, 3), 7), ((3, 3, 1), 9), ((1, 1, 1), 2)])
def test_dot_unique_dof(nel, N):
    from oracle import operator
    h, o = make(nel, N)
    a = si.uniform(o.shape, 50)
    b = si.uniform(o.shape, 51)
    out = torch.empty(1, dtype=torch.float64, device=DEV)
    sem.sem_dot(h, to_dev(a).view(-1), to_dev(b).view(-1), out)
    ref = operator.weighted_dot(a, b, o.mult)
    assert abs(float(out) - ref) <= 1e-13 * np.sum(np.abs(a * b / o.mult))
    # continuous fields: equals the plain sum over unique points
    ga = si.uniform(int(o.gid.max()) + 1, 52)
    gb = si.uniform(int(o.gid.max()) + 1, 53)
    sem.sem_dot(h, to_dev(ga[o.gid]).view(-1), to_dev(gb[o.gid]).view(-1), out)
    assert abs(float(out) - float(np.dot(ga, gb))) <= 1e-13 * float(np.sum(np.abs(ga * gb)))
    # reproducible bit for bit
    first = float(out)
    sem.sem_dot(h, to_dev(ga[o.gid]).view(-1), to_dev(gb[o.gid]).view(-1), out)
    assert float(out) == first


@pytest.mark.parametrize("nel,N", [((5, 3, 3), 7), ((4, 3, 2), 5), ((3, 2, 3), 9), ((7, 1, 1), 7)])
@pytest.mark.parametrize("h1,h2", [(1.0, 0.0), (0.37, 4.25)])
def test_ax_fp64_native_and_doublefloat(nel, N, h1, h2):
    """Both FP64 kernels against the oracle at the FP64 tolerance; the
    double-float one also on smooth input, where cancellation is strongest."""
    h, o = make(nel, N)
    inputs = [si.uniform(o.shape, 54), si.eval_fourier(si.fourier_modes(55), o.x, o.y, o.z)]
    for kind in (sem.SEM_F64_KERNEL_NATIVE, sem.SEM_F64_KERNEL_DOUBLEFLOAT):
        sem.sem_set_f64_kernel(h, kind)
        for u in inputs:
            w = torch.empty(h.n_local, dtype=torch.float64, device=DEV)
            sem.sem_ax(h, to_dev(u).view(-1), w, h1, h2)
            sem.sem_sync(h)
            err = rel_inf(to_np(w).reshape(o.shape), o.ax(u, h1, h2))
            assert err < TOL64, (kind, err)


def test_doublefloat_rejects_unsupported_order():
    h, _ = make((2, 2, 2), 4)
    with pytest.raises(sem.SemError):
        sem.sem_set_f64_kernel(h, sem.SEM_F64_KERNEL_DOUBLEFLOAT)


def per_element_rel(a, ref):
    """max over elements of ||a_e - ref_e||_inf / ||ref_e||_inf."""
    d = np.abs(a - ref).reshape(ref.shape[0], -1).max(axis=1)
    m = np.abs(ref).reshape(ref.shape[0], -1).max(axis=1)
    return float((d / m).max())


@pytest.mark.parametrize("N", [5, 7, 9])
@pytest.mark.parametrize("seed", [3, 1234])
def test_ax_fp64_smooth_fields(N, seed):
    """Smooth inputs are the hardest case of the double-float element
    kernel: the derivatives of a smooth u cancel, so the result is small
    against the products that form it.  Eight Fourier modes with
    wavenumbers up to 4 on 4^3 elements of [0, 2 pi]^3 (each element spans
    up to one wavelength); every element within 1e-12 of its own largest
    output (a float32 emulation of the kernel's arithmetic gives at most
    4.3e-13, at N = 9)."""
    h, o = make((4, 4, 4), N)
    u = si.eval_fourier(si.fourier_modes(seed), o.x, o.y, o.z)
    for h1, h2 in ((1.0, 0.0), (0.37, 4.25)):
        w = torch.empty(h.n_local, dtype=torch.float64, device=DEV)
        sem.sem_ax(h, to_dev(u).view(-1), w, h1, h2)
        torch.cuda.synchronize()
        assert per_element_rel(to_np(w).reshape(o.shape), o.ax(u, h1, h2)) < TOL64, (h1, h2)


@pytest.mark.parametrize("N", [5, 7, 9])
def test_ax_fp64_strongly_deformed(N):
    """A deformation amplitude of 0.3 (three times the workload's) makes the
    off-diagonal geometric factors comparable to the diagonal ones; the
    kernel's per-point bound of the G products takes the largest of all
    six."""
    h, o = make((3, 3, 2), N, deform=0.3)
    assert np.all(o.detJ > 0)
    for u in (si.uniform(o.shape, 71), si.eval_fourier(si.fourier_modes(72), o.x, o.y, o.z)):
        w = torch.empty(h.n_local, dtype=torch.float64, device=DEV)
        sem.sem_ax(h, to_dev(u).view(-1), w)
        torch.cuda.synchronize()
        assert per_element_rel(to_np(w).reshape(o.shape), o.ax(u)) < TOL64


@pytest.mark.parametrize("N", [1, 2, 3, 5, 7, 9])
def test_ax_fp64_native_every_path(N):
    """IEEE FP64 Ax (SEM_F64_KERNEL_NATIVE): the even-odd kernel at N = 7
    and 9, the column kernel at the other orders, with constant h1, a
    per-point h1 and the Helmholtz term, against the oracle at the FP64
    tolerance."""
    h, o = make((3, 2, 2), N)
    sem.sem_set_f64_kernel(h, sem.SEM_F64_KERNEL_NATIVE)
    u = si.uniform(o.shape, 81)
    h1f = si.smooth_coefficient(o.x, o.y, o.z, 82)
    for h1, h2, field in ((1.0, 0.0, None), (0.37, 4.25, None), (0.0, 1.5, h1f)):
        w = torch.empty(h.n_local, dtype=torch.float64, device=DEV)
        sem.sem_ax(h, to_dev(u).view(-1), w, h1, h2,
                   h1_field=None if field is None else to_dev(field).view(-1))
        sem.sem_sync(h)
        ref = o.ax(u, h1, h2, field)
        assert rel_inf(to_np(w).reshape(o.shape), ref) < TOL64, (h1, h2, field is None)
