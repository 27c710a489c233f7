"""GPU parity of the default FP64 operator (double-float arithmetic) on inputs
far from unit scale, through the C ABI.

Double-float arithmetic keeps FP64 accuracy only while every intermediate
lies inside FP32's exponent range.  The kernel normalises the geometric
factors and the coefficients by powers of two and rescales elements whose
largest |u| lies outside [2^-60, 2^76) (see include/sem.h,
sem_set_f64_kernel).  The operator is linear, so each case has an exact
reference: the oracle at unit scale times the same power of two.  Cases:
u scaled by 2^+-130, 2^+-140, 2^-100 and 2^-1060 (subnormal), values that span
2^60 inside one element, elements at 2^+-60 beside unit elements, a mesh of
side 1e-9 (B near 2^-100, G near 2^-36) with coefficients from 1e-30 to 1e18,
and Inf / NaN entries, through sem_ax, sem_apply, sem_apply_host and the FP64
sem_cg_solve.
"""
import math

import numpy as np
import pytest
import torch

import paper_2107_01243_gb300 as sem
import seeded_inputs as si
from tests.helpers import OracleProblem, rel_inf, TWO_PI

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
TOL64 = 1e-12

SCALES = [130, -130, 140, -140, -100, 75, 76, -60, -61]


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV, torch.float64)


def make(nel, N, length=(TWO_PI,) * 3, deform=0.1):
    h = sem.sem_setup(nel, N, length=length, deform=deform)
    o = OracleProblem(nel, N, length=length, deform=deform)
    return h, o


def ax_gpu(h, u, h1=1.0, h2=0.0, kind=sem.SEM_F64_KERNEL_AUTO):
    sem.sem_set_f64_kernel(h, kind)
    w = torch.empty(h.n_local, dtype=torch.float64, device=DEV)
    sem.sem_ax(h, to_dev(u).view(-1), w, h1, h2)
    sem.sem_sync(h)
    return w.cpu().numpy().reshape(u.shape)


def per_element_rel(a, ref):
    """max over elements of ||a_e - ref_e||_inf / ||ref_e||_inf."""
    d = np.abs(a - ref).reshape(ref.shape[0], -1).max(axis=1)
    m = np.abs(ref).reshape(ref.shape[0], -1).max(axis=1)
    return float((d / m).max())


@pytest.mark.parametrize("N", [5, 7, 9])
@pytest.mark.parametrize("k", SCALES)
@pytest.mark.parametrize("h1,h2", [(1.0, 0.0), (0.37, 4.25)])
def test_ax_scaled_input(N, k, h1, h2):
    h, o = make((3, 2, 2), N)
    u = si.uniform(o.shape, 60)
    ref = o.ax(u, h1, h2) * 2.0 ** k
    w = ax_gpu(h, u * 2.0 ** k, h1, h2)
    assert np.all(np.isfinite(w))
    assert rel_inf(w, ref) < TOL64, k


def test_ax_subnormal_input_with_large_h1():
    """u at 2^-1060 (subnormal: about 14 significant bits, exact multiples of
    2^-1074) with h1 = 2^1000: the result is about 2^-60 and must still carry
    the operator's accuracy, because the subnormal values are exact."""
    h, o = make((2, 2, 2), 7)
    u = np.round(si.uniform(o.shape, 61) * 2.0 ** 13)      # integers below 2^13
    usub = u * 2.0 ** -1074                               # exact subnormals
    assert np.all(usub[u != 0] != 0) and np.abs(usub).max() < 2.0 ** -1022
    w = ax_gpu(h, usub, 2.0 ** 1000, 0.0)
    ref = o.ax(u, 1.0) * 2.0 ** -74
    assert rel_inf(w, ref) < TOL64


def test_ax_wide_range_within_and_across_elements():
    """Element 0 spans 2^60 inside itself (u times 2^(60 i / N) along x),
    element 1 sits at 2^60 and element 2 at 2^-60 beside unit elements; each
    element must be accurate relative to its own largest output."""
    N = 7
    h, o = make((4, 3, 2), N)
    u = si.uniform(o.shape, 62)
    i = np.arange(N + 1)
    u[0] *= 2.0 ** (60.0 * i / N)[None, None, :]
    u[1] *= 2.0 ** 60
    u[2] *= 2.0 ** -60
    u[5] *= 2.0 ** -90
    u[6] *= 2.0 ** 90
    for h1, h2 in ((1.0, 0.0), (0.37, 4.25)):
        w = ax_gpu(h, u, h1, h2)
        assert per_element_rel(w, o.ax(u, h1, h2)) < TOL64


@pytest.mark.parametrize("h1,h2", [(1.0, 0.0), (1.0, 1e18), (1e-30, 1.0), (3e20, 0.0),
                                   (1.0, 1e-25)])
def test_ax_nanometre_mesh(h1, h2):
    """Mesh of side 1e-9: G near 2^-36 and B near 2^-100, both normalised per
    element; the stiffness and mass terms are scaled against each other."""
    L = (1e-9,) * 3
    h, o = make((3, 2, 2), 7, length=L, deform=0.1)
    assert np.abs(o.B).max() < 2.0 ** -80
    for u in (si.uniform(o.shape, 63), si.uniform(o.shape, 64) * 2.0 ** -70):
        ref = o.ax(u, h1, h2)
        w = ax_gpu(h, u, h1, h2)
        assert per_element_rel(w, ref) < TOL64, (h1, h2)


@pytest.mark.parametrize("k", [140, -140, -100, 0])
def test_apply_and_apply_host_scaled(k):
    """The assembled operator (fused element kernel, split gather-scatter) and
    its host-buffer form on 2^k u."""
    h, o = make((5, 3, 4), 7)
    u = si.uniform(o.shape, 65)
    ref = o.matvec(u, 1.0, 0.5) * 2.0 ** k
    us = u * 2.0 ** k
    wd = torch.empty(h.n_local, dtype=torch.float64, device=DEV)
    sem.sem_apply(h, to_dev(us).view(-1), wd, 1.0, 0.5)
    sem.sem_sync(h)
    assert rel_inf(wd.cpu().numpy().reshape(o.shape), ref) < TOL64
    # host buffers (Poisson, the pipelined slabs)
    uh = torch.from_numpy(us).view(-1).pin_memory()
    wh = torch.empty_like(uh).pin_memory()
    sem.sem_apply_host(h, uh, wh)
    assert rel_inf(wh.numpy().reshape(o.shape), o.matvec(u) * 2.0 ** k) < TOL64


def test_apply_nanometre_mesh():
    L = (1e-9,) * 3
    h, o = make((4, 3, 3), 7, length=L)
    u = si.uniform(o.shape, 66)
    for h1, h2 in ((1.0, 0.0), (1.0, 1e18)):
        wd = torch.empty(h.n_local, dtype=torch.float64, device=DEV)
        sem.sem_apply(h, to_dev(u).view(-1), wd, h1, h2)
        sem.sem_sync(h)
        assert rel_inf(wd.cpu().numpy().reshape(o.shape), o.matvec(u, h1, h2)) < TOL64


@pytest.mark.parametrize("bad", [float("nan"), float("inf"), -float("inf")])
def test_ax_nonfinite_entry(bad):
    """An Inf or NaN in u_e makes every output of element e NaN; the other
    elements are untouched and match the oracle.  The native kernel also gives
    non-finite values in e (point by point) and the same values elsewhere."""
    N = 7
    h, o = make((3, 2, 2), N)
    u = si.uniform(o.shape, 67)
    e, pt = 4, (3, 5, 2)
    u[e][pt] = bad
    w = ax_gpu(h, u)
    assert np.all(np.isnan(w[e]))
    others = [f for f in range(o.shape[0]) if f != e]
    uo = u.copy()
    uo[e] = 0.0
    ref = o.ax(uo)
    assert rel_inf(w[others], ref[others]) < TOL64
    wn = ax_gpu(h, u, kind=sem.SEM_F64_KERNEL_NATIVE)
    assert not np.all(np.isfinite(wn[e]))
    assert rel_inf(wn[others], ref[others]) < TOL64


def test_ax_overflowing_result_is_infinite():
    """Inputs near the top of FP64's range: where the exact result overflows,
    the output is +-Inf with the oracle's sign, and never a finite wrong value."""
    h, o = make((2, 2, 2), 7)
    u = si.uniform(o.shape, 68)
    ref = o.ax(u)                              # unit scale
    w = ax_gpu(h, u * 2.0 ** 1022)             # |ref| reaches 9.5: |w| about 2^1025
    # |ref| 2^1022 above 2^1024 (a Python float cannot hold 2^1024 itself)
    big = np.abs(ref) > 2.0 ** 2 * (1 + 1e-12)
    assert big.any()
    assert np.all(np.isinf(w[big])) and np.all(np.sign(w[big]) == np.sign(ref[big]))
    small = np.abs(ref) < 2.0
    assert small.any()
    np.testing.assert_allclose(w[small] * 2.0 ** -1022, ref[small],
                               rtol=0, atol=TOL64 * np.abs(ref).max())


@pytest.mark.parametrize("k", [0, 140, -140, -100])
def test_cg_fp64_scaled_rhs(k):
    """FP64 PCG on 2^k b: the fused element kernel forms <p, H p> with the
    element scaling; the solution is 2^k times the unit-scale solution, and
    the oracle's residual of the returned x meets the tolerance."""
    h, o = make((4, 3, 3), 7)
    f = si.eval_fourier(si.fourier_modes(1234), o.x, o.y, o.z)
    b = o.rhs(f)
    xs = []
    iters = []
    for kk in (0, k):
        bd = to_dev(b * 2.0 ** kk).view(-1)
        xd = torch.empty_like(bd)
        info = sem.sem_cg_solve(h, bd, xd, tol=1e-10)
        assert info["status"] == "SEM_OK", info
        x = xd.cpu().numpy().reshape(o.shape)
        assert o.residual(x * 2.0 ** -kk, b) <= 1.05e-10
        xs.append(x * 2.0 ** -kk)
        iters.append(info["iters"])
    ref = o.pcg(b, tol=1e-10)
    assert abs(iters[1] - iters[0]) <= 1 and abs(iters[0] - ref.iters) <= 1
    assert rel_inf(xs[1], xs[0]) < 1e-9


def test_cg_fp64_nanometre_mesh():
    """FP64 PCG on the 1e-9 mesh: b near 2^-100 (the GLL-lumped mass), the
    solution near 2^-64."""
    L = (1e-9,) * 3
    h, o = make((4, 3, 3), 7, length=L)
    f = si.eval_fourier(si.fourier_modes(1234), o.x * 2e9 * math.pi, o.y * 2e9 * math.pi,
                        o.z * 2e9 * math.pi)
    b = o.rhs(f)
    assert 0 < np.abs(b).max() < 2.0 ** -80
    bd = to_dev(b).view(-1)
    xd = torch.empty_like(bd)
    info = sem.sem_cg_solve(h, bd, xd, tol=1e-10)
    assert info["status"] == "SEM_OK", info
    x = xd.cpu().numpy().reshape(o.shape)
    assert o.residual(x, b) <= 1.05e-10
    ref = o.pcg(b, tol=1e-10)
    assert abs(info["iters"] - ref.iters) <= 1
    assert rel_inf(x, ref.x) < 1e-8


@pytest.mark.parametrize("k", [140, -140, -100])
@pytest.mark.parametrize("inner", [sem.SEM_INNER_GLOBAL, sem.SEM_INNER_LOCAL],
                         ids=["global-vectors", "local-vectors"])
def test_cg_mixed_scaled_rhs(k, inner):
    """FP32-inner / FP64-refinement PCG on 2^k b: the inner solves work on the
    FP64 residual times a power of two chosen from ||b||, so the FP32 vectors
    stay in FP32's normal range and the iterations repeat those at unit scale."""
    h, o = make((4, 3, 3), 7)
    sem.sem_set_inner_vectors(h, inner)
    b = o.rhs(si.eval_fourier(si.fourier_modes(1235), o.x, o.y, o.z))
    its = []
    for kk in (0, k):
        bd = to_dev(b * 2.0 ** kk).view(-1)
        xd = torch.empty_like(bd)
        info = sem.sem_cg_solve(h, bd, xd, tol=1e-8, precision=sem.SEM_SOLVE_MIXED)
        assert info["status"] == "SEM_OK", (kk, info)
        x = xd.cpu().numpy().reshape(o.shape) * 2.0 ** -kk
        assert o.residual(x, b) <= 1.05e-8, kk
        its.append(info["iters"])
    assert abs(its[1] - its[0]) <= 1, its


@pytest.mark.parametrize("k", [140, -140])
def test_gmres_mixed_scaled_rhs(k):
    """Mixed-precision FGMRES with the two-level Schwarz preconditioner on 2^k b."""
    h, o = make((4, 3, 3), 7)
    b = o.rhs(si.eval_fourier(si.fourier_modes(1236), o.x, o.y, o.z))
    pre = sem.sem_schwarz_create(h, 1.0, 0.0, coarse_iters=10)
    bd = to_dev(b * 2.0 ** k).view(-1)
    xd = torch.empty_like(bd)
    info = sem.sem_gmres_solve(h, bd, xd, tol=1e-8, restart=10, precond=pre,
                               precision=sem.SEM_SOLVE_MIXED)
    assert info["status"] == "SEM_OK", info
    assert o.residual(xd.cpu().numpy().reshape(o.shape) * 2.0 ** -k, b) <= 1.05e-8
    sem.sem_schwarz_destroy(pre)


def test_batch_scaled_rhs():
    """Batched mixed-precision Helmholtz solves whose right-hand sides sit at
    2^-140, 1 and 2^140 side by side."""
    shapes = [((3, 3, 2), 7, 0.5, -140), ((3, 2, 2), 5, 2.0, 0), ((2, 2, 3), 9, 7.0, 140)]
    hs, os_, bs, refs = [], [], [], []
    for q, (nel, N, lam, k) in enumerate(shapes):
        h, o = make(nel, N)
        b = o.rhs(si.eval_fourier(si.fourier_modes(1240 + q), o.x, o.y, o.z))
        hs.append(h)
        os_.append(o)
        refs.append(b)
        bs.append(to_dev(b * 2.0 ** k).view(-1))
    batch = sem.sem_batch_create(hs)
    xs = [torch.empty_like(b) for b in bs]
    infos = sem.sem_batch_solve(batch, bs, xs, [1.0] * 3, [s[2] for s in shapes], tol=1e-8)
    for (nel, N, lam, k), o, b, x, info in zip(shapes, os_, refs, xs, infos):
        assert info["status"] == "SEM_OK", info
        xr = x.cpu().numpy().reshape(o.shape) * 2.0 ** -k
        assert o.residual(xr, b, h1=1.0, h2=lam) <= 1.05e-8
    sem.sem_batch_destroy(batch)
