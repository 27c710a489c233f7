"""Python entry points with the names of the C ABI (include/sem.h).

Vectors are torch tensors: L-vectors of n_L = E (N+1)^3 values on the CUDA
device, contiguous, float64 or float32.  These functions only check and
marshal arguments; the work is done by the library's kernels on the current
torch stream (or the stream given).
"""
import ctypes

import torch

from . import _lib
from ._lib import (SemError, MeshDesc, SolveOpts, SolveInfo, check, SEM_F64, SEM_F32,
                   SEM_PREC_F64, SEM_PREC_F32, SEM_SOLVE_F64, SEM_SOLVE_MIXED, SEM_FACE_ALL,
                   SEM_ERR_NOCONV, SEM_ERR_BREAKDOWN, STATUS_NAMES)


def _stream(stream):
    if stream is None:
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, torch.cuda.Stream):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _copy_x0(x, x0, stream):
    """x <- x0 on torch's current stream, ordered before work on `stream`."""
    x.copy_(x0)
    if stream is None:
        return
    if isinstance(stream, torch.cuda.Stream):
        stream.wait_stream(torch.cuda.current_stream())
    else:                                 # a raw cudaStream_t: wait on the host
        torch.cuda.current_stream().synchronize()


def _dtype_code(t):
    if t.dtype == torch.float64:
        return SEM_F64
    if t.dtype == torch.float32:
        return SEM_F32
    raise SemError(1, f"unsupported dtype {t.dtype}")


class Handle:
    """Owns a sem_handle*; sizes cached at creation."""

    def __init__(self, ptr, nel, N):
        self.ptr = ptr
        self.nel = tuple(nel)
        n_local, n_global, n_ord, E = (ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int(),
                                       ctypes.c_int64())
        check(_lib.load().sem_get_sizes(ptr, ctypes.byref(n_local), ctypes.byref(n_global),
                                        ctypes.byref(n_ord), ctypes.byref(E)))
        self.n_local = n_local.value
        self.n_global = n_global.value
        self.N = n_ord.value
        self.E = E.value
        self.shape = (self.E, N + 1, N + 1, N + 1)

    def __del__(self):
        try:
            sem_destroy(self)
        except Exception:
            pass

    def _gvec(self, t, name):
        """A contiguous FP32 CUDA tensor of n_G values (a global vector)."""
        if not isinstance(t, torch.Tensor) or not t.is_cuda or not t.is_contiguous():
            raise SemError(1, f"{name} must be a contiguous CUDA tensor")
        if t.numel() != self.n_global or t.dtype != torch.float32:
            raise SemError(1, f"{name} must hold n_G = {self.n_global} float32 values")
        return ctypes.c_void_p(t.data_ptr())

    def _vec(self, t, name, dtype=None):
        if not isinstance(t, torch.Tensor):
            raise SemError(1, f"{name} must be a torch tensor")
        if not t.is_cuda:
            raise SemError(1, f"{name} must be on the CUDA device")
        if not t.is_contiguous():
            raise SemError(1, f"{name} must be contiguous")
        if t.numel() != self.n_local:
            raise SemError(1, f"{name} has {t.numel()} values, expected n_L = {self.n_local}")
        if dtype is not None and t.dtype != dtype:
            raise SemError(1, f"{name} must be {dtype}")
        return ctypes.c_void_p(t.data_ptr())


def sem_setup(nel, N, x0=(0.0, 0.0, 0.0), length=(1.0, 1.0, 1.0), deform=0.0,
              faces=SEM_FACE_ALL, precision=SEM_PREC_F64 | SEM_PREC_F32, xyz=None,
              stream=None):
    """Build the operator data for a nelx x nely x nelz box of order N."""
    lib = _lib.load()
    m = MeshDesc()
    m.nelx, m.nely, m.nelz = (int(v) for v in nel)
    for a in range(3):
        m.x0[a] = float(x0[a])
        m.len[a] = float(length[a])
    m.deform_amp = float(deform)
    m.dirichlet_faces = int(faces)
    keep = None
    if xyz is not None:
        import numpy as np
        keep = np.ascontiguousarray(xyz, dtype=np.float64)
        n_l = m.nelx * m.nely * m.nelz * (int(N) + 1) ** 3
        if keep.size != 3 * n_l:       # the library reads exactly 3 n_L host values
            raise SemError(1, f"xyz must hold 3 x n_L = {3 * n_l} coordinates "
                              f"(x, y, z L-vectors), got {keep.size}")
        m.xyz_gll = keep.ctypes.data
    out = ctypes.c_void_p()
    check(lib.sem_setup(ctypes.byref(m), int(N), int(precision), _stream(stream),
                        ctypes.byref(out)))
    return Handle(out, nel, N)


def sem_destroy(h):
    if h is not None and h.ptr:
        ptr, h.ptr = h.ptr, None
        check(_lib.load().sem_destroy(ptr))


def sem_get_sizes(h):
    return dict(n_local=h.n_local, n_global=h.n_global, N=h.N, E=h.E)


def sem_get_field(h, which, dst, stream=None):
    n = h.n_local * (6 if which == _lib.SEM_FIELD_G else 1)
    if not dst.is_cuda or not dst.is_contiguous() or dst.numel() != n:
        raise SemError(1, "sem_get_field: dst must be a contiguous CUDA tensor of the field size")
    if which == _lib.SEM_FIELD_GID and dst.dtype != torch.int64:
        raise SemError(1, "sem_get_field: gid needs an int64 tensor")
    code = SEM_F64 if dst.dtype in (torch.float64, torch.int64) else _dtype_code(dst)
    check(_lib.load().sem_get_field(h.ptr, int(which), ctypes.c_void_p(dst.data_ptr()), code,
                                    _stream(stream)))
    return dst


def sem_ax(h, u, w, h1=1.0, h2=0.0, h1_field=None, stream=None):
    """w = (h1 A_L + h2 B_L) u, element by element (no gather-scatter)."""
    pu = h._vec(u, "u")
    pw = h._vec(w, "w", u.dtype)
    pf = h._vec(h1_field, "h1_field", u.dtype) if h1_field is not None else None
    check(_lib.load().sem_ax(h.ptr, pu, pw, float(h1), float(h2), pf, _dtype_code(u),
                             _stream(stream)))
    return w


def sem_apply(h, u, w, h1=1.0, h2=0.0, h1_field=None, phase=_lib.SEM_APPLY_FULL, stream=None):
    """w = mask o QQ^T (h1 A_L + h2 B_L) u: the assembled operator (one CG matvec)."""
    pu = h._vec(u, "u")
    pw = h._vec(w, "w", u.dtype)
    pf = h._vec(h1_field, "h1_field", u.dtype) if h1_field is not None else None
    check(_lib.load().sem_apply(h.ptr, pu, pw, float(h1), float(h2), pf, _dtype_code(u),
                                int(phase), _stream(stream)))
    return w


def sem_apply_global(h, u_g, w_g, h1=1.0, h2=0.0, stream=None):
    """w_g = mask o Q^T (h1 A_L + h2 B_L) Q u_g on FP32 global vectors (n_G values)."""
    pu = h._gvec(u_g, "u_g")
    pw = h._gvec(w_g, "w_g")
    check(_lib.load().sem_apply_global(h.ptr, pu, pw, float(h1), float(h2), SEM_F32,
                                       _stream(stream)))
    return w_g


def sem_to_global(h, u, out_g, stream=None):
    """out_g[g] = u at a local copy of g (u continuous, FP64 or FP32; out_g FP32)."""
    pu = h._vec(u, "u")
    po = h._gvec(out_g, "out_g")
    check(_lib.load().sem_to_global(h.ptr, pu, po, _dtype_code(u), _stream(stream)))
    return out_g


def sem_set_cg_variant(h, kind):
    """Recurrences of the FP64 CG solves: SEM_CG_STANDARD or SEM_CG_PIPELINED."""
    check(_lib.load().sem_set_cg_variant(h.ptr, int(kind)))


def sem_set_inner_vectors(h, kind):
    """Vectors of the FP32 inner solves: SEM_INNER_AUTO, SEM_INNER_LOCAL or SEM_INNER_GLOBAL."""
    check(_lib.load().sem_set_inner_vectors(h.ptr, int(kind)))


def sem_dssum(h, w, apply_mask=True, stream=None):
    """In place w <- QQ^T w (then the Dirichlet mask if apply_mask)."""
    pw = h._vec(w, "w")
    check(_lib.load().sem_dssum(h.ptr, pw, int(bool(apply_mask)), _dtype_code(w),
                                _stream(stream)))
    return w


def sem_rhs(h, f, b, stream=None):
    """b = mask o QQ^T (B f)."""
    check(_lib.load().sem_rhs(h.ptr, h._vec(f, "f", torch.float64),
                              h._vec(b, "b", torch.float64), _stream(stream)))
    return b


def sem_cg_solve(h, b, x, h1=1.0, h2=0.0, h1_field=None, tol=1e-8, maxit=20000,
                 precision=SEM_SOLVE_F64, inner_tol=1e-4, max_outer=30, check_every=16,
                 use_graph=True, x0=None, stream=None, raise_on_fail=True):
    """Jacobi-PCG solve of mask o QQ^T H x = b; returns the info dict."""
    lib = _lib.load()
    o = SolveOpts()
    lib.sem_solve_opts_default(ctypes.byref(o))
    o.h1, o.h2 = float(h1), float(h2)
    o.h1_field = (h._vec(h1_field, "h1_field", torch.float64).value
                  if h1_field is not None else None)
    o.tol, o.maxit = float(tol), int(maxit)
    o.precision = int(precision)
    o.inner_tol, o.max_outer = float(inner_tol), int(max_outer)
    o.check_every, o.use_graph = int(check_every), int(bool(use_graph))
    pb = h._vec(b, "b", torch.float64)
    px = h._vec(x, "x", torch.float64)
    if x0 is not None:
        _copy_x0(x, x0, stream)
        o.x0_is_zero = 0
    o.stream = _stream(stream).value
    info = SolveInfo()
    st = lib.sem_cg_solve(h.ptr, pb, px, ctypes.byref(o), ctypes.byref(info))
    res = dict(iters=info.iters, outer_iters=info.outer_iters, rel_res=info.rel_res,
               status=STATUS_NAMES.get(info.status, info.status))
    if st != 0 and (raise_on_fail or st not in (SEM_ERR_NOCONV, SEM_ERR_BREAKDOWN)):
        check(st)
    return res


def sem_helmholtz_grad(h, u, lam, g, stream=None):
    """g = -(D^ lam)^T G (D^ u) at every local point (FP64)."""
    check(_lib.load().sem_helmholtz_grad(h.ptr, h._vec(u, "u", torch.float64),
                                         h._vec(lam, "lambda", torch.float64),
                                         h._vec(g, "g", torch.float64), _stream(stream)))
    return g


def sem_apply_host(h, u_host, w_host, stream=None):
    """w = mask o QQ^T A_L u with host tensors (copies inside the call)."""
    for t, name in ((u_host, "u_host"), (w_host, "w_host")):
        if t.is_cuda or not t.is_contiguous() or t.numel() != h.n_local:
            raise SemError(1, f"{name} must be a contiguous host tensor of n_L values")
    if u_host.dtype != w_host.dtype:
        raise SemError(1, "u_host and w_host must share a dtype")
    check(_lib.load().sem_apply_host(h.ptr, ctypes.c_void_p(u_host.data_ptr()),
                                     ctypes.c_void_p(w_host.data_ptr()), _dtype_code(u_host),
                                     _stream(stream)))
    return w_host


def sem_set_f64_kernel(h, kind):
    """Select the FP64 Ax kernel: SEM_F64_KERNEL_AUTO / _NATIVE / _DOUBLEFLOAT."""
    check(_lib.load().sem_set_f64_kernel(h.ptr, int(kind)))


def sem_set_dssum_kernel(h, kind):
    """Select the gather-scatter kernel: SEM_DSSUM_BOX or SEM_DSSUM_SEGMENTS."""
    check(_lib.load().sem_set_dssum_kernel(h.ptr, int(kind)))


def sem_autotune(h, stream=None):
    """Time the candidate Ax tiles on this handle and keep the fastest; returns the choice."""
    t = _lib.Tuning()
    check(_lib.load().sem_autotune(h.ptr, _stream(stream), ctypes.byref(t)))
    return dict(ax32_kernel="global-load" if t.ax32_kernel else "bulk-copy",
                ax32_stages=t.ax32_stages, ax32_elems_per_cta=t.ax32_elems_per_cta,
                f64_stages=t.f64_stages, ax32_ms=t.ax32_ms, ax64_ms=t.ax64_ms,
                from_cache=bool(t.from_cache))


def sem_set_tuning(h, ax32_kernel="bulk-copy", ax32_stages=2, ax32_elems_per_cta=1,
                   f64_stages=1):
    """Pin a tile choice (the same fields sem_autotune returns)."""
    t = _lib.Tuning()
    t.ax32_kernel = 1 if ax32_kernel == "global-load" else 0
    t.ax32_stages, t.ax32_elems_per_cta, t.f64_stages = ax32_stages, ax32_elems_per_cta, f64_stages
    check(_lib.load().sem_set_tuning(h.ptr, ctypes.byref(t)))


def sem_sync(h, stream=None):
    """Synchronise and raise SemError(SEM_ERR_TIMEOUT) if a device wait gave up."""
    check(_lib.load().sem_sync(h.ptr, _stream(stream)))


def sem_selftest_timeout(h, timeout_ms=20.0, stream=None):
    """Run the starved-barrier diagnostic; returns the status name it produced."""
    st = _lib.load().sem_selftest_timeout(h.ptr, float(timeout_ms), _stream(stream))
    return STATUS_NAMES.get(st, st)


def sem_dot(h, a, b, out, stream=None):
    """out[0] = sum_L a b / mult (unique-dof inner product), FP64, on the device."""
    if not out.is_cuda or out.dtype != torch.float64 or out.numel() < 1:
        raise SemError(1, "sem_dot: out must be a CUDA float64 tensor")
    check(_lib.load().sem_dot(h.ptr, h._vec(a, "a", torch.float64), h._vec(b, "b", torch.float64),
                              ctypes.c_void_p(out.data_ptr()), _stream(stream)))
    return out


def sem_dot_noalloc(h, a, b, out, stream=None):
    """Same as sem_dot, but the library allocates nothing for the call (its
    scratch is a static device array); for callers that cannot allocate."""
    if not out.is_cuda or out.dtype != torch.float64 or out.numel() < 1:
        raise SemError(1, "sem_dot_noalloc: out must be a CUDA float64 tensor")
    check(_lib.load().sem_dot_noalloc(h.ptr, h._vec(a, "a", torch.float64),
                                      h._vec(b, "b", torch.float64),
                                      ctypes.c_void_p(out.data_ptr()), _stream(stream)))
    return out


class Batch:
    """Owns a sem_batch* over a list of Handles (which must outlive it)."""

    def __init__(self, handles):
        lib = _lib.load()
        self.handles = list(handles)
        arr = (ctypes.c_void_p * len(self.handles))(*[h.ptr.value if isinstance(h.ptr, ctypes.c_void_p)
                                                     else h.ptr for h in self.handles])
        out = ctypes.c_void_p()
        check(lib.sem_batch_create(arr, len(self.handles), ctypes.byref(out)))
        self.ptr = out

    def __del__(self):
        try:
            sem_batch_destroy(self)
        except Exception:
            pass


def sem_batch_create(handles):
    """Group handles (FP32 geometry, odd N) into a batch for sem_batch_solve."""
    return Batch(handles)


def sem_batch_destroy(batch):
    if batch is not None and batch.ptr:
        ptr, batch.ptr = batch.ptr, None
        check(_lib.load().sem_batch_destroy(ptr))


def sem_batch_set_concurrency(batch, concurrent=True):
    """Launch the order classes' element kernels as concurrent branches (True)
    or one after another (False, the library's default)."""
    check(_lib.load().sem_batch_set_concurrency(batch.ptr, int(bool(concurrent))))


def sem_batch_solve(batch, bs, xs, h1s, h2s, tol=1e-8, maxit=20000, inner_tol=1e-4,
                    max_outer=30, check_every=16, use_graph=True, stream=None):
    """Solve every problem of the batch (FP32 inner / FP64 refinement);
    returns one info dict per problem."""
    lib = _lib.load()
    n = len(batch.handles)
    if not (len(bs) == len(xs) == len(h1s) == len(h2s) == n):
        raise SemError(1, "sem_batch_solve: one b, x, h1, h2 per problem")
    pb = (ctypes.c_void_p * n)(*[h._vec(b, "b", torch.float64).value
                                 for h, b in zip(batch.handles, bs)])
    px = (ctypes.c_void_p * n)(*[h._vec(x, "x", torch.float64).value
                                 for h, x in zip(batch.handles, xs)])
    c1 = (ctypes.c_double * n)(*[float(v) for v in h1s])
    c2 = (ctypes.c_double * n)(*[float(v) for v in h2s])
    o = SolveOpts()
    lib.sem_solve_opts_default(ctypes.byref(o))
    o.tol, o.maxit, o.inner_tol, o.max_outer = float(tol), int(maxit), float(inner_tol), int(max_outer)
    o.check_every, o.use_graph = int(check_every), int(bool(use_graph))
    o.precision = SEM_SOLVE_MIXED
    o.stream = _stream(stream).value
    infos = (SolveInfo * n)()
    check(lib.sem_batch_solve(batch.ptr, pb, px, c1, c2, ctypes.byref(o), infos))
    return [dict(iters=i.iters, outer_iters=i.outer_iters, rel_res=i.rel_res,
                 status=STATUS_NAMES.get(i.status, i.status)) for i in infos]


class Projection:
    """Owns a sem_proj* (space of previous solutions) on a Handle that must outlive it."""

    def __init__(self, h, m=20):
        out = ctypes.c_void_p()
        check(_lib.load().sem_proj_create(h.ptr, int(m), ctypes.byref(out)))
        self.h = h
        self.m = int(m)
        self.ptr = out

    def __del__(self):
        try:
            sem_proj_destroy(self)
        except Exception:
            pass


def sem_proj_create(h, m=20):
    """Space of at most m previous solutions of H x = b on handle h."""
    return Projection(h, m)


def sem_proj_destroy(p):
    if p is not None and p.ptr:
        ptr, p.ptr = p.ptr, None
        check(_lib.load().sem_proj_destroy(ptr))


def sem_proj_size(p):
    n = ctypes.c_int()
    check(_lib.load().sem_proj_size(p.ptr, ctypes.byref(n)))
    return n.value


def sem_proj_reset(p):
    check(_lib.load().sem_proj_reset(p.ptr))


def sem_proj_solve(p, b, x, h1=1.0, h2=0.0, tol=1e-8, maxit=20000, precision=SEM_SOLVE_F64,
                   inner_tol=1e-4, max_outer=30, check_every=16, use_graph=True, stream=None,
                   raise_on_fail=True):
    """Solve H x = b starting from the projection onto the space p, then add
    the correction to the space; returns the info dict."""
    lib = _lib.load()
    h = p.h
    o = SolveOpts()
    lib.sem_solve_opts_default(ctypes.byref(o))
    o.h1, o.h2 = float(h1), float(h2)
    o.tol, o.maxit = float(tol), int(maxit)
    o.precision = int(precision)
    o.inner_tol, o.max_outer = float(inner_tol), int(max_outer)
    o.check_every, o.use_graph = int(check_every), int(bool(use_graph))
    o.stream = _stream(stream).value
    pb = h._vec(b, "b", torch.float64)
    px = h._vec(x, "x", torch.float64)
    info = SolveInfo()
    st = lib.sem_proj_solve(p.ptr, pb, px, ctypes.byref(o), ctypes.byref(info))
    res = dict(iters=info.iters, outer_iters=info.outer_iters, rel_res=info.rel_res,
               status=STATUS_NAMES.get(info.status, info.status))
    if st != 0 and (raise_on_fail or st not in (SEM_ERR_NOCONV, SEM_ERR_BREAKDOWN)):
        check(st)
    return res


class Schwarz:
    """Owns a sem_schwarz* (two-level Schwarz preconditioner) on a Handle that
    must outlive it."""

    def __init__(self, h, h1=1.0, h2=0.0, levels=_lib.SEM_SCHWARZ_BOTH, coarse_iters=10,
                 stream=None):
        out = ctypes.c_void_p()
        check(_lib.load().sem_schwarz_create(h.ptr, float(h1), float(h2), int(levels),
                                             int(coarse_iters), _stream(stream),
                                             ctypes.byref(out)))
        self.h = h
        self.ptr = out

    def __del__(self):
        try:
            sem_schwarz_destroy(self)
        except Exception:
            pass


def sem_schwarz_create(h, h1=1.0, h2=0.0, levels=_lib.SEM_SCHWARZ_BOTH, coarse_iters=10,
                       stream=None):
    """Two-level additive Schwarz preconditioner for H = h1 A + h2 B on handle h."""
    return Schwarz(h, h1, h2, levels, coarse_iters, stream)


def sem_schwarz_destroy(sw):
    if sw is not None and sw.ptr:
        ptr, sw.ptr = sw.ptr, None
        check(_lib.load().sem_schwarz_destroy(ptr))


def sem_schwarz_apply(sw, r, z, stream=None):
    """z = M^-1 r (continuous, masked FP64 L-vectors)."""
    h = sw.h
    check(_lib.load().sem_schwarz_apply(sw.ptr, h._vec(r, "r", torch.float64),
                                        h._vec(z, "z", torch.float64), _stream(stream)))
    return z


def sem_gmres_solve(h, b, x, h1=1.0, h2=0.0, tol=1e-8, maxit=5000, restart=30, precond=None,
                    precision=SEM_SOLVE_F64, inner_tol=1e-4, max_outer=30, x0=None, stream=None,
                    raise_on_fail=True):
    """Flexible GMRES(restart) for mask o QQ^T H x = b, right-preconditioned by a
    Schwarz object (or point Jacobi when precond is None); returns the info dict
    (outer_iters = restart cycles in FP64, refinement steps in mixed precision).
    precision=SEM_SOLVE_MIXED with a Schwarz object runs FP32 inner GMRES on
    global vectors inside FP64 refinement."""
    lib = _lib.load()
    o = SolveOpts()
    lib.sem_solve_opts_default(ctypes.byref(o))
    o.h1, o.h2 = float(h1), float(h2)
    o.tol, o.maxit = float(tol), int(maxit)
    o.precision = int(precision)
    o.inner_tol, o.max_outer = float(inner_tol), int(max_outer)
    pb = h._vec(b, "b", torch.float64)
    px = h._vec(x, "x", torch.float64)
    if x0 is not None:
        _copy_x0(x, x0, stream)
        o.x0_is_zero = 0
    o.stream = _stream(stream).value
    info = SolveInfo()
    st = lib.sem_gmres_solve(h.ptr, pb, px, ctypes.byref(o), int(restart),
                             precond.ptr if precond is not None else None, ctypes.byref(info))
    res = dict(iters=info.iters, outer_iters=info.outer_iters, rel_res=info.rel_res,
               status=STATUS_NAMES.get(info.status, info.status))
    if st != 0 and (raise_on_fail or st not in (SEM_ERR_NOCONV, SEM_ERR_BREAKDOWN)):
        check(st)
    return res


# ---------------------------------------------------------------- partition primitives
def _dev_tensor(t, name, dtype, n=None):
    if not isinstance(t, torch.Tensor) or not t.is_cuda or not t.is_contiguous():
        raise SemError(1, f"{name} must be a contiguous CUDA tensor")
    if t.dtype != dtype:
        raise SemError(1, f"{name} must be {dtype}")
    if n is not None and t.numel() != n:
        raise SemError(1, f"{name} has {t.numel()} values, expected {n}")
    return ctypes.c_void_p(t.data_ptr())


def sem_gather(h, src, idx, dst, stream=None):
    """dst[t] = src[idx[t]] (src an FP64 L-vector, idx int64 on the device)."""
    n = idx.numel()
    check(_lib.load().sem_gather(h.ptr, h._vec(src, "src", torch.float64),
                                 _dev_tensor(idx, "idx", torch.int64), int(n),
                                 _dev_tensor(dst, "dst", torch.float64, n), _stream(stream)))
    return dst


def sem_scatter_add(h, dst, idx, pos, src, stream=None):
    """dst[idx[t]] += src[pos[t]] (dst an FP64 L-vector; the idx[t] distinct)."""
    n = idx.numel()
    check(_lib.load().sem_scatter_add(h.ptr, h._vec(dst, "dst", torch.float64),
                                      _dev_tensor(idx, "idx", torch.int64),
                                      _dev_tensor(pos, "pos", torch.int64, n), int(n),
                                      _dev_tensor(src, "src", torch.float64), int(src.numel()),
                                      _stream(stream)))
    return dst


def sem_set_multiplicity(h, mult, stream=None):
    """The dots' multiplicities replaced by mult (copies over all ranks)."""
    check(_lib.load().sem_set_multiplicity(h.ptr, h._vec(mult, "mult", torch.float64),
                                           _stream(stream)))


def sem_jacobi_diag(h, d, h1=1.0, h2=0.0, stream=None):
    """d = QQ^T diag(h1 A_L + h2 B_L) inside the handle (no mask)."""
    check(_lib.load().sem_jacobi_diag(h.ptr, float(h1), float(h2),
                                      h._vec(d, "d", torch.float64), _stream(stream)))
    return d


def sem_jacobi_invert(h, d, dinv, stream=None):
    """dinv = mask / d."""
    check(_lib.load().sem_jacobi_invert(h.ptr, h._vec(d, "d", torch.float64),
                                        h._vec(dinv, "dinv", torch.float64), _stream(stream)))
    return dinv


def sem_cg_update(h, alpha, p, w, x, r, dinv, z, dots, stream=None):
    """x += alpha p, r -= alpha w, z = dinv r; dots <- this rank's <r, z>, <r, r>."""
    f = torch.float64
    check(_lib.load().sem_cg_update(h.ptr, float(alpha), h._vec(p, "p", f), h._vec(w, "w", f),
                                    h._vec(x, "x", f), h._vec(r, "r", f),
                                    h._vec(dinv, "dinv", f), h._vec(z, "z", f),
                                    _dev_tensor(dots, "dots", f, 2), _stream(stream)))
    return dots


def sem_cg_direction(h, beta, z, p, stream=None):
    """p = z + beta p."""
    f = torch.float64
    check(_lib.load().sem_cg_direction(h.ptr, float(beta), h._vec(z, "z", f), h._vec(p, "p", f),
                                       _stream(stream)))
    return p
