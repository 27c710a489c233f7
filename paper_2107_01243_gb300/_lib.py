"""ctypes binding of libsem_gb300.so (include/sem.h).

Argument marshalling only: every computation runs in the library's CUDA
kernels.  Importing this module does not need a GPU; the first call that
reaches the library raises ``SemError`` when the library is missing or a
call fails.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libsem_gb300.so")

# status codes (sem_status)
SEM_OK, SEM_ERR_ARG, SEM_ERR_CUDA, SEM_ERR_NOCONV = 0, 1, 2, 3
SEM_ERR_BREAKDOWN, SEM_ERR_TIMEOUT, SEM_ERR_OOM, SEM_ERR_STATE = 4, 5, 6, 7
STATUS_NAMES = {0: "SEM_OK", 1: "SEM_ERR_ARG", 2: "SEM_ERR_CUDA", 3: "SEM_ERR_NOCONV",
                4: "SEM_ERR_BREAKDOWN", 5: "SEM_ERR_TIMEOUT", 6: "SEM_ERR_OOM",
                7: "SEM_ERR_STATE"}
SEM_F64, SEM_F32 = 0, 1
SEM_PREC_F64, SEM_PREC_F32 = 1, 2
SEM_SOLVE_F64, SEM_SOLVE_MIXED = 0, 1
SEM_FACE_XMIN, SEM_FACE_XMAX, SEM_FACE_YMIN, SEM_FACE_YMAX, SEM_FACE_ZMIN, SEM_FACE_ZMAX = (
    1, 2, 4, 8, 16, 32)
SEM_FACE_ALL = 63
SEM_F64_KERNEL_AUTO, SEM_F64_KERNEL_NATIVE, SEM_F64_KERNEL_DOUBLEFLOAT = 0, 1, 2
SEM_DSSUM_BOX, SEM_DSSUM_SEGMENTS = 0, 1
SEM_APPLY_LOCAL, SEM_APPLY_FINISH, SEM_APPLY_FULL = 1, 2, 3
SEM_NOALLOC_MAX_POINTS = 67108864
SEM_INNER_AUTO, SEM_INNER_LOCAL, SEM_INNER_GLOBAL = 0, 1, 2
SEM_SCHWARZ_LOCAL, SEM_SCHWARZ_COARSE, SEM_SCHWARZ_BOTH = 1, 2, 3
SEM_CG_STANDARD, SEM_CG_PIPELINED = 0, 1
(SEM_FIELD_X, SEM_FIELD_Y, SEM_FIELD_Z, SEM_FIELD_G, SEM_FIELD_B, SEM_FIELD_MULT,
 SEM_FIELD_MASK, SEM_FIELD_GID, SEM_FIELD_DINV) = range(9)


class SemError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class MeshDesc(ctypes.Structure):
    _fields_ = [("nelx", ctypes.c_int), ("nely", ctypes.c_int), ("nelz", ctypes.c_int),
                ("x0", ctypes.c_double * 3), ("len", ctypes.c_double * 3),
                ("deform_amp", ctypes.c_double), ("xyz_gll", ctypes.c_void_p),
                ("dirichlet_faces", ctypes.c_int)]


class SolveOpts(ctypes.Structure):
    _fields_ = [("h1", ctypes.c_double), ("h2", ctypes.c_double),
                ("h1_field", ctypes.c_void_p), ("tol", ctypes.c_double),
                ("maxit", ctypes.c_int), ("precision", ctypes.c_int),
                ("inner_tol", ctypes.c_double), ("max_outer", ctypes.c_int),
                ("check_every", ctypes.c_int), ("use_graph", ctypes.c_int),
                ("x0_is_zero", ctypes.c_int), ("stream", ctypes.c_void_p)]


class Tuning(ctypes.Structure):
    _fields_ = [("ax32_kernel", ctypes.c_int), ("ax32_stages", ctypes.c_int),
                ("ax32_elems_per_cta", ctypes.c_int), ("f64_stages", ctypes.c_int),
                ("ax32_ms", ctypes.c_double), ("ax64_ms", ctypes.c_double),
                ("from_cache", ctypes.c_int)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("outer_iters", ctypes.c_int),
                ("rel_res", ctypes.c_double), ("status", ctypes.c_int)]


_P = ctypes.c_void_p
_I64P = ctypes.POINTER(ctypes.c_int64)
# name -> (restype, argtypes); every symbol declared in include/sem.h
SIGNATURES = {
    "sem_setup": (ctypes.c_int, [ctypes.POINTER(MeshDesc), ctypes.c_int, ctypes.c_int, _P,
                                 ctypes.POINTER(_P)]),
    "sem_destroy": (ctypes.c_int, [_P]),
    "sem_last_error": (ctypes.c_char_p, []),
    "sem_get_sizes": (ctypes.c_int, [_P, _I64P, _I64P, ctypes.POINTER(ctypes.c_int), _I64P]),
    "sem_get_field": (ctypes.c_int, [_P, ctypes.c_int, _P, ctypes.c_int, _P]),
    "sem_ax": (ctypes.c_int, [_P, _P, _P, ctypes.c_double, ctypes.c_double, _P, ctypes.c_int,
                              _P]),
    "sem_dssum": (ctypes.c_int, [_P, _P, ctypes.c_int, ctypes.c_int, _P]),
    "sem_apply": (ctypes.c_int, [_P, _P, _P, ctypes.c_double, ctypes.c_double, _P,
                                 ctypes.c_int, ctypes.c_int, _P]),
    "sem_proj_create": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)]),
    "sem_proj_solve": (ctypes.c_int, [_P, _P, _P, ctypes.POINTER(SolveOpts),
                                      ctypes.POINTER(SolveInfo)]),
    "sem_proj_size": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int)]),
    "sem_proj_reset": (ctypes.c_int, [_P]),
    "sem_proj_destroy": (ctypes.c_int, [_P]),
    "sem_rhs": (ctypes.c_int, [_P, _P, _P, _P]),
    "sem_solve_opts_default": (None, [ctypes.POINTER(SolveOpts)]),
    "sem_cg_solve": (ctypes.c_int, [_P, _P, _P, ctypes.POINTER(SolveOpts),
                                    ctypes.POINTER(SolveInfo)]),
    "sem_helmholtz_grad": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "sem_apply_host": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, _P]),
    "sem_dot": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "sem_batch_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, ctypes.POINTER(_P)]),
    "sem_batch_solve": (ctypes.c_int, [_P, ctypes.POINTER(_P), ctypes.POINTER(_P),
                                       ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(SolveOpts), ctypes.POINTER(SolveInfo)]),
    "sem_batch_destroy": (ctypes.c_int, [_P]),
    "sem_batch_set_concurrency": (ctypes.c_int, [_P, ctypes.c_int]),
    "sem_sync": (ctypes.c_int, [_P, _P]),
    "sem_autotune": (ctypes.c_int, [_P, _P, ctypes.c_void_p]),
    "sem_set_tuning": (ctypes.c_int, [_P, ctypes.c_void_p]),
    "sem_set_f64_kernel": (ctypes.c_int, [_P, ctypes.c_int]),
    "sem_set_dssum_kernel": (ctypes.c_int, [_P, ctypes.c_int]),
    "sem_apply_global": (ctypes.c_int, [_P, _P, _P, ctypes.c_double, ctypes.c_double,
                                        ctypes.c_int, _P]),
    "sem_to_global": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, _P]),
    "sem_set_inner_vectors": (ctypes.c_int, [_P, ctypes.c_int]),
    "sem_set_cg_variant": (ctypes.c_int, [_P, ctypes.c_int]),
    "sem_schwarz_create": (ctypes.c_int, [_P, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                          ctypes.c_int, _P, ctypes.POINTER(ctypes.c_void_p)]),
    "sem_schwarz_apply": (ctypes.c_int, [_P, _P, _P, _P]),
    "sem_schwarz_destroy": (ctypes.c_int, [_P]),
    "sem_gmres_solve": (ctypes.c_int, [_P, _P, _P, ctypes.POINTER(SolveOpts), ctypes.c_int, _P,
                                       ctypes.POINTER(SolveInfo)]),
    "sem_selftest_timeout": (ctypes.c_int, [_P, ctypes.c_double, _P]),
    "sem_dot_noalloc": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "sem_gather": (ctypes.c_int, [_P, _P, _P, ctypes.c_int64, _P, _P]),
    "sem_scatter_add": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_int64, _P, ctypes.c_int64, _P]),
    "sem_set_multiplicity": (ctypes.c_int, [_P, _P, _P]),
    "sem_jacobi_diag": (ctypes.c_int, [_P, ctypes.c_double, ctypes.c_double, _P, _P]),
    "sem_jacobi_invert": (ctypes.c_int, [_P, _P, _P, _P]),
    "sem_cg_update": (ctypes.c_int, [_P, ctypes.c_double, _P, _P, _P, _P, _P, _P, _P, _P]),
    "sem_cg_direction": (ctypes.c_int, [_P, ctypes.c_double, _P, _P, _P]),
}

_lib = None


def load():
    """Load the library (once).  Raises SemError if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise SemError(SEM_ERR_STATE, f"CUDA library not built: {LIB_PATH} is missing "
                       "(run __graft_entry__.build())")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(status):
    if status != SEM_OK:
        msg = load().sem_last_error().decode(errors="replace")
        raise SemError(status, msg)
