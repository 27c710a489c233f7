"""GB300-native matrix-free spectral-element operator and solver.

Implements the data-parallel hot path of the SEM described in arXiv
2107.01243 (Neko): the element operator w_e = D^T G_e D u_e on hexahedra with
(N+1)^3 GLL points, the gather-scatter QQ^T with a Dirichlet mask, Jacobi-
preconditioned CG with FP32-inner / FP64 refinement, and the adjoint
gradient with respect to a per-point diffusion coefficient.  All compute runs
in the hand-written sm_103a kernels of ``lib/libsem_gb300.so`` (C ABI in
include/sem.h); this package is its Python binding.
"""
from ._lib import (SemError, SEM_F64, SEM_F32, SEM_PREC_F64, SEM_PREC_F32, SEM_SOLVE_F64,
                   SEM_SOLVE_MIXED, SEM_FACE_ALL, SEM_FIELD_X, SEM_FIELD_Y, SEM_FIELD_Z,
                   SEM_FIELD_G, SEM_FIELD_B, SEM_FIELD_MULT, SEM_FIELD_MASK, SEM_FIELD_GID,
                   SEM_FIELD_DINV, LIB_PATH, SEM_F64_KERNEL_AUTO,
                   SEM_F64_KERNEL_NATIVE, SEM_F64_KERNEL_DOUBLEFLOAT, SEM_DSSUM_BOX,
                   SEM_DSSUM_SEGMENTS, SEM_APPLY_LOCAL, SEM_APPLY_FINISH, SEM_APPLY_FULL,
                   SEM_INNER_AUTO, SEM_INNER_LOCAL, SEM_INNER_GLOBAL, SEM_SCHWARZ_LOCAL,
                   SEM_SCHWARZ_COARSE, SEM_SCHWARZ_BOTH, SEM_CG_STANDARD, SEM_CG_PIPELINED,
                   SEM_ERR_ARG, SEM_NOALLOC_MAX_POINTS)
from ._lib import (SEM_FACE_XMIN, SEM_FACE_XMAX, SEM_FACE_YMIN, SEM_FACE_YMAX, SEM_FACE_ZMIN,
                   SEM_FACE_ZMAX)
from .api import (Handle, sem_setup, sem_destroy, sem_get_sizes, sem_get_field, sem_ax,
                  sem_apply, sem_apply_global, sem_to_global, sem_set_inner_vectors,
                  sem_set_cg_variant, sem_dssum, sem_rhs, sem_cg_solve, sem_helmholtz_grad,
                  sem_apply_host, sem_dot, sem_sync,
                  sem_selftest_timeout, sem_set_f64_kernel, sem_set_dssum_kernel,
                  sem_autotune, sem_set_tuning,
                  sem_dot_noalloc, Batch, sem_batch_create, sem_batch_solve,
                  sem_batch_destroy, sem_batch_set_concurrency, Projection, sem_proj_create, sem_proj_solve,
                  sem_proj_size, sem_proj_reset, sem_proj_destroy, Schwarz,
                  sem_schwarz_create, sem_schwarz_apply, sem_schwarz_destroy, sem_gmres_solve,
                  sem_gather, sem_scatter_add, sem_set_multiplicity, sem_jacobi_diag,
                  sem_jacobi_invert, sem_cg_update, sem_cg_direction)
from .autograd import HelmholtzSolve, helmholtz_solve
from . import partition
