/*
 * sem.h -- C ABI of the GB300 spectral-element operator / solver library.
 *
 * The library applies and inverts the matrix-free SEM Poisson/Helmholtz
 * operator on hexahedral elements with (N+1)^3 Gauss-Lobatto-Legendre points:
 *
 *   w_L = mask o QQ^T (h1 A_L + h2 B_L) u_L,   A^e = D^T G^e D
 *
 * (arXiv 2107.01243, §2, Eq. 9-10; gather-scatter §3.2; Krylov solve §2 end
 * and §4).  Everything runs in hand-written sm_103a CUDA kernels; the host
 * code only builds the mesh topology and launches.
 *
 * Conventions shared by every call:
 *  - "L-vector": one value per local GLL point, n_L = E (N+1)^3 values, laid
 *    out [e][k][j][i] with i fastest (the Fortran w(:,:,:,:) order of
 *    Listing 1).  Element e = ex + nelx (ey + nely ez).
 *  - Unless stated otherwise a vector argument is a DEVICE pointer owned by
 *    the caller.  The library owns everything inside a handle (geometric
 *    factors, mass, numbering, preconditioner, solver scratch).
 *  - dtype: SEM_F64 (double) or SEM_F32 (float).
 *  - stream: a cudaStream_t passed as void*; NULL means the legacy default
 *    stream.  Calls are asynchronous on that stream unless stated.
 *  - Errors: every call returns a sem_status; no exception crosses the ABI.
 *    sem_last_error() gives a thread-local message for the last failure.
 *  - A handle is not thread-safe: one host thread at a time per handle.
 *  - One CUDA device per process: the first sem_setup binds the device that
 *    is current then (per-order constant tables and kernel attributes are set
 *    up once per process); every later call must run with that device
 *    current.  Run one process per GPU to use several.
 */
#ifndef SEM_GB300_H
#define SEM_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sem_handle sem_handle;
typedef struct sem_batch sem_batch;
typedef struct sem_proj sem_proj;
typedef struct sem_schwarz sem_schwarz;

typedef enum {
  SEM_OK = 0,
  SEM_ERR_ARG = 1,        /* invalid argument (sizes, null pointers, dtype) */
  SEM_ERR_CUDA = 2,       /* a CUDA runtime call failed */
  SEM_ERR_NOCONV = 3,     /* solver hit maxit before reaching tol */
  SEM_ERR_BREAKDOWN = 4,  /* CG found <p, Hp> <= 0 or a NaN (operator not SPD) */
  SEM_ERR_TIMEOUT = 5,    /* a bounded device wait ran out */
  SEM_ERR_OOM = 6,        /* device allocation failed */
  SEM_ERR_STATE = 7       /* call not valid for this handle's state */
} sem_status;

enum { SEM_F64 = 0, SEM_F32 = 1 };

/* precision_flags of sem_setup: which copies of the geometric factors to keep */
enum { SEM_PREC_F64 = 1, SEM_PREC_F32 = 2 };

/* solver precision (sem_solve_opts.precision) */
enum { SEM_SOLVE_F64 = 0, SEM_SOLVE_MIXED = 1 };

/* FP64 Ax kernel selection (sem_set_f64_kernel) */
enum { SEM_F64_KERNEL_AUTO = 0,        /* double-float where supported, else native */
       SEM_F64_KERNEL_NATIVE = 1,      /* IEEE FP64 FMA (bound by the FP64 pipe) */
       SEM_F64_KERNEL_DOUBLEFLOAT = 2  /* float-pair arithmetic, FP64 in and out */
};

/* gather-scatter kernel selection (sem_set_dssum_kernel) */
enum { SEM_DSSUM_BOX = 0,       /* copies computed from the box topology (default) */
       SEM_DSSUM_SEGMENTS = 1   /* precomputed segment lists of shared local points */
};

/* vectors of the FP32 inner solves of SEM_SOLVE_MIXED (sem_set_inner_vectors) */
enum { SEM_INNER_AUTO = 0,      /* global where supported (constant h1, odd N), else local */
       SEM_INNER_LOCAL = 1,     /* L-vectors, assembled operator with gather-scatter passes */
       SEM_INNER_GLOBAL = 2     /* unique-dof vectors, element kernels assemble by atomics */
};

/* CG recurrences of SEM_SOLVE_F64 (sem_set_cg_variant) */
enum { SEM_CG_STANDARD = 0,     /* Jacobi-PCG, three kernels after the operator */
       SEM_CG_PIPELINED = 1     /* pipelined PCG: one reduction, one vector pass */
};

/* levels of the Schwarz preconditioner (sem_schwarz_create) */
enum { SEM_SCHWARZ_LOCAL = 1,   /* overlapping element subdomains, fast diagonalisation */
       SEM_SCHWARZ_COARSE = 2,  /* trilinear coarse level, fixed-count CG */
       SEM_SCHWARZ_BOTH = 3     /* the two-level additive method */
};

/* phases of sem_apply */
enum { SEM_APPLY_LOCAL = 1,     /* element operator, x-neighbour sums inside CTAs, mask */
       SEM_APPLY_FINISH = 2,    /* remaining gather-scatter passes */
       SEM_APPLY_FULL = 3       /* both */
};

/* Dirichlet face bits */
enum { SEM_FACE_XMIN = 1, SEM_FACE_XMAX = 2, SEM_FACE_YMIN = 4,
       SEM_FACE_YMAX = 8, SEM_FACE_ZMIN = 16, SEM_FACE_ZMAX = 32,
       SEM_FACE_ALL = 63 };

/* fields readable with sem_get_field */
enum { SEM_FIELD_X = 0, SEM_FIELD_Y = 1, SEM_FIELD_Z = 2,  /* GLL coordinates (n_L) */
       SEM_FIELD_G = 3,      /* geometric factors, [e][6][p^3], order G11,G22,G33,G12,G13,G23 */
       SEM_FIELD_B = 4,      /* lumped mass W detJ (n_L) */
       SEM_FIELD_MULT = 5,   /* multiplicity of each local point (n_L) */
       SEM_FIELD_MASK = 6,   /* Dirichlet mask 0/1 (n_L) */
       SEM_FIELD_GID = 7,    /* global number (n_L), written as int64 whatever dtype says */
       SEM_FIELD_DINV = 8    /* Jacobi inverse diagonal of the last solve's operator (n_L) */
};

/*
 * Mesh description: a structured nelx x nely x nelz box of hexahedra
 * (§2: "E non-overlapping hexahedral elements").  GLL nodes are placed at
 * x0 + (ex + (xi+1)/2) len/nelx, then, if deform_amp != 0, moved by
 * x += a sin(y) sin(z), y += a sin(z) sin(x), z += a sin(x) sin(y) evaluated
 * at the undeformed position.  xyz_gll, if not NULL, is a HOST array of
 * 3 * n_L doubles ([x | y | z], each an L-vector) that replaces the generated
 * coordinates (same box topology).  dirichlet_faces selects the faces with
 * u = 0 (§2, Eq. 5).
 */
typedef struct {
  int nelx, nely, nelz;
  double x0[3];
  double len[3];
  double deform_amp;
  const double* xyz_gll;
  int dirichlet_faces;
} sem_mesh_desc;

/*
 * sem_setup -- build a handle for polynomial order N (1 <= N <= 10).
 * Host: GLL nodes/weights, derivative matrix D (§2, Eq. 7-9), global
 * numbering, multiplicity, Dirichlet mask and the gather-scatter segment
 * lists (§3.2).  Device: GLL coordinates, geometric factors G (6 per point)
 * and mass B (§2, Eq. 9) in the precisions named by precision_flags.  Also
 * does the once-per-process setup of the kernels the handle's order uses
 * (constant tables, kernel attributes), so that later calls can be captured
 * into CUDA graphs from the first one.  Synchronises the stream before
 * returning (the first handle of an order in a process synchronises the
 * device).  *out receives the handle; release it with sem_destroy.
 * Errors: SEM_ERR_ARG (bad sizes or N, a non-positive Jacobian),
 * SEM_ERR_STATE (the current device is not the one an earlier sem_setup of
 * this process bound), SEM_ERR_OOM, SEM_ERR_CUDA.
 */
sem_status sem_setup(const sem_mesh_desc* mesh, int N, int precision_flags,
                     void* stream, sem_handle** out);

/* Release every device and host resource of the handle (NULL is a no-op). */
sem_status sem_destroy(sem_handle* h);

/* Message of the last failed call on this host thread ("" if none). */
const char* sem_last_error(void);

/*
 * sem_sync -- synchronise the stream, then report a device-side failure
 * recorded by an earlier asynchronous call on this handle: SEM_ERR_TIMEOUT if
 * a bounded wait inside a kernel gave up (the kernel then returned early and
 * its output is incomplete), SEM_ERR_ARG if sem_gather, sem_scatter_add or
 * sem_set_multiplicity met an index or a multiplicity out of range (the
 * entry was skipped).  Clears the record.
 */
sem_status sem_sync(sem_handle* h, void* stream);

/*
 * sem_selftest_timeout -- diagnostic: launches the bulk-copy Ax kernel with
 * an mbarrier that expects 16 bytes more than its copies deliver, so its
 * wait can never complete, with the given limit (0 < timeout_ms <= 2000).
 * Returns SEM_ERR_TIMEOUT when the kernel gave up, recorded the failure and
 * returned (the GPU context stays usable); SEM_OK would mean the wait was
 * not bounded.  Needs FP32 geometry and even N+1.
 */
sem_status sem_selftest_timeout(sem_handle* h, double timeout_ms, void* stream);

/* Sizes: local points n_L, unique global points, order N, elements E. */
sem_status sem_get_sizes(const sem_handle* h, int64_t* n_local, int64_t* n_global,
                         int* N, int64_t* E);

/*
 * Copy one setup field (SEM_FIELD_*) into the device buffer dst, converted
 * to dtype (SEM_FIELD_GID is always int64).  dst holds n_L values (6 n_L for
 * SEM_FIELD_G).  SEM_ERR_STATE if the field is not kept in that precision.
 */
sem_status sem_get_field(sem_handle* h, int which, void* dst, int dtype, void* stream);

/*
 * sem_ax -- w_L = (h1 A_L + h2 B_L) u_L element by element, no gather-scatter
 * (§2, Eq. 9; the ax_t compute of Listing 1).  If h1_field is not NULL it is
 * an L-vector of per-point coefficients (same dtype) that replaces h1 at
 * every GLL point.  u_L and w_L are distinct L-vectors of the given dtype.
 */
sem_status sem_ax(sem_handle* h, const void* u_L, void* w_L, double h1, double h2,
                  const void* h1_field, int dtype, void* stream);

/*
 * sem_set_f64_kernel -- choose how FP64 Ax (sem_ax with SEM_F64, the FP64
 * matvecs of sem_cg_solve and sem_apply_host) is computed.  GB300's FP64 pipe
 * runs FMA about 60 times slower than its FP32 pipes, which makes the native
 * kernel compute bound at roughly a tenth of the HBM rate.  The double-float
 * kernel (default where supported: N in {5, 7, 9}, constant h1, 16-byte
 * aligned vectors) keeps FP64 inputs and outputs, stores G and B as float
 * pairs (8 bytes per value) and evaluates every sum with error-free float
 * transformations (TwoSum for the derivatives of u, extraction against a
 * power-of-two bound for the geometric-factor products and the transposed
 * contractions); its error against FP64 is 1e-14 to a few 1e-13 relative to
 * the largest |w| of an element (smooth u, whose derivatives cancel, at the
 * high end; below 1e-12 in every case).  Range: the operator is linear, so the kernel
 * scales by exact powers of two to keep every intermediate inside FP32's
 * exponent range, and undoes the scaling on the FP64 result.  G and B of an
 * element whose largest magnitude lies outside [2^-16, 2^16), and h1 or h2
 * outside that range, are normalised at setup or per call; an element whose
 * largest |u| lies outside [2^-60, 2^76) (including subnormal-only elements)
 * is rescaled by its own maximum in the kernel.  So every finite FP64 input
 * keeps the stated accuracy, up to FP64's own overflow and underflow of the
 * result.  An element whose u holds an Inf or a NaN gives NaN at all of its
 * points (the native kernel lets them spread through the element's contractions
 * instead, so some of its points stay finite).
 * SEM_F64_KERNEL_NATIVE forces IEEE FP64 arithmetic (at N = 7 and 9 with the
 * even-odd split of D, about 20% fewer FP64 operations).  Returns SEM_ERR_ARG
 * for an unknown kind.
 */
sem_status sem_set_f64_kernel(sem_handle* h, int kind);

/* Tile chosen by sem_autotune (times in ms per Ax launch, -1 if not timed). */
typedef struct {
  int ax32_kernel;          /* FP32 Ax: 0 bulk-copy (TMA) pipeline, 1 global-load kernel */
  int ax32_stages;          /* bulk-copy stages in flight per CTA (1..3) */
  int ax32_elems_per_cta;   /* elements per CTA of the bulk-copy kernel (1 or 2) */
  int f64_stages;           /* double-float FP64 Ax: bulk-copy stages (1 or 2) */
  double ax32_ms, ax64_ms;  /* best measured times */
  int from_cache;           /* 1 if taken from the process or file cache */
} sem_tuning;

/*
 * sem_autotune -- time every candidate tile of the FP32 Ax (global loads, or
 * bulk copies with 1-3 stages and 1-2 elements per CTA) and of the
 * double-float FP64 Ax (1-2 stages) on this handle's geometry and keep the
 * fastest for all later calls on the handle.  Choices are cached per (order,
 * element-count bucket) for the process and, if the environment variable
 * SEM_AUTOTUNE_CACHE names a file, in that file.  Synchronises the stream;
 * allocates two scratch vectors while timing.  *out (may be NULL) receives
 * the choice.
 */
sem_status sem_autotune(sem_handle* h, void* stream, sem_tuning* out);

/* sem_set_tuning -- apply a tile choice (fields as in sem_tuning; the times
 * and from_cache are ignored).  SEM_ERR_ARG for a combination that does not
 * exist (stages 1-3 with 1 element per CTA, or 1-2 with 2; f64_stages 1-2). */
sem_status sem_set_tuning(sem_handle* h, const sem_tuning* t);

/*
 * sem_apply -- the assembled operator w_L = mask o QQ^T (h1 A_L + h2 B_L) u_L
 * (§2, Eq. 9-10; one CG matvec), the same result as sem_ax followed by
 * sem_dssum with the mask, computed with the gather-scatter split by
 * direction.  The element kernel walks segments of four consecutive
 * elements per CTA and sums the copies of x-interface points inside a
 * segment itself; short passes then add the x-pairs between segments and
 * the y- and z-pairs.  The copies of a point on several interfaces are summed
 * pair by pair, (w0 + w1) + (w2 + w3) ..., so FP64 results can differ from
 * sem_dssum's increasing-index order in the last bits.
 * phase: SEM_APPLY_FULL, or SEM_APPLY_LOCAL then SEM_APPLY_FINISH (the
 * finish phase must follow a local phase on the same handle, dtype and
 * vectors; splitting lets a caller time or overlap the two).  Orders,
 * dtypes or alignments the fused kernels do not cover (odd N, the native
 * FP64 kernel, a per-point h1 in FP64) run sem_ax and sem_dssum's kernels
 * instead, the local phase being the element operator and the finish phase
 * the whole gather-scatter.  u_L and w_L are distinct L-vectors of the
 * dtype (SEM_F64 or SEM_F32); SEM_ERR_ARG otherwise.
 */
sem_status sem_apply(sem_handle* h, const void* u_L, void* w_L, double h1, double h2,
                     const void* h1_field, int dtype, int phase, void* stream);

/*
 * sem_apply_global -- the same operator on global (unique-dof) vectors:
 * w_g = mask o Q^T (h1 A_L + h2 B_L) Q u_g (§2, Eq. 9-10 with the scatter Q
 * and gather Q^T applied by the element kernel itself).  u_g and w_g are
 * distinct FP32 device arrays of n_G values (sem_get_sizes), numbered
 * g = ix + gx (iy + gy iz) on the GLL lattice of the box, gx = N nelx + 1,
 * gy = N nely + 1 (the numbering of SEM_FIELD_GID).  Each element reads its
 * values from u_g, stores the points inside it and adds those on its faces
 * to w_g with atomics, so results can differ in the last bits from run to
 * run.  Needs FP32 geometry, odd N (even P) and n_L < 2^31; SEM_ERR_ARG
 * otherwise.  dtype must be SEM_F32.  Asynchronous on stream.
 */
sem_status sem_apply_global(sem_handle* h, const void* u_g, void* w_g, double h1, double h2,
                            int dtype, void* stream);

/*
 * sem_to_global -- out_g[g] = in_L at a local copy of g (FP32 out_g of n_G
 * values; in_L an L-vector of dtype SEM_F32 or SEM_F64 that must be
 * continuous, every copy of a point holding the same value, as sem_dssum or
 * sem_apply leave it).  Needs n_L < 2^31.  Asynchronous on stream.
 */
sem_status sem_to_global(sem_handle* h, const void* in_L, void* out_g, int dtype, void* stream);

/*
 * sem_set_cg_variant -- choose the recurrences of the FP64 solves
 * (SEM_SOLVE_F64) of sem_cg_solve.  SEM_CG_PIPELINED is the pipelined PCG of
 * Ghysels and Vanroose (the non-blocking Krylov method the paper's outlook
 * names, §10): both inner products of an iteration come from one reduction
 * that is independent of the operator, and all vectors (x, r, u = M r,
 * w = H u, and the z, q, s, p recurrences) are updated in one pass; in exact
 * arithmetic its iterates are those of standard PCG.  When its recurrence
 * residual reaches tol, the true residual is checked and the recurrences
 * restart from it (up to 6 cycles; info.outer_iters counts them).  Needs six
 * more FP64 L-vectors, kept on the handle.
 */
sem_status sem_set_cg_variant(sem_handle* h, int kind);

/*
 * sem_set_inner_vectors -- choose the vectors of the FP32 inner PCG of
 * SEM_SOLVE_MIXED: SEM_INNER_LOCAL runs it on L-vectors with sem_apply's
 * operator; SEM_INNER_GLOBAL on global vectors with sem_apply_global's
 * (a third fewer bytes per vector pass at N = 7, no gather-scatter passes);
 * SEM_INNER_AUTO (the default) takes the global form where it is supported
 * (constant h1, odd N) and the local one elsewhere.  SEM_INNER_GLOBAL on an
 * unsupported problem falls back to the local form.  The FP64 outer
 * refinement is the same in all cases.
 */
sem_status sem_set_inner_vectors(sem_handle* h, int kind);

/*
 * sem_dssum -- in place w_L <- QQ^T w_L: every local copy of a global point
 * receives the sum of all its copies, summed in increasing local index
 * (§2, Eq. 10; §3.2).  With apply_mask != 0 the Dirichlet points are then
 * set to 0.
 */
sem_status sem_dssum(sem_handle* h, void* w_L, int apply_mask, int dtype, void* stream);

/*
 * sem_set_dssum_kernel -- choose how QQ^T runs: SEM_DSSUM_BOX computes the
 * copies of every shared point from the box topology (no index lists read),
 * SEM_DSSUM_SEGMENTS walks precomputed segment lists of shared local points
 * (the gslib-style layout of §3.2).  Both sum the copies of a point in
 * increasing local index, so their results are bitwise identical.
 */
sem_status sem_set_dssum_kernel(sem_handle* h, int kind);

/* b_L = mask o QQ^T (B f_L): the discrete right-hand side of §2, Eq. 6 for a
 * nodal source f (FP64 device L-vectors). */
sem_status sem_rhs(sem_handle* h, const double* f_L, double* b_L, void* stream);

/* Solver options; sem_solve_opts_default fills the defaults noted here. */
typedef struct {
  double h1;              /* constant diffusion coefficient (1.0) */
  double h2;              /* mass coefficient (0.0) */
  const double* h1_field; /* device L-vector of per-point h1 or NULL (NULL) */
  double tol;             /* relative residual ||b - Hx|| / ||b|| (1e-8) */
  int maxit;              /* CG iteration limit, counted over inner iterations (20000) */
  int precision;          /* SEM_SOLVE_F64 or SEM_SOLVE_MIXED (SEM_SOLVE_F64) */
  double inner_tol;       /* mixed: FP32 inner relative tolerance (1e-4); a step
                             whose outer residual needs less reduction than that
                             to reach tol stops at 0.5 tol / (outer rel. residual) */
  int max_outer;          /* mixed: refinement steps limit (30) */
  int check_every;        /* iterations per host convergence check (16) */
  int use_graph;          /* capture check_every iterations in a CUDA graph (1) */
  int x0_is_zero;         /* 1: ignore x_L on input and start from 0 (1) */
  void* stream;           /* stream of the solve (NULL) */
} sem_solve_opts;

typedef struct {
  int iters;          /* CG iterations (all inner iterations for mixed) */
  int outer_iters;    /* refinement steps (0 for SEM_SOLVE_F64) */
  double rel_res;     /* final FP64 relative residual in the unique-dof norm */
  int status;         /* sem_status of the solve */
} sem_solve_info;

void sem_solve_opts_default(sem_solve_opts* o);

/*
 * sem_cg_solve -- solve mask o QQ^T (h1 A_L + h2 B_L) x = b by Jacobi-
 * preconditioned CG (§2 end; §4 uses PCG for the Helmholtz solves).  b_L is
 * an assembled, masked FP64 L-vector (as from sem_rhs); x_L (FP64) receives
 * the continuous solution.  Dots are the unique-dof inner products
 * sum_L a b / mult accumulated in FP64.  SEM_SOLVE_MIXED runs FP32 inner PCG
 * (FP32 G, B and vectors) inside an FP64 iterative-refinement loop whose
 * residual r = b - Hx and update x += d are FP64.  Stops when the FP64
 * relative residual <= tol.  Synchronises the stream once per check_every
 * iterations and at the end.  Returns SEM_ERR_NOCONV / SEM_ERR_BREAKDOWN
 * (with info filled) when the solve fails.
 */
sem_status sem_cg_solve(sem_handle* h, const double* b_L, double* x_L,
                        const sem_solve_opts* opts, sem_solve_info* info);

/*
 * Two-level additive overlapping Schwarz preconditioner (§4: Neko's pressure
 * preconditioner, M^-1 = R_0^T A_0^-1 R_0 + sum_e R_e^T A~_e^-1 R_e).
 * Local level: each element grown by one GLL point into its neighbours
 * ((N+3)^3 lattice points, none outside the box, no Dirichlet points); A~_e
 * is the Kronecker sum of the 1D stiffness and mass matrices of the element
 * and its neighbours on the undeformed box spacing (len / nel of the mesh
 * description), inverted by fast diagonalisation; overlapping corrections
 * add.  Coarse level: trilinear functions on the element vertices, Galerkin
 * A_0 = R_0 H R_0^T from 8 x 8 element matrices, solved by coarse_iters
 * Jacobi-CG iterations from zero.  Applied in FP32 (FP64 in and out).
 * sem_schwarz_create: for H = h1 A + h2 B (h1 > 0, h2 >= 0) and N >= 2 (so
 * that the point a subdomain takes from a neighbour lies inside it); levels is a
 * SEM_SCHWARZ_* value; synchronises the stream.  The object refers to h,
 * which must outlive it.  sem_schwarz_apply: z_L = M^-1 r_L for a continuous,
 * masked FP64 L-vector r_L (distinct from z_L); z_L is continuous and
 * masked.  Asynchronous on stream.
 */
sem_status sem_schwarz_create(sem_handle* h, double h1, double h2, int levels, int coarse_iters,
                              void* stream, sem_schwarz** out);
sem_status sem_schwarz_apply(sem_schwarz* s, const double* r_L, double* z_L, void* stream);
sem_status sem_schwarz_destroy(sem_schwarz* s);

/*
 * sem_gmres_solve -- flexible GMRES(restart) with right preconditioning (§4,
 * Table 2: Neko's pressure solver) for mask o QQ^T (h1 A_L + h2 B_L) x = b in
 * FP64: Arnoldi with classical Gram-Schmidt applied twice in the unique-dof
 * inner product, Givens rotations, x formed from the preconditioned
 * directions; restarts from the true residual.  precond: a Schwarz object
 * made for the same handle (and coefficients), or NULL for point Jacobi.
 * opts: h1, h2, tol (relative residual), maxit (iterations), x0_is_zero,
 * stream as for sem_cg_solve (h1_field must be NULL).  With precision
 * SEM_SOLVE_MIXED, a Schwarz preconditioner and a handle that allows global
 * vectors (FP32 geometry, odd N), the solve is FP64 iterative refinement on
 * L-vectors around an FP32 flexible GMRES on global vectors (operator as
 * sem_apply_global, preconditioner on global vectors), each inner solve to
 * the relative tolerance of sem_cg_solve's mixed solves (inner_tol,
 * max_outer); info.outer_iters then counts refinement steps.  Otherwise the
 * FP64 solve runs.
 * The workspace (2 restart + 2 FP64 L-vectors) is allocated on the first
 * solve and kept on the handle until it is destroyed.  Synchronises once per
 * iteration.  info: iterations, restart cycles in outer_iters, final
 * relative residual.  restart in [1, 32].
 */
sem_status sem_gmres_solve(sem_handle* h, const double* b_L, double* x_L,
                           const sem_solve_opts* opts, int restart, sem_schwarz* precond,
                           sem_solve_info* info);

/*
 * Batched solves.  sem_batch_create groups n (<= 256) handles, each built with
 * SEM_PREC_F32 and an odd N (even points per direction), into a batch that
 * advances all their solves together: every stage of an FP32 inner CG
 * iteration (the operator, the vector updates with per-problem dot products)
 * is one kernel launch over all problems (the element kernels one persistent
 * launch per order present), and batches of iterations are captured in a
 * CUDA graph.  The inner PCG runs on global vectors (as sem_apply_global)
 * unless a handle asks for L-vectors (sem_set_inner_vectors).  Each problem refines in FP64 as
 * in sem_cg_solve with SEM_SOLVE_MIXED (constant h1, h2 per problem).
 * sem_batch_solve: b_L[p] and x_L[p] are device pointers (host array of n
 * pointers) as for sem_cg_solve on handle p; h1[p], h2[p] the coefficients;
 * opts as for sem_cg_solve (precision ignored: always mixed); infos receives
 * n results.  The call synchronises.  The batch does not own the handles.
 */
sem_status sem_batch_create(sem_handle* const* handles, int n, sem_batch** out);
sem_status sem_batch_solve(sem_batch* b, const double* const* b_L, double* const* x_L,
                           const double* h1, const double* h2, const sem_solve_opts* opts,
                           sem_solve_info* infos);
sem_status sem_batch_destroy(sem_batch* b);
/* sem_batch_set_concurrency: concurrent = 1 launches the element kernels of
 * the order classes of an inner iteration as concurrent branches (side
 * streams forked from and joined back into the solve's stream; parallel paths
 * of the iteration graph), so that the persistent grids of the classes can
 * fill one another's tails; 0 (the default) launches them one after another.
 * The classes touch disjoint problems, so either way computes the same
 * iteration.  SEM_ERR_ARG for a NULL batch or a flag other than 0 or 1. */
sem_status sem_batch_set_concurrency(sem_batch* b, int concurrent);

/*
 * Projection onto previous solutions for successive right-hand sides (§4,
 * Table 2: Neko keeps 20 previous pressure solutions).  A space of at most m
 * previous solutions of H x = b on handle h is kept H-orthonormal in the
 * unique-dof inner product, with H X stored beside it (2 m FP64 L-vectors,
 * owned by the space).  sem_proj_solve(b, x): x_bar = X X^T b (the best
 * approximation in the H-norm from the space, no matvec), then PCG (any
 * sem_solve_opts precision) on the remainder to ||b - H x|| <= tol ||b||,
 * x = x_bar + correction; the correction is H-orthonormalised against the
 * space (Gram-Schmidt twice, one matvec) and appended, and a full space
 * restarts from x alone.  info->iters counts the PCG iterations of the
 * correction (0 when the projection already meets tol), info->rel_res is
 * ||b - H x|| / ||b|| of the returned x.  Constant h1 only (h1_field must be
 * NULL); the same h1, h2 must be used for every solve of a space (reset it
 * otherwise).  Synchronises the stream.  Errors: SEM_ERR_ARG (m outside
 * [0, 64], null pointers), the statuses of sem_cg_solve.
 */
sem_status sem_proj_create(sem_handle* h, int m, sem_proj** out);
sem_status sem_proj_solve(sem_proj* p, const double* b_L, double* x_L,
                          const sem_solve_opts* opts, sem_solve_info* info);
sem_status sem_proj_size(const sem_proj* p, int* l);     /* vectors in the space */
sem_status sem_proj_reset(sem_proj* p);                  /* empty the space */
sem_status sem_proj_destroy(sem_proj* p);

/*
 * sem_helmholtz_grad --g_L = -(D^ lambda)^T G (D^ u) at every local point,
 * D^ the reference gradient: the derivative of lambda^T H(h1) u with
 * respect to each local h1 value, negated -- the adjoint gradient dL/dh1 when
 * lambda solves H lambda = mask o QQ^T dL/du (structure of §2, Eq. 9).
 * FP64 device L-vectors.
 */
sem_status sem_helmholtz_grad(sem_handle* h, const double* u_L, const double* lambda_L,
                              double* g_L, void* stream);

/*
 * sem_dot -- *out = sum_L a b / mult: the inner product on the unique degrees
 * of freedom (every global point counted once for continuous a, b), i.e. the
 * dot product of the Krylov solvers (§2 end; on one device it replaces the
 * MPI_Allreduce of every CG dot, §8 Eq. 14).  a, b: FP64 device L-vectors;
 * out: one device double.  Accumulated in FP64 with a fixed reduction order
 * (bitwise reproducible).  Uses the handle's reduction scratch: do not
 * overlap it with other calls on the same handle.
 */
sem_status sem_dot(sem_handle* h, const double* a, const double* b, double* out, void* stream);

/*
 * sem_dot_noalloc -- the same inner product as sem_dot, for callers that must
 * not allocate device memory at the call site (for example while a stream is
 * being captured into a CUDA graph, or under a device-memory budget fixed up
 * front).  The paper has no counterpart; this is a library convenience.
 * Allocates nothing: the partial sums live in a static device array of the
 * library (128 KiB, held by every GPU that loads the library until exit), so
 * n_L may be at most 67,108,864 local points (SEM_ERR_ARG beyond that).  All
 * calls share the array; calls whose kernels overlap on the GPU race, so
 * order them on one stream.  sem_setup looks up the array's address, so a
 * first call inside a stream capture makes no synchronous call.
 */
sem_status sem_dot_noalloc(sem_handle* h, const double* a, const double* b, double* out,
                           void* stream);
/* the largest n_L sem_dot_noalloc accepts (16,384 blocks of 4,096 points) */
enum { SEM_NOALLOC_MAX_POINTS = 67108864 };

/*
 * Element partition across processes (§3.2, Algorithm 1).
 *
 * Each rank owns a sub-box of the element box and its own handle: sem_setup
 * on the sub-box (x0 and len of its elements, the same element size and
 * deformation map as the whole box) with Dirichlet faces only where the
 * sub-box touches the global boundary.  The rank's sem_apply then sums the
 * copies of a shared point inside the rank; the copies on other ranks are
 * added by an interface exchange that the caller runs (over MPI, NCCL or
 * gloo): for each direction x, then y, then z, gather the values of the
 * rank's face planes into buffers, send them to the neighbours across those
 * faces, and add what the neighbours sent to every local copy of the face
 * points.  Summing direction by direction also completes the points on the
 * edges and corners shared by 4 or 8 ranks.  The Krylov dots end in a sum
 * over the ranks.  The calls below are the device side of that scheme;
 * paper_2107_01243_gb300/partition.py builds the index lists, runs the
 * exchange over torch.distributed and drives a partitioned PCG with them.
 *
 * Index arrays are DEVICE arrays of int64 owned by the caller.  Indices are
 * checked in the kernels: an entry outside its vector is skipped and
 * recorded as SEM_ERR_ARG for sem_sync.  All calls are asynchronous on
 * stream.
 */

/* dst[t] = src_L[idx[t]] for t < n (src_L an L-vector of this handle). */
sem_status sem_gather(sem_handle* h, const double* src_L, const int64_t* idx, int64_t n,
                      double* dst, void* stream);

/* dst_L[idx[t]] += src[pos[t]] for t < n; src holds n_src values and the
 * idx[t] must be distinct (each local copy receives one value per call). */
sem_status sem_scatter_add(sem_handle* h, double* dst_L, const int64_t* idx, const int64_t* pos,
                           int64_t n, const double* src, int64_t n_src, void* stream);

/* Replace the multiplicities the dots divide by (sem_dot, the solvers'
 * <a, b> = sum_L a b / mult) with mult_L, the number of copies of each local
 * point over ALL ranks (>= 1; the exchange applied to the handle's own
 * multiplicity, SEM_FIELD_MULT, gives it).  sem_dot then returns this rank's
 * share of the unique-dof inner product. */
sem_status sem_set_multiplicity(sem_handle* h, const double* mult_L, void* stream);

/* d_L = QQ^T diag(h1 A_L + h2 B_L) inside this handle (no mask): the Jacobi
 * diagonal before the interface exchange. */
sem_status sem_jacobi_diag(sem_handle* h, double h1, double h2, double* d_L, void* stream);

/* dinv_L = mask / d_L (0 on Dirichlet points). */
sem_status sem_jacobi_invert(sem_handle* h, const double* d_L, double* dinv_L, void* stream);

/* One PCG vector step: x += alpha p, r -= alpha w, z = dinv o r, and this
 * rank's shares of <r, z> and <r, r> (unique-dof weights) into dots[0],
 * dots[1] (a DEVICE array of 2 doubles). */
sem_status sem_cg_update(sem_handle* h, double alpha, const double* p, const double* w,
                         double* x, double* r, const double* dinv, double* z, double* dots,
                         void* stream);

/* p = z + beta p. */
sem_status sem_cg_direction(sem_handle* h, double beta, const double* z, double* p,
                            void* stream);

/*
 * sem_apply_host -- w = mask o QQ^T A_L u with HOST buffers: copies u_host
 * (n_L values of dtype) to the device, applies the assembled operator as
 * sem_apply does, copies the result to w_host and synchronises the stream.
 * Pinned host memory gives full copy bandwidth.  In FP64 on the fused path
 * (N in {5, 7, 9}, at least two element planes in z) the box is cut into up
 * to 8 slabs of element planes and the copies overlap the work: slab q is
 * copied in while earlier slabs are computed and copied out, on streams of
 * the handle ordered after the caller's stream; the result is the same, bit
 * for bit, as sem_apply's.
 */
sem_status sem_apply_host(sem_handle* h, const void* u_host, void* w_host, int dtype,
                          void* stream);

#ifdef __cplusplus
}
#endif
#endif
