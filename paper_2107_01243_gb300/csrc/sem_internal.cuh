// Internal declarations shared by the library's translation units.
#pragma once
#include <type_traits>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>
#include <string>
#include <vector>
#include <memory>
#include <algorithm>
#include <cmath>
#include <stdexcept>

#include "../../include/sem.h"

namespace sem {

struct GmresWork;                    // gmres.cu
struct GmresWorkF;                   // gmres.cu
struct HostPipe;                     // apply.cu

constexpr int kMaxN = 10;            // highest supported polynomial order
constexpr int kMaxP = kMaxN + 1;
// blocks of every reduction kernel (four per SM of a 152-SM GB300).  A fixed
// count, not the device's: the partial sums, and so the rounding of every dot
// product, are then the same on any device.
constexpr int kRedBlocks = 608;
constexpr int kRedThreads = 256;
constexpr int kFusedPartials = 2048;   // partials of the element kernels' fused <p, Hp>
constexpr uint64_t kWaitTimeoutNs = 2000000000ull;   // bounded device waits give up after 2 s

// SM count of the device the library is bound to, set by the first sem_setup
// (every entry point that launches a kernel holds a handle, so it is set by then).
// Grids of the grid-stride kernels are sized in multiples of it.
int sem_num_sms();

// ------------------------------------------------------------------ errors
struct Error : std::runtime_error {
  sem_status code;
  Error(sem_status c, const std::string& m) : std::runtime_error(m), code(c) {}
};

void set_last_error(const std::string& msg);

#define SEM_CUDA(call)                                                          \
  do {                                                                          \
    cudaError_t e__ = (call);                                                   \
    if (e__ != cudaSuccess)                                                     \
      throw ::sem::Error(e__ == cudaErrorMemoryAllocation ? SEM_ERR_OOM         \
                                                         : SEM_ERR_CUDA,       \
                         std::string(#call) + ": " + cudaGetErrorString(e__));  \
  } while (0)

#define SEM_CHECK_LAUNCH() SEM_CUDA(cudaGetLastError())

#define SEM_REQUIRE(cond, msg)                                                  \
  do {                                                                          \
    if (!(cond)) throw ::sem::Error(SEM_ERR_ARG, msg);                          \
  } while (0)

// Run a body, translating exceptions into a status + thread-local message.
template <class F>
sem_status guarded(F&& f) {
  try {
    f();
    set_last_error("");
    return SEM_OK;
  } catch (const Error& e) {
    set_last_error(e.what());
    return e.code;
  } catch (const std::exception& e) {
    set_last_error(e.what());
    return SEM_ERR_CUDA;
  }
}

// NVTX range around a scope: profilers (Nsight Systems, ncu --nvtx) show
// which API call issued which kernels.  NVTX 3 is header-only; with no tool
// attached a range costs a few nanoseconds.
struct TraceRange {
  explicit TraceRange(const char* name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange&) = delete;
  TraceRange& operator=(const TraceRange&) = delete;
};

// guarded() inside an NVTX range named after the API call
template <class F>
sem_status guarded(const char* name, F&& f) {
  TraceRange range(name);
  return guarded(std::forward<F>(f));
}

// ------------------------------------------------------------------ device buffers
template <class T>
struct DevBuf {
  T* ptr = nullptr;
  size_t n = 0;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf() { release(); }
  void alloc(size_t count) {
    release();
    if (count == 0) return;
    SEM_CUDA(cudaMalloc(&ptr, count * sizeof(T)));
    n = count;
  }
  void release() {
    if (ptr) cudaFree(ptr);
    ptr = nullptr;
    n = 0;
  }
  void upload(const T* h, size_t count, cudaStream_t s) {
    SEM_CUDA(cudaMemcpyAsync(ptr, h, count * sizeof(T), cudaMemcpyHostToDevice, s));
  }
};

// Division of 32-bit unsigned n < 2^31 by a runtime divisor d >= 1 as a
// multiply and shift (Granlund and Montgomery, 1994): q = (umulhi(n, m) + n) >> s
struct FastDiv {
  uint32_t d, m, s;
  __host__ __device__ FastDiv() : d(1), m(0), s(0) {}
  explicit FastDiv(uint32_t dd) : d(dd) {
    s = 0;
    while ((1ull << s) < dd) ++s;
    m = dd == 1 ? 0u : (uint32_t)((((1ull << 32) * ((1ull << s) - dd)) / dd) + 1);
  }
  __device__ __forceinline__ uint32_t div(uint32_t n) const {
    return d == 1 ? n : (__umulhi(n, m) + n) >> s;
  }
};

// CG scalars kept on the device so that iterations need no host round trip.
struct CGState {
  double rz;        // <r, z> of the current residual
  double pw;        // <p, H p>
  double rr;        // <r, r>
  double bb;        // <b, b>
  double alpha, beta;
  double tol2;      // (tol)^2 * <b,b>: convergence threshold on <r,r>
  int iter;         // completed iterations
  int done;         // 1 once converged or failed
  int status;       // SEM_OK / SEM_ERR_BREAKDOWN
  int maxit;
  unsigned int counter;   // last-block-done ticket for the reductions
  int pad;
};

// Precision-specific operator data (geometry in one float type).
template <class T>
struct OpData {
  DevBuf<T> G;      // [E][6][p^3]
  DevBuf<T> B;      // [E][p^3]
  DevBuf<T> D;      // [p][p] row-major D[i][l] = l_l'(xi_i)
  DevBuf<T> dinv;   // Jacobi inverse diagonal (mask folded in)
  DevBuf<T> dmi;    // dinv / mult (FP64 only: <r, z> = sum r^2 dinv / mult)
  DevBuf<T> h1f;    // per-point h1 in this precision (mixed solves)
};

}  // namespace sem

struct sem_handle {
  int N = 0, P = 0, P3 = 0;
  int nelx = 0, nely = 0, nelz = 0;
  int64_t E = 0, nL = 0, nG = 0;
  int prec_flags = 0;
  int faces = 0;
  double len[3] = {1.0, 1.0, 1.0};         // box lengths of the mesh description
  std::vector<double> xi, wq, Dh;          // host GLL nodes, weights, D

  sem::DevBuf<double> coords;               // [3][nL]
  sem::OpData<double> f64;
  sem::OpData<float> f32;
  sem::DevBuf<float> imult;                 // 1 / multiplicity (exact)
  sem::DevBuf<uint8_t> mask;                // 0 on Dirichlet points
  sem::DevBuf<int64_t> gid;                 // global numbers
  sem::DevBuf<int> dev_err;                 // device-side error word (SEM_ERR_TIMEOUT)
  sem::DevBuf<float2> gdf, bdf;             // G and B as float pairs (double-float kernel)
  sem::DevBuf<int> escale;                  // per element: exponents sG | sB << 16 of gdf, bdf
  int f64_kernel = SEM_F64_KERNEL_AUTO;     // which FP64 Ax kernel runs
  struct Tune {
    int ax32_ldg = 0;          // 1: FP32 Ax by the global-load kernel instead of bulk copies
    int ax32_variant = 1;      // bulk-copy variant: (stages, elements per CTA), see ax_tma.cu
    int df_variant = 0;        // double-float Ax: 0 = one stage, 1 = two stages
    int tuned = 0;
  } tune;

  // gather-scatter: segments of >= 2 local copies of one global point,
  // unmasked ones first; masked local points listed separately
  int64_t nseg_all = 0, nseg_free = 0, nmasked = 0;
  sem::DevBuf<int> seg_ptr;                 // [nseg_all + 1]
  sem::DevBuf<int> seg_idx;                 // local indices
  sem::DevBuf<int> masked_idx;              // local indices with mask 0
  int64_t nmasked_free = 0;                 // masked points owned by one element
  sem::DevBuf<int> masked_free_idx;
  int dssum_kernel = SEM_DSSUM_BOX;         // which gather-scatter kernel runs
  int segments_built = 0;                   // segment lists exist (built on first use)

  // solver scratch (allocated on first use)
  sem::DevBuf<double> r, p, w, x64, tmp64;
  sem::DevBuf<float> r32, p32, w32, x32;
  // FP32 inner solves on global vectors (n_G values padded with zeros to a
  // multiple of 4): residual, direction, H p, correction, Jacobi diagonal
  sem::DevBuf<float> rg, pg, wg, xg, dinvg;
  int inner_vectors = SEM_INNER_AUTO;       // sem_set_inner_vectors
  int cg_variant = SEM_CG_STANDARD;         // sem_set_cg_variant
  sem::DevBuf<double> pipe_u, pipe_z, pipe_q, pipe_s, pipe_m, pipe_n;   // pipelined CG
  // reduction partials (B = kRedBlocks): [0,2B) solves, [2B,3B) sem_dot,
  // [4B,4B+F) the element kernels' fused <p, Hp>, [4B+F,6B+F) sem_cg_update
  sem::DevBuf<double> partials;
  // [4]: outer/FP64, inner/FP32, sem_dot ticket, sem_cg_update ticket
  sem::DevBuf<sem::CGState> state;
  // host staging for sem_apply_host
  sem::DevBuf<double> stage_in, stage_out;
  std::shared_ptr<sem::GmresWork> gmres;    // GMRES workspace, kept between solves
  std::shared_ptr<sem::GmresWorkF> gmres32; // mixed-precision GMRES workspace
  std::shared_ptr<sem::HostPipe> host_pipe; // streams of the pipelined sem_apply_host
  // The FP32 inner solves of the mixed-precision solvers work on rscale times
  // the FP64 residual and add the correction divided by it: a power of two
  // chosen from ||b|| that keeps the FP32 vectors in FP32's normal range
  double rscale = 1.0;
  double dinv_h1 = NAN, dinv_h2 = NAN;
  const void* dinv_h1f = nullptr;
  int dinv_valid = 0;
};

// segment lists and the Dirichlet list of the segment-list gather-scatter
void sem_build_segments(sem_handle* h, cudaStream_t s);

namespace sem {

// ---- setup.cu
void gll_host(int N, std::vector<double>& xi, std::vector<double>& w, std::vector<double>& D);

// ---- ax.cu: w = (h1 A + h2 B) u (no dssum).  state may be null.
template <class T>
void launch_ax(const sem_handle* h, const OpData<T>& op, const T* u, T* w, T h1, T h2,
               const T* h1f, const CGState* state, cudaStream_t s);
// bulk-copy staged variant (even P, 16-byte aligned vectors)
template <class T>
bool tma_ax_supported(const sem_handle* h, const void* u, const void* w, const void* h1f);
// the assembled operator (apply.cu); phase = SEM_APPLY_* bits.  pwst (may be
// NULL): a CG state that the element kernel gives <p, H p> and alpha (p = u);
// returns whether it did
template <class T>
bool apply_fused_supported(const sem_handle* h, const void* u, const void* w, const void* h1f);
template <class T>
bool launch_apply(sem_handle* h, const OpData<T>& op, const T* u, T* w, T h1, T h2, const T* h1f,
                  const CGState* st, int phase, cudaStream_t s, CGState* pwst = nullptr);
template <class T>
void launch_ax_tma(const sem_handle* h, const OpData<T>& op, const T* u, T* w, T h1, T h2,
                   const T* h1f, const CGState* state, int* err, uint64_t timeout_ns,
                   uint32_t starve_bytes, cudaStream_t s);
// FP64-accurate double-float variant (even P in {6, 8, 10}, constant h1)
bool df_ax_supported(const sem_handle* h, const void* u, const void* w, const void* h1f);
void df_prepare(const sem_handle* h);          // once-per-process setup, run by sem_setup
void eo_prepare(const sem_handle* h);          // the same for the IEEE FP64 even-order kernel
void noalloc_prepare();                        // resolves sem_dot_noalloc's static array
void launch_ax_df(const sem_handle* h, const double* u, double* w, double h1, double h2,
                  const CGState* state, cudaStream_t s);
// diag(H_L) at every local point
template <class T>
void launch_local_diag(const sem_handle* h, const OpData<T>& op, T* d, T h1, T h2,
                       const T* h1f, cudaStream_t s);

// ---- dssum.cu
template <class T>
void launch_dssum(const sem_handle* h, T* w, bool apply_mask, const CGState* state,
                  cudaStream_t s);

// index-free variant for the structured box (same summation order)
template <class T>
void launch_dssum_box(const sem_handle* h, T* w, bool apply_mask, const CGState* state,
                      cudaStream_t s);

// ---- cg.cu: pieces of the mixed-precision solve reused by the batched solver
double inner_target(double inner_tol, double tol, double rel);
void mixed_prepare(sem_handle* h, const sem_solve_opts& o, cudaStream_t s);
void outer_norm_b(sem_handle* h, const double* b, cudaStream_t s);    // <b,b> -> state[0].bb
void outer_residual(sem_handle* h, const double* b, const double* x, const sem_solve_opts& o,
                    cudaStream_t s);                                   // r, r32, <r,r> -> state[0]
void outer_update(sem_handle* h, double* x, cudaStream_t s);          // x += x32 / rscale
// rscale from <b,b> in state[0] (reads it: synchronises the stream)
void inner_scale_from_b(sem_handle* h, cudaStream_t s);
// global-vector inner solves: vectors and the global Jacobi diagonal; the
// FP64 residual r (state[0].rr) and its global copy rg
void glob_prepare(sem_handle* h, cudaStream_t s);
void outer_residual_global(sem_handle* h, const double* b, const double* x,
                           const sem_solve_opts& o, cudaStream_t s);
CGState state_to_host(const CGState* d, cudaStream_t s, int* dev_err);

// ---- global.cu: the FP32 operator on global vectors, w_g = mask Q^T H_L Q u_g
// (w_g must hold zeros at unmasked element-face points); pwst as launch_apply
bool glob_supported(const sem_handle* h);
int64_t glob_padded(const sem_handle* h);          // n_G rounded up to a multiple of 4
bool launch_apply_global(const sem_handle* h, const float* u, float* w, float h1, float h2,
                         const CGState* st, CGState* pwst, cudaStream_t s);
template <class Tin>
void to_global(const sem_handle* h, const Tin* in, float* out, cudaStream_t s,
               double scale = 1.0);                                    // owner copies x scale
void add_from_global(const sem_handle* h, double* x, const float* d, cudaStream_t s,
                     double scale = 1.0);                              // x += d x scale

// ---- apply.cu: FP64 operator with host buffers, copies overlapped by slabs
bool host_pipeline_supported(const sem_handle* h, const void* din, const void* dout);
void apply_host_pipelined(sem_handle* h, const double* u_host, double* w_host, double* din,
                          double* dout, cudaStream_t user);

// ---- cg.cu: FP32 CG steps on vectors padded to a multiple of 4 with zeros
// (nv4 = padded length / 4), plain dots (each entry counted once); w must
// hold zeros before an operator assembles into it (init and update clear it).
// Used by the global-vector inner solves and the Schwarz coarse level.
void vcg_init(int64_t nv4, const float* r, const float* dinv, float* p, float* x, float* w,
              CGState* st, double* partials, double tol, int maxit, cudaStream_t s);
void vcg_pw(int64_t nv4, const float* p, const float* w, CGState* st, double* partials,
            cudaStream_t s);
void vcg_update(int64_t nv4, float* x, float* r, const float* p, float* w, const float* dinv,
                CGState* st, double* partials, cudaStream_t s);
void vcg_pupd(int64_t nv4, float* p, const float* r, const float* dinv, const CGState* st,
              cudaStream_t s);
// Jacobi inverse diagonal of (h1, h2) for the FP64 operator (L-vector, masked)
const double* jacobi_dinv64(sem_handle* h, double h1, double h2, cudaStream_t s);
// w = mask o QQ^T H x, r = b - w and <r, r> into st->rr (FP64 L-vectors)
void residual_f64(sem_handle* h, const double* b, const double* x, double h1, double h2,
                  double* w, double* r, CGState* st, cudaStream_t s);

// ---- schwarz.cu: z = M^-1 r (FP64 L-vectors)
void schwarz_apply(sem_schwarz* sw, const double* r, double* z, cudaStream_t s);
// z_g = M^-1 r_g on FP32 global vectors (z_g padded like r_g; padding stays zero)
void schwarz_apply_global(sem_schwarz* sw, const float* r_g, float* z_g, cudaStream_t s);
sem_handle* schwarz_handle(const sem_schwarz* sw);

// ---- grad.cu
void launch_grad(const sem_handle* h, const double* u, const double* lam, double* g,
                 cudaStream_t s);

}  // namespace sem
