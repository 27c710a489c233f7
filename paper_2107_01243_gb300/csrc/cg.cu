// Jacobi-preconditioned CG on the matrix-free operator and FP32-inner / FP64
// iterative refinement (arXiv 2107.01243 §2 end: matrix-free Krylov
// solvers; §4: PCG for the Helmholtz systems; Table 1: variable precision).
//
// Iteration (unique-dof inner products <a,b> = sum_L a b / mult):
//   w = mask o QQ^T H_L p;  alpha = <r,z>/<p,w>;  x += alpha p;  r -= alpha w;
//   stop if <r,r> <= tol^2 <b,b>;  z = dinv r;  beta = <r,z>_new/<r,z>;  p = z + beta p
// alpha, beta and the stop flag live on the device (CGState); every kernel
// returns at once when the flag is set, so a batch of iterations can be
// captured in a CUDA graph and the host reads the state once per batch.
//
// The mixed solve's FP32 inner PCG runs on global (unique-dof) vectors when
// the handle allows it (glob_iterations: the operator of global.cu and
// padded float4 vector kernels), else on L-vectors.  The FP64 solve can also
// run the pipelined recurrences of Ghysels and Vanroose (solve_pipelined,
// §10 outlook): one fused vector kernel with a single three-value reduction
// per iteration, and a check of the true residual at the end of each cycle.
#include <cmath>
#include <algorithm>
#include <cstdint>
#include <initializer_list>
#include <type_traits>

#include "sem_internal.cuh"
#include "reduce.cuh"
#include "cg_state.cuh"
#include "df.cuh"

namespace sem {

// ------------------------------------------------------------------ kernels
// Per-thread accumulation of a b / mult before the FP64 block and grid sums:
// FP64 for FP64 vectors; for FP32 vectors an FP32 Kahan-compensated sum
// (the FP64 pipe of GB300 is 60x slower than FP32, and per-point float to
// double conversions would dominate these memory-bound kernels).
template <class T>
struct Acc;
template <>
struct Acc<double> {
  double s = 0.0;
  __device__ __forceinline__ void add(double a, double b, float im) { s += a * b * (double)im; }
  __device__ __forceinline__ double value() const { return s; }
};
template <>
struct Acc<float> {
  float s = 0.0f, c = 0.0f;
  __device__ __forceinline__ void add(float a, float b, float im) {
    const float y = __fsub_rn(__fmul_rn(__fmul_rn(a, b), im), c);
    const float t = __fadd_rn(s, y);
    c = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

// ---- vectorised forms of k_pw / k_update / k_pupd: 16-byte loads (float4 for
// FP32, double2 for FP64), used when nL is a multiple of the lane count and
// the vectors are 16-byte aligned; same per-point arithmetic as the scalar forms.
template <class T>
struct Vec;
template <>
struct Vec<float> {
  using V = float4;
  using M = float4;
  static constexpr int L = 4;
};
template <>
struct Vec<double> {
  using V = double2;
  using M = float2;
  static constexpr int L = 2;
};

template <class T>
__global__ void __launch_bounds__(kRedThreads)
k_pw_v(int64_t nv, const typename Vec<T>::V* __restrict__ p, const typename Vec<T>::V* __restrict__ w,
       const typename Vec<T>::M* __restrict__ imult, CGState* __restrict__ st,
       double* __restrict__ partials) {
  using VT = Vec<T>;
  if (st->done) return;
  Acc<T> a0;
#pragma unroll 4
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nv;
       q += (int64_t)gridDim.x * blockDim.x) {
    const typename VT::V a = p[q], b = w[q];
    const typename VT::M m = imult[q];
    const T* ae = reinterpret_cast<const T*>(&a);
    const T* be = reinterpret_cast<const T*>(&b);
    const float* me = reinterpret_cast<const float*>(&m);
#pragma unroll
    for (int l = 0; l < VT::L; ++l) a0.add(ae[l], be[l], me[l]);
  }
  double v[1] = {a0.value()};
  double tot[1];
  if (grid_sum<1>(v, partials, &st->counter, tot) && threadIdx.x == 0) st_after_pw(st, tot[0]);
}

template <class T>
__global__ void __launch_bounds__(kRedThreads)
k_update_v(int64_t nv, typename Vec<T>::V* __restrict__ x, typename Vec<T>::V* __restrict__ r,
           const typename Vec<T>::V* __restrict__ p, const typename Vec<T>::V* __restrict__ w,
           const typename Vec<T>::V* __restrict__ dinv, const typename Vec<T>::M* __restrict__ imult,
           CGState* __restrict__ st, double* __restrict__ partials) {
  using VT = Vec<T>;
  if (st->done) return;
  const T alpha = (T)st->alpha;
  Acc<T> a0, a1;
#pragma unroll 2
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nv;
       q += (int64_t)gridDim.x * blockDim.x) {
    typename VT::V xq = x[q], rq = r[q];
    const typename VT::V pq = p[q], wq = w[q], dq = dinv[q];
    const typename VT::M mq = imult[q];
    T* xe = reinterpret_cast<T*>(&xq);
    T* re = reinterpret_cast<T*>(&rq);
    const T* pe = reinterpret_cast<const T*>(&pq);
    const T* we = reinterpret_cast<const T*>(&wq);
    const T* de = reinterpret_cast<const T*>(&dq);
    const float* me = reinterpret_cast<const float*>(&mq);
#pragma unroll
    for (int l = 0; l < VT::L; ++l) {
      xe[l] += alpha * pe[l];
      re[l] = re[l] - alpha * we[l];
      const T z = de[l] * re[l];
      a0.add(re[l], z, me[l]);
      a1.add(re[l], re[l], me[l]);
    }
    x[q] = xq;
    r[q] = rq;
  }
  double v[2] = {a0.value(), a1.value()};
  double tot[2];
  if (grid_sum<2>(v, partials, &st->counter, tot) && threadIdx.x == 0) st_after_update(st, tot);
}

template <class T>
__global__ void __launch_bounds__(kRedThreads)
k_pupd_v(int64_t nv, typename Vec<T>::V* __restrict__ p, const typename Vec<T>::V* __restrict__ r,
         const typename Vec<T>::V* __restrict__ dinv, const CGState* __restrict__ st) {
  using VT = Vec<T>;
  if (st->done) return;
  const T beta = (T)st->beta;
#pragma unroll 4
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nv;
       q += (int64_t)gridDim.x * blockDim.x) {
    typename VT::V pq = p[q];
    const typename VT::V rq = r[q], dq = dinv[q];
    T* pe = reinterpret_cast<T*>(&pq);
    const T* re = reinterpret_cast<const T*>(&rq);
    const T* de = reinterpret_cast<const T*>(&dq);
#pragma unroll
    for (int l = 0; l < VT::L; ++l) pe[l] = de[l] * re[l] + beta * pe[l];
    p[q] = pq;
  }
}

// ---- FP32 CG on global (unique-dof) vectors, padded with zeros to a
// multiple of 4 values: plain dots (every point counted once), and the
// update pass also clears w for the next operator's atomic assembly.
__device__ __forceinline__ void rz_rr4(const float4& r, const float4& z, Acc<float>& a0,
                                       Acc<float>& a1) {
  a0.add(r.x, z.x, 1.0f); a0.add(r.y, z.y, 1.0f); a0.add(r.z, z.z, 1.0f); a0.add(r.w, z.w, 1.0f);
  a1.add(r.x, r.x, 1.0f); a1.add(r.y, r.y, 1.0f); a1.add(r.z, r.z, 1.0f); a1.add(r.w, r.w, 1.0f);
}

__global__ void __launch_bounds__(kRedThreads)
k_ginit(int64_t nv, const float4* __restrict__ r, const float4* __restrict__ dinv,
        float4* __restrict__ p, float4* __restrict__ x, float4* __restrict__ w,
        CGState* __restrict__ st, double* __restrict__ partials, double tol, int maxit) {
  Acc<float> a0, a1;
  const float4 zero = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nv;
       q += (int64_t)gridDim.x * blockDim.x) {
    const float4 rq = r[q], dq = dinv[q];
    const float4 z = make_float4(dq.x * rq.x, dq.y * rq.y, dq.z * rq.z, dq.w * rq.w);
    p[q] = z;
    x[q] = zero;
    w[q] = zero;
    rz_rr4(rq, z, a0, a1);
  }
  double v[2] = {a0.value(), a1.value()};
  double tot[2];
  if (grid_sum<2>(v, partials, &st->counter, tot) && threadIdx.x == 0)
    st_after_init(st, tot, tol, maxit, 1);
}

__global__ void __launch_bounds__(kRedThreads)
k_gpw(int64_t nv, const float4* __restrict__ p, const float4* __restrict__ w,
      CGState* __restrict__ st, double* __restrict__ partials) {
  if (st->done) return;
  Acc<float> a0;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nv;
       q += (int64_t)gridDim.x * blockDim.x) {
    const float4 a = p[q], b = w[q];
    a0.add(a.x, b.x, 1.0f); a0.add(a.y, b.y, 1.0f); a0.add(a.z, b.z, 1.0f); a0.add(a.w, b.w, 1.0f);
  }
  double v[1] = {a0.value()};
  double tot[1];
  if (grid_sum<1>(v, partials, &st->counter, tot) && threadIdx.x == 0) st_after_pw(st, tot[0]);
}

__global__ void __launch_bounds__(kRedThreads)
k_gupdate(int64_t nv, float4* __restrict__ x, float4* __restrict__ r, const float4* __restrict__ p,
          float4* __restrict__ w, const float4* __restrict__ dinv, CGState* __restrict__ st,
          double* __restrict__ partials) {
  if (st->done) return;
  const float alpha = (float)st->alpha;
  const float4 zero = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  Acc<float> a0, a1;
#pragma unroll 2
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nv;
       q += (int64_t)gridDim.x * blockDim.x) {
    float4 xq = x[q], rq = r[q];
    const float4 pq = p[q], wq = w[q], dq = dinv[q];
    xq.x += alpha * pq.x; xq.y += alpha * pq.y; xq.z += alpha * pq.z; xq.w += alpha * pq.w;
    rq.x -= alpha * wq.x; rq.y -= alpha * wq.y; rq.z -= alpha * wq.z; rq.w -= alpha * wq.w;
    const float4 z = make_float4(dq.x * rq.x, dq.y * rq.y, dq.z * rq.z, dq.w * rq.w);
    rz_rr4(rq, z, a0, a1);
    x[q] = xq;
    r[q] = rq;
    w[q] = zero;
  }
  double v[2] = {a0.value(), a1.value()};
  double tot[2];
  if (grid_sum<2>(v, partials, &st->counter, tot) && threadIdx.x == 0) st_after_update(st, tot);
}

// grid of the padded-vector CG kernels: a thread per float4 up to kRedBlocks
// blocks (small vectors, such as the Schwarz coarse level, take fewer)
static int vcg_grid(int64_t nv4) {
  return (int)std::max<int64_t>(1, std::min<int64_t>(kRedBlocks, (nv4 + kRedThreads - 1) / kRedThreads));
}

void vcg_init(int64_t nv4, const float* r, const float* dinv, float* p, float* x, float* w,
              CGState* st, double* partials, double tol, int maxit, cudaStream_t s) {
  k_ginit<<<vcg_grid(nv4), kRedThreads, 0, s>>>(nv4, (const float4*)r, (const float4*)dinv,
                                             (float4*)p, (float4*)x, (float4*)w, st, partials,
                                             tol, maxit);
  SEM_CHECK_LAUNCH();
}

void vcg_pw(int64_t nv4, const float* p, const float* w, CGState* st, double* partials,
            cudaStream_t s) {
  k_gpw<<<vcg_grid(nv4), kRedThreads, 0, s>>>(nv4, (const float4*)p, (const float4*)w, st,
                                              partials);
  SEM_CHECK_LAUNCH();
}

void vcg_update(int64_t nv4, float* x, float* r, const float* p, float* w, const float* dinv,
                CGState* st, double* partials, cudaStream_t s) {
  k_gupdate<<<vcg_grid(nv4), kRedThreads, 0, s>>>(nv4, (float4*)x, (float4*)r,
                                                  (const float4*)p, (float4*)w,
                                                  (const float4*)dinv, st, partials);
  SEM_CHECK_LAUNCH();
}

void vcg_pupd(int64_t nv4, float* p, const float* r, const float* dinv, const CGState* st,
              cudaStream_t s) {
  k_pupd_v<float><<<vcg_grid(nv4), kRedThreads, 0, s>>>(nv4, (float4*)p, (const float4*)r,
                                                        (const float4*)dinv, st);
  SEM_CHECK_LAUNCH();
}

// ---- FP64 forms with fewer FP64-pipe operations (that pipe, not HBM, bounds
// the FP64 vector kernels on GB300).  1/mult is a power of two (mult = 1, 2,
// 4 or 8 copies on the box), so it is widened to double by moving its
// exponent bits instead of a conversion instruction; <r, z> uses the
// precomputed dinv / mult:  <p, w>: 2 FP64 operations per point,
// update: x, r, r^2, <r,z>, <r,r>: 5.
__device__ __forceinline__ double pow2_widen(float f) {
  return __longlong_as_double((long long)((__float_as_uint(f) >> 23) + 896u) << 52);
}

__global__ void __launch_bounds__(kRedThreads)
k_pw_v64(int64_t nv, const double2* __restrict__ p, const double2* __restrict__ w,
         const float2* __restrict__ imult, CGState* __restrict__ st,
         double* __restrict__ partials) {
  if (st->done) return;
  double acc = 0.0;
#pragma unroll 4
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nv;
       q += (int64_t)gridDim.x * blockDim.x) {
    const double2 a = p[q], b = w[q];
    const float2 m = imult[q];
    acc = fma(a.x * b.x, pow2_widen(m.x), acc);
    acc = fma(a.y * b.y, pow2_widen(m.y), acc);
  }
  double v[1] = {acc};
  double tot[1];
  if (grid_sum<1>(v, partials, &st->counter, tot) && threadIdx.x == 0) st_after_pw(st, tot[0]);
}

__global__ void __launch_bounds__(kRedThreads)
k_update_v64(int64_t nv, double2* __restrict__ x, double2* __restrict__ r,
             const double2* __restrict__ p, const double2* __restrict__ w,
             const double2* __restrict__ dmi, const float2* __restrict__ imult,
             CGState* __restrict__ st, double* __restrict__ partials) {
  if (st->done) return;
  const double alpha = st->alpha;
  double rz = 0.0, rr = 0.0;
#pragma unroll 2
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nv;
       q += (int64_t)gridDim.x * blockDim.x) {
    double2 xq = x[q], rq = r[q];
    const double2 pq = p[q], wq = w[q], dq = dmi[q];
    const float2 mq = imult[q];
    xq.x = fma(alpha, pq.x, xq.x);
    xq.y = fma(alpha, pq.y, xq.y);
    rq.x = fma(-alpha, wq.x, rq.x);
    rq.y = fma(-alpha, wq.y, rq.y);
    const double sx = rq.x * rq.x, sy = rq.y * rq.y;
    rz = fma(sx, dq.x, rz);
    rz = fma(sy, dq.y, rz);
    rr = fma(sx, pow2_widen(mq.x), rr);
    rr = fma(sy, pow2_widen(mq.y), rr);
    x[q] = xq;
    r[q] = rq;
  }
  double v[2] = {rz, rr};
  double tot[2];
  if (grid_sum<2>(v, partials, &st->counter, tot) && threadIdx.x == 0) st_after_update(st, tot);
}

template <class T>
__global__ void __launch_bounds__(kRedThreads)
k_init(int64_t n, const T* __restrict__ r, const T* __restrict__ dinv,
       const float* __restrict__ imult, T* __restrict__ p, T* __restrict__ xzero,
       CGState* __restrict__ st, double* __restrict__ partials, double tol, int maxit,
       int bb_from_rr) {
  Acc<T> a0, a1;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
       q += (int64_t)gridDim.x * blockDim.x) {
    T rq = r[q];
    T z = dinv[q] * rq;
    p[q] = z;
    if (xzero) xzero[q] = T(0);
    const float im = imult[q];
    a0.add(rq, z, im);
    a1.add(rq, rq, im);
  }
  double v[2] = {a0.value(), a1.value()};
  double tot[2];
  if (grid_sum<2>(v, partials, &st->counter, tot) && threadIdx.x == 0)
    st_after_init(st, tot, tol, maxit, bb_from_rr);
}

template <class T>
__global__ void __launch_bounds__(kRedThreads)
k_pw(int64_t n, const T* __restrict__ p, const T* __restrict__ w, const float* __restrict__ imult,
     CGState* __restrict__ st, double* __restrict__ partials) {
  if (st->done) return;
  Acc<T> a0;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
       q += (int64_t)gridDim.x * blockDim.x)
    a0.add(p[q], w[q], imult[q]);
  double v[1] = {a0.value()};
  double tot[1];
  if (grid_sum<1>(v, partials, &st->counter, tot) && threadIdx.x == 0) st_after_pw(st, tot[0]);
}

template <class T>
__global__ void __launch_bounds__(kRedThreads)
k_update(int64_t n, T* __restrict__ x, T* __restrict__ r, const T* __restrict__ p,
         const T* __restrict__ w, const T* __restrict__ dinv, const float* __restrict__ imult,
         CGState* __restrict__ st, double* __restrict__ partials) {
  if (st->done) return;
  const T alpha = (T)st->alpha;
  Acc<T> a0, a1;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
       q += (int64_t)gridDim.x * blockDim.x) {
    x[q] += alpha * p[q];
    T rq = r[q] - alpha * w[q];
    r[q] = rq;
    T z = dinv[q] * rq;
    const float im = imult[q];
    a0.add(rq, z, im);
    a1.add(rq, rq, im);
  }
  double v[2] = {a0.value(), a1.value()};
  double tot[2];
  if (grid_sum<2>(v, partials, &st->counter, tot) && threadIdx.x == 0) st_after_update(st, tot);
}

template <class T>
__global__ void __launch_bounds__(kRedThreads)
k_pupd(int64_t n, T* __restrict__ p, const T* __restrict__ r, const T* __restrict__ dinv,
       const CGState* __restrict__ st) {
  if (st->done) return;
  const T beta = (T)st->beta;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
       q += (int64_t)gridDim.x * blockDim.x)
    p[q] = dinv[q] * r[q] + beta * p[q];
}

// r64 = b - w64 (FP64 residual), optional FP32 copy of rscale r64, <r,r> into st->rr
__global__ void __launch_bounds__(kRedThreads)
k_resid(int64_t n, const double* __restrict__ b, const double* __restrict__ w,
        double* __restrict__ r, float* __restrict__ r32, const float* __restrict__ imult,
        CGState* __restrict__ st, double* __restrict__ partials, double rscale) {
  double v[1] = {0.0};
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
       q += (int64_t)gridDim.x * blockDim.x) {
    double rq = b[q] - w[q];
    r[q] = rq;
    if (r32) r32[q] = (float)(rq * rscale);
    v[0] += rq * rq * (double)imult[q];
  }
  double tot[1];
  if (grid_sum<1>(v, partials, &st->counter, tot) && threadIdx.x == 0) st->rr = tot[0];
}

// <a, a> into st->bb
__global__ void __launch_bounds__(kRedThreads)
k_norm_bb(int64_t n, const double* __restrict__ a, const float* __restrict__ imult,
          CGState* __restrict__ st, double* __restrict__ partials) {
  double v[1] = {0.0};
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
       q += (int64_t)gridDim.x * blockDim.x)
    v[0] += a[q] * a[q] * (double)imult[q];
  double tot[1];
  if (grid_sum<1>(v, partials, &st->counter, tot) && threadIdx.x == 0) st->bb = tot[0];
}

// sum a b / mult into *out (fixed grid, fixed order)
__global__ void __launch_bounds__(kRedThreads)
k_wdot(int64_t n, const double* __restrict__ a, const double* __restrict__ b,
       const float* __restrict__ imult, double* __restrict__ out, double* __restrict__ partials,
       unsigned int* __restrict__ counter) {
  double v[1] = {0.0};
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
       q += (int64_t)gridDim.x * blockDim.x)
    v[0] += a[q] * b[q] * (double)imult[q];
  double tot[1];
  if (grid_sum<1>(v, partials, counter, tot) && threadIdx.x == 0) *out = tot[0];
}

// x += d scale (the FP32 correction of a refinement step, scale = 1 / rscale)
__global__ void k_addx(int64_t n, double* __restrict__ x, const float* __restrict__ d,
                       double scale) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
       q += (int64_t)gridDim.x * blockDim.x)
    x[q] += (double)d[q] * scale;
}

__global__ void k_dinv(int64_t n, const double* __restrict__ dg, const uint8_t* __restrict__ mask,
                       const float* __restrict__ imult, double* __restrict__ dinv,
                       double* __restrict__ dmi, float* __restrict__ dinv32) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
       q += (int64_t)gridDim.x * blockDim.x) {
    double v = mask[q] ? 1.0 / dg[q] : 0.0;
    dinv[q] = v;
    dmi[q] = v * (double)imult[q];
    if (dinv32) dinv32[q] = (float)v;
  }
}

__global__ void k_mul(int64_t n, const double* __restrict__ a, const double* __restrict__ b,
                      double* __restrict__ c) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
       q += (int64_t)gridDim.x * blockDim.x)
    c[q] = a[q] * b[q];
}

__global__ void k_d2f(int64_t n, const double* __restrict__ a, float* __restrict__ b) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
       q += (int64_t)gridDim.x * blockDim.x)
    b[q] = (float)a[q];
}

// ---- pipelined PCG (Ghysels and Vanroose): one reduction per iteration, all
// vectors updated by recurrences in one pass after the operator.
// Start of a cycle (r holds the residual): u = dinv r, z = q = s = p = 0.
__global__ void k_pipe_start(int64_t n, const double* __restrict__ r, const double* __restrict__ dinv,
                             double* __restrict__ u, double* __restrict__ z, double* __restrict__ q,
                             double* __restrict__ s, double* __restrict__ p) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    u[i] = dinv[i] * r[i];
    z[i] = 0.0;
    q[i] = 0.0;
    s[i] = 0.0;
    p[i] = 0.0;
  }
}

// After w = H u: m = dinv w; gamma = <r, u>, delta = <w, u>, <r, r>;
// alpha = gamma / delta, beta = 0.
__global__ void __launch_bounds__(kRedThreads)
k_pipe_first(int64_t n, const double* __restrict__ r, const double* __restrict__ u,
             const double* __restrict__ w, const double* __restrict__ dinv,
             const float* __restrict__ imult, double* __restrict__ m, CGState* __restrict__ st,
             double* __restrict__ partials, double tol, int maxit, int iter0) {
  double v[3] = {0.0, 0.0, 0.0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double ri = r[i], ui = u[i], wi = w[i], im = (double)imult[i];
    m[i] = dinv[i] * wi;
    v[0] = fma(ri * ui, im, v[0]);
    v[1] = fma(wi * ui, im, v[1]);
    v[2] = fma(ri * ri, im, v[2]);
  }
  double tot[3];
  if (grid_sum<3>(v, partials, &st->counter, tot) && threadIdx.x == 0) {
    st->rz = tot[0];
    st->pw = tot[1];
    st->rr = tot[2];
    st->tol2 = tol * tol * st->bb;
    st->iter = iter0;
    st->maxit = maxit;
    st->status = SEM_OK;
    st->beta = 0.0;
    st->done = 0;
    if (!(tot[2] == tot[2])) {
      st->status = SEM_ERR_BREAKDOWN;
      st->done = 1;
    } else if (tot[2] <= st->tol2 || st->bb == 0.0) {
      st->done = 1;
    } else if (iter0 >= maxit) {
      st->status = SEM_ERR_NOCONV;
      st->done = 1;
    } else if (!(tot[1] > 0.0)) {
      st->status = SEM_ERR_BREAKDOWN;
      st->done = 1;
    } else {
      st->alpha = tot[0] / tot[1];
    }
  }
}

// One iteration after nv = H m (alpha, beta from the state); then the dots of
// the new vectors and alpha, beta of the next iteration.
__global__ void __launch_bounds__(kRedThreads)
k_pipe_update(int64_t n, double* __restrict__ x, double* __restrict__ r, double* __restrict__ u,
              double* __restrict__ w, double* __restrict__ z, double* __restrict__ q,
              double* __restrict__ s, double* __restrict__ p, double* __restrict__ m,
              const double* __restrict__ nv, const double* __restrict__ dinv,
              const float* __restrict__ imult, CGState* __restrict__ st,
              double* __restrict__ partials) {
  if (st->done) return;
  const double alpha = st->alpha, beta = st->beta;
  double v[3] = {0.0, 0.0, 0.0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double zi = fma(beta, z[i], nv[i]);
    const double qi = fma(beta, q[i], m[i]);
    const double wi0 = w[i], ui0 = u[i];
    const double si = fma(beta, s[i], wi0);
    const double pi = fma(beta, p[i], ui0);
    z[i] = zi;
    q[i] = qi;
    s[i] = si;
    p[i] = pi;
    x[i] = fma(alpha, pi, x[i]);
    const double ri = fma(-alpha, si, r[i]);
    const double ui = fma(-alpha, qi, ui0);
    const double wi = fma(-alpha, zi, wi0);
    r[i] = ri;
    u[i] = ui;
    w[i] = wi;
    m[i] = dinv[i] * wi;
    const double im = (double)imult[i];
    v[0] = fma(ri * ui, im, v[0]);
    v[1] = fma(wi * ui, im, v[1]);
    v[2] = fma(ri * ri, im, v[2]);
  }
  double tot[3];
  if (grid_sum<3>(v, partials, &st->counter, tot) && threadIdx.x == 0) {
    st->iter += 1;
    st->rr = tot[2];
    if (!(tot[0] == tot[0]) || !(tot[1] == tot[1]) || !(tot[2] == tot[2])) {
      st->status = SEM_ERR_BREAKDOWN;
      st->done = 1;
    } else if (tot[2] <= st->tol2) {
      st->done = 1;
    } else if (st->iter >= st->maxit) {
      st->status = SEM_ERR_NOCONV;
      st->done = 1;
    } else {
      const double b2 = tot[0] / st->rz;
      const double den = tot[1] - b2 * tot[0] / st->alpha;
      if (!(den > 0.0)) {
        st->status = SEM_ERR_BREAKDOWN;
        st->done = 1;
      } else {
        st->beta = b2;
        st->alpha = tot[0] / den;
        st->rz = tot[0];
        st->pw = tot[1];
      }
    }
  }
}

static int ew_grid(int64_t n) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 8 * sem_num_sms()));
}

// ------------------------------------------------------------------ host drivers
struct Pinned {
  CGState* p = nullptr;
  Pinned() { SEM_CUDA(cudaMallocHost(&p, 2 * sizeof(CGState))); }
  ~Pinned() { if (p) cudaFreeHost(p); }
};

// Copies the solver state to the host; raises SEM_ERR_TIMEOUT if a bounded
// device wait gave up since the last check.
static CGState read_state(const CGState* d, cudaStream_t s, int* dev_err = nullptr) {
  static thread_local Pinned pin;
  SEM_CUDA(cudaMemcpyAsync(pin.p, d, sizeof(CGState), cudaMemcpyDeviceToHost, s));
  if (dev_err)
    SEM_CUDA(cudaMemcpyAsync(&pin.p[1].status, dev_err, sizeof(int), cudaMemcpyDeviceToHost, s));
  SEM_CUDA(cudaStreamSynchronize(s));
  if (dev_err && pin.p[1].status) {
    SEM_CUDA(cudaMemsetAsync(dev_err, 0, sizeof(int), s));
    SEM_CUDA(cudaStreamSynchronize(s));
    pin.p[1].status = 0;
    throw Error(SEM_ERR_TIMEOUT, "a bounded device wait timed out during the solve");
  }
  return *pin.p;
}

template <class T>
struct PcgArgs {
  const OpData<T>* op;
  T* x;
  T* r;
  T* p;
  T* w;
  const T* dinv;
  const T* h1f;
  T h1, h2;
  CGState* st;
  const T* dmi = nullptr;     // dinv / mult (FP64 solves)
};

// true when the vectorised kernels apply: n a multiple of the lane count and
// every vector (and the multiplicity array) 16-byte (FP32 imult: 8-byte) aligned
template <class T>
static bool vec_ok(int64_t n, std::initializer_list<const T*> ptrs, const float* imult) {
  if (n % Vec<T>::L) return false;
  for (const T* q : ptrs)
    if (reinterpret_cast<uintptr_t>(q) % 16) return false;
  return reinterpret_cast<uintptr_t>(imult) % (Vec<T>::L * sizeof(float)) == 0;
}

// FP64 pw / update / p-update with the reduced-FP64-operation kernels
static void launch_vec64(sem_handle* h, const PcgArgs<double>& a, bool pw_done, cudaStream_t s) {
  const int64_t nv = h->nL / 2;
  if (!pw_done) {
    k_pw_v64<<<kRedBlocks, kRedThreads, 0, s>>>(nv, (const double2*)a.p, (const double2*)a.w,
                                                (const float2*)h->imult.ptr, a.st,
                                                h->partials.ptr);
    SEM_CHECK_LAUNCH();
  }
  k_update_v64<<<kRedBlocks, kRedThreads, 0, s>>>(
      nv, (double2*)a.x, (double2*)a.r, (const double2*)a.p, (const double2*)a.w,
      (const double2*)a.dmi, (const float2*)h->imult.ptr, a.st, h->partials.ptr);
  SEM_CHECK_LAUNCH();
  k_pupd_v<double><<<kRedBlocks, kRedThreads, 0, s>>>(nv, (double2*)a.p, (const double2*)a.r,
                                                      (const double2*)a.dinv, a.st);
  SEM_CHECK_LAUNCH();
}

template <class T>
static void pcg_iterations(sem_handle* h, const PcgArgs<T>& a, int count, cudaStream_t s) {
  const int64_t n = h->nL;
  const bool vec = vec_ok<T>(n, {a.x, a.r, a.p, a.w, a.dinv, a.dmi}, h->imult.ptr);
  for (int c = 0; c < count; ++c) {
    // the element kernel may take <p, w> and alpha itself (FP32, P = 8)
    const bool pw_done =
        launch_apply<T>(h, *a.op, a.p, a.w, a.h1, a.h2, a.h1f, a.st, SEM_APPLY_FULL, s, a.st);
    bool done64 = false;
    if constexpr (std::is_same<T, double>::value) {
      if (vec && a.dmi) {
        launch_vec64(h, a, pw_done, s);
        done64 = true;
      }
    }
    if (done64) continue;
    if (vec) {
      using V = typename Vec<T>::V;
      using M = typename Vec<T>::M;
      const int64_t nv = n / Vec<T>::L;
      if (!pw_done) {
        k_pw_v<T><<<kRedBlocks, kRedThreads, 0, s>>>(nv, (const V*)a.p, (const V*)a.w,
                                                     (const M*)h->imult.ptr, a.st,
                                                     h->partials.ptr);
        SEM_CHECK_LAUNCH();
      }
      k_update_v<T><<<kRedBlocks, kRedThreads, 0, s>>>(nv, (V*)a.x, (V*)a.r, (const V*)a.p,
                                                       (const V*)a.w, (const V*)a.dinv,
                                                       (const M*)h->imult.ptr, a.st,
                                                       h->partials.ptr);
      SEM_CHECK_LAUNCH();
      k_pupd_v<T><<<kRedBlocks, kRedThreads, 0, s>>>(nv, (V*)a.p, (const V*)a.r,
                                                     (const V*)a.dinv, a.st);
      SEM_CHECK_LAUNCH();
    } else {
      if (!pw_done) {
        k_pw<T><<<kRedBlocks, kRedThreads, 0, s>>>(n, a.p, a.w, h->imult.ptr, a.st,
                                                   h->partials.ptr);
        SEM_CHECK_LAUNCH();
      }
      k_update<T><<<kRedBlocks, kRedThreads, 0, s>>>(n, a.x, a.r, a.p, a.w, a.dinv, h->imult.ptr,
                                                     a.st, h->partials.ptr);
      SEM_CHECK_LAUNCH();
      k_pupd<T><<<kRedBlocks, kRedThreads, 0, s>>>(n, a.p, a.r, a.dinv, a.st);
      SEM_CHECK_LAUNCH();
    }
  }
}

// FP32 PCG iterations on the global vectors of the handle
static void glob_iterations(sem_handle* h, CGState* st, float h1, float h2, int count,
                            cudaStream_t s) {
  const int64_t nv4 = glob_padded(h) / 4;
  for (int c = 0; c < count; ++c) {
    const bool pw_done = launch_apply_global(h, h->pg.ptr, h->wg.ptr, h1, h2, st, st, s);
    if (!pw_done) vcg_pw(nv4, h->pg.ptr, h->wg.ptr, st, h->partials.ptr, s);
    vcg_update(nv4, h->xg.ptr, h->rg.ptr, h->pg.ptr, h->wg.ptr, h->dinvg.ptr, st,
               h->partials.ptr, s);
    vcg_pupd(nv4, h->pg.ptr, h->rg.ptr, h->dinvg.ptr, st, s);
  }
}

// Runs iterations(count) until the device state st says done (check_every
// iterations per host check, captured once in a CUDA graph when use_graph);
// returns the final state.
template <class F>
static CGState run_pcg_loop(sem_handle* h, CGState* st, const sem_solve_opts& o, cudaStream_t s,
                            F iterations) {
  CGState hs = read_state(st, s);
  if (hs.done) return hs;
  const int batch = std::max(1, o.check_every);
  cudaGraphExec_t exec = nullptr;
  if (o.use_graph) {
    cudaGraph_t graph = nullptr;
    SEM_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    try {
      iterations(batch);
    } catch (...) {
      cudaStreamEndCapture(s, &graph);
      if (graph) cudaGraphDestroy(graph);
      throw;
    }
    SEM_CUDA(cudaStreamEndCapture(s, &graph));
    cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) throw Error(SEM_ERR_CUDA, std::string("cudaGraphInstantiate: ") +
                                                        cudaGetErrorString(e));
  }
  try {
    while (true) {
      if (exec) SEM_CUDA(cudaGraphLaunch(exec, s));
      else iterations(batch);
      hs = read_state(st, s, h->dev_err.ptr);
      if (hs.done) break;
    }
  } catch (...) {
    if (exec) cudaGraphExecDestroy(exec);
    throw;
  }
  if (exec) cudaGraphExecDestroy(exec);
  return hs;
}

template <class T>
static CGState run_pcg(sem_handle* h, const PcgArgs<T>& a, const sem_solve_opts& o,
                       cudaStream_t s) {
  return run_pcg_loop(h, a.st, o, s, [&](int count) { pcg_iterations<T>(h, a, count, s); });
}

static void ensure(DevBuf<double>& b, int64_t n) { if (b.n < (size_t)n) b.alloc(n); }
static void ensure(DevBuf<float>& b, int64_t n) { if (b.n < (size_t)n) b.alloc(n); }

// Jacobi inverse diagonal for (h1 | h1_field, h2): mask / QQ^T diag(H_L)
static void ensure_dinv(sem_handle* h, double h1, double h2, const double* h1f, bool need32,
                        cudaStream_t s) {
  const int64_t n = h->nL;
  bool same = h->dinv_valid && h->dinv_h1 == h1 && h->dinv_h2 == h2 && h->dinv_h1f == h1f &&
              (!need32 || h->f32.dinv.ptr);
  if (same && !h1f) return;      // a field may have changed in place: recompute
  ensure(h->f64.dinv, n);
  ensure(h->f64.dmi, n);
  if (need32) ensure(h->f32.dinv, n);
  ensure(h->tmp64, n);
  launch_local_diag<double>(h, h->f64, h->tmp64.ptr, h1, h2, h1f, s);
  launch_dssum<double>(h, h->tmp64.ptr, false, nullptr, s);
  k_dinv<<<ew_grid(n), 256, 0, s>>>(n, h->tmp64.ptr, h->mask.ptr, h->imult.ptr,
                                   h->f64.dinv.ptr, h->f64.dmi.ptr,
                                   need32 ? h->f32.dinv.ptr : nullptr);
  SEM_CHECK_LAUNCH();
  h->dinv_h1 = h1;
  h->dinv_h2 = h2;
  h->dinv_h1f = h1f;
  h->dinv_valid = 1;
}

// H x -> w (FP64, masked, assembled), then r = b - w and <r,r> into st->rr
static void residual64(sem_handle* h, const double* b, const double* x, double h1, double h2,
                       const double* h1f, float* r32, CGState* st, cudaStream_t s) {
  const int64_t n = h->nL;
  launch_apply<double>(h, h->f64, x, h->w.ptr, h1, h2, h1f, nullptr, SEM_APPLY_FULL, s);
  k_resid<<<kRedBlocks, kRedThreads, 0, s>>>(n, b, h->w.ptr, h->r.ptr, r32, h->imult.ptr, st,
                                             h->partials.ptr, h->rscale);
  SEM_CHECK_LAUNCH();
}

static void solve_fp64(sem_handle* h, const double* b, double* x, const sem_solve_opts& o,
                       sem_solve_info& info, cudaStream_t s) {
  const int64_t n = h->nL;
  ensure(h->r, n); ensure(h->p, n); ensure(h->w, n);
  ensure_dinv(h, o.h1, o.h2, o.h1_field, false, s);
  CGState* st = h->state.ptr;
  k_norm_bb<<<kRedBlocks, kRedThreads, 0, s>>>(n, b, h->imult.ptr, st, h->partials.ptr);
  SEM_CHECK_LAUNCH();
  double* xz = nullptr;
  if (o.x0_is_zero) {
    SEM_CUDA(cudaMemcpyAsync(h->r.ptr, b, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    xz = x;
  } else {
    residual64(h, b, x, o.h1, o.h2, o.h1_field, nullptr, st, s);
  }
  k_init<double><<<kRedBlocks, kRedThreads, 0, s>>>(n, h->r.ptr, h->f64.dinv.ptr, h->imult.ptr,
                                                    h->p.ptr, xz, st, h->partials.ptr, o.tol,
                                                    o.maxit, 0);
  SEM_CHECK_LAUNCH();
  PcgArgs<double> a{&h->f64, x, h->r.ptr, h->p.ptr, h->w.ptr, h->f64.dinv.ptr, o.h1_field,
                    o.h1, o.h2, st, h->f64.dmi.ptr};
  CGState fin = run_pcg<double>(h, a, o, s);
  // true residual of the returned x
  residual64(h, b, x, o.h1, o.h2, o.h1_field, nullptr, st, s);
  CGState chk = read_state(st, s);
  info.iters = fin.iter;
  info.outer_iters = 0;
  info.rel_res = chk.bb > 0 ? std::sqrt(chk.rr / chk.bb) : 0.0;
  info.status = fin.status;
}

// Pipelined PCG in FP64 (SEM_CG_PIPELINED): cycles of recurrences checked
// against the true residual when the recurrence residual converges.
static void solve_pipelined(sem_handle* h, const double* b, double* x, const sem_solve_opts& o,
                            sem_solve_info& info, cudaStream_t s) {
  const int64_t n = h->nL;
  ensure(h->r, n); ensure(h->p, n); ensure(h->w, n);
  for (DevBuf<double>* v : {&h->pipe_u, &h->pipe_z, &h->pipe_q, &h->pipe_s, &h->pipe_m,
                            &h->pipe_n})
    ensure(*v, n);
  ensure_dinv(h, o.h1, o.h2, o.h1_field, false, s);
  CGState* st = h->state.ptr;
  k_norm_bb<<<kRedBlocks, kRedThreads, 0, s>>>(n, b, h->imult.ptr, st, h->partials.ptr);
  SEM_CHECK_LAUNCH();
  if (o.x0_is_zero) SEM_CUDA(cudaMemsetAsync(x, 0, n * sizeof(double), s));
  const double* dinv = h->f64.dinv.ptr;
  int iters = 0, cycles = 0, status = SEM_ERR_NOCONV;
  double rel = 0.0;
  constexpr int kMaxCycles = 6;
  for (;;) {
    residual64(h, b, x, o.h1, o.h2, o.h1_field, nullptr, st, s);   // r = b - H x
    const CGState hs = read_state(st, s, h->dev_err.ptr);
    rel = hs.bb > 0 ? std::sqrt(hs.rr / hs.bb) : 0.0;
    if (!(rel == rel)) { status = SEM_ERR_BREAKDOWN; break; }
    if (rel <= o.tol) { status = SEM_OK; break; }
    if (iters >= o.maxit || cycles >= kMaxCycles) { status = SEM_ERR_NOCONV; break; }
    ++cycles;
    k_pipe_start<<<ew_grid(n), 256, 0, s>>>(n, h->r.ptr, dinv, h->pipe_u.ptr, h->pipe_z.ptr,
                                           h->pipe_q.ptr, h->pipe_s.ptr, h->p.ptr);
    SEM_CHECK_LAUNCH();
    launch_apply<double>(h, h->f64, h->pipe_u.ptr, h->w.ptr, o.h1, o.h2, o.h1_field, nullptr,
                         SEM_APPLY_FULL, s);
    k_pipe_first<<<kRedBlocks, kRedThreads, 0, s>>>(n, h->r.ptr, h->pipe_u.ptr, h->w.ptr, dinv,
                                                   h->imult.ptr, h->pipe_m.ptr, st,
                                                   h->partials.ptr, o.tol, o.maxit, iters);
    SEM_CHECK_LAUNCH();
    const CGState fin = run_pcg_loop(h, st, o, s, [&](int count) {
      for (int c = 0; c < count; ++c) {
        launch_apply<double>(h, h->f64, h->pipe_m.ptr, h->pipe_n.ptr, o.h1, o.h2, o.h1_field, st,
                             SEM_APPLY_FULL, s);
        k_pipe_update<<<kRedBlocks, kRedThreads, 0, s>>>(
            n, x, h->r.ptr, h->pipe_u.ptr, h->w.ptr, h->pipe_z.ptr, h->pipe_q.ptr,
            h->pipe_s.ptr, h->p.ptr, h->pipe_m.ptr, h->pipe_n.ptr, dinv, h->imult.ptr, st,
            h->partials.ptr);
        SEM_CHECK_LAUNCH();
      }
    });
    iters = fin.iter;
    if (fin.status == SEM_ERR_BREAKDOWN) { status = SEM_ERR_BREAKDOWN; break; }
  }
  info.iters = iters;
  info.outer_iters = cycles;
  info.rel_res = rel;
  info.status = status;
}

// Relative tolerance of the next inner FP32 solve when the outer relative
// residual is rel: inner_tol (the reduction FP32 can be trusted with), or,
// once less is needed, the reduction that reaches the outer tolerance with a
// factor kInnerMargin to spare, so that the last refinement step does only
// the iterations it needs.
double inner_target(double inner_tol, double tol, double rel) {
  constexpr double kInnerMargin = 0.5;
  const double need = rel > 0.0 ? kInnerMargin * tol / rel : inner_tol;
  return std::max(inner_tol, std::min(0.5, need));
}

// global inner vectors (allocated zeroed, so that the padding stays zero) and
// the Jacobi diagonal in global form
void glob_prepare(sem_handle* h, cudaStream_t s) {
  const int64_t n = glob_padded(h);
  for (DevBuf<float>* b : {&h->rg, &h->pg, &h->wg, &h->xg, &h->dinvg}) {
    if (b->n < (size_t)n) {
      b->alloc(n);
      SEM_CUDA(cudaMemsetAsync(b->ptr, 0, n * sizeof(float), s));
    }
  }
  to_global<float>(h, h->f32.dinv.ptr, h->dinvg.ptr, s);
}

static void solve_mixed(sem_handle* h, const double* b, double* x, const sem_solve_opts& o,
                        sem_solve_info& info, cudaStream_t s) {
  const int64_t n = h->nL;
  if (!h->f32.G.ptr) throw Error(SEM_ERR_STATE, "mixed solve needs FP32 geometry (SEM_PREC_F32)");
  const bool glob = h->inner_vectors != SEM_INNER_LOCAL && !o.h1_field && glob_supported(h);
  ensure(h->r, n); ensure(h->w, n);
  if (!glob) {
    ensure(h->r32, n); ensure(h->p32, n); ensure(h->w32, n); ensure(h->x32, n);
  }
  ensure_dinv(h, o.h1, o.h2, o.h1_field, true, s);
  if (glob) glob_prepare(h, s);
  const float* h1f32 = nullptr;
  if (o.h1_field) {
    ensure(h->f32.h1f, n);
    k_d2f<<<ew_grid(n), 256, 0, s>>>(n, o.h1_field, h->f32.h1f.ptr);
    SEM_CHECK_LAUNCH();
    h1f32 = h->f32.h1f.ptr;
  }
  CGState* st0 = h->state.ptr;
  CGState* st1 = h->state.ptr + 1;
  k_norm_bb<<<kRedBlocks, kRedThreads, 0, s>>>(n, b, h->imult.ptr, st0, h->partials.ptr);
  SEM_CHECK_LAUNCH();
  inner_scale_from_b(h, s);
  if (o.x0_is_zero) SEM_CUDA(cudaMemsetAsync(x, 0, n * sizeof(double), s));
  int total = 0, outer = 0;
  int status = SEM_ERR_NOCONV;
  double rel = 0.0;
  for (;;) {
    residual64(h, b, x, o.h1, o.h2, o.h1_field, glob ? nullptr : h->r32.ptr, st0, s);
    CGState hs = read_state(st0, s);
    rel = hs.bb > 0 ? std::sqrt(hs.rr / hs.bb) : 0.0;
    if (!(rel == rel)) { status = SEM_ERR_BREAKDOWN; break; }
    if (rel <= o.tol) { status = SEM_OK; break; }
    if (outer >= o.max_outer || total >= o.maxit) { status = SEM_ERR_NOCONV; break; }
    // inner FP32 PCG on H d = r, d = 0 initially
    const double itol = inner_target(o.inner_tol, o.tol, rel);
    CGState in;
    if (glob) {
      to_global<double>(h, h->r.ptr, h->rg.ptr, s, h->rscale);
      vcg_init(glob_padded(h) / 4, h->rg.ptr, h->dinvg.ptr, h->pg.ptr, h->xg.ptr, h->wg.ptr,
               st1, h->partials.ptr, itol, o.maxit - total, s);
      in = run_pcg_loop(h, st1, o, s, [&](int count) {
        glob_iterations(h, st1, (float)o.h1, (float)o.h2, count, s);
      });
    } else {
      k_init<float><<<kRedBlocks, kRedThreads, 0, s>>>(n, h->r32.ptr, h->f32.dinv.ptr,
                                                       h->imult.ptr, h->p32.ptr, h->x32.ptr, st1,
                                                       h->partials.ptr, itol, o.maxit - total, 1);
      SEM_CHECK_LAUNCH();
      PcgArgs<float> a{&h->f32, h->x32.ptr, h->r32.ptr, h->p32.ptr, h->w32.ptr,
                       h->f32.dinv.ptr, h1f32, (float)o.h1, (float)o.h2, st1};
      in = run_pcg<float>(h, a, o, s);
    }
    total += in.iter;
    ++outer;
    if (in.status == SEM_ERR_BREAKDOWN && in.iter == 0) { status = SEM_ERR_BREAKDOWN; break; }
    if (glob) {
      add_from_global(h, x, h->xg.ptr, s, 1.0 / h->rscale);
    } else {
      k_addx<<<ew_grid(n), 256, 0, s>>>(n, x, h->x32.ptr, 1.0 / h->rscale);
      SEM_CHECK_LAUNCH();
    }
  }
  info.iters = total;
  info.outer_iters = outer;
  info.rel_res = rel;
  info.status = status;
}

// Runs fn on the handle's private stream, ordered after the caller's stream.
struct StreamScope {
  cudaStream_t user, own;
  cudaEvent_t ev;
  StreamScope(cudaStream_t u) : user(u) {
    SEM_CUDA(cudaStreamCreateWithFlags(&own, cudaStreamNonBlocking));
    SEM_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    SEM_CUDA(cudaEventRecord(ev, user));
    SEM_CUDA(cudaStreamWaitEvent(own, ev, 0));
  }
  ~StreamScope() {
    cudaEventRecord(ev, own);
    cudaStreamWaitEvent(user, ev, 0);
    cudaStreamSynchronize(own);
    cudaEventDestroy(ev);
    cudaStreamDestroy(own);
  }
};

// ---- pieces of the mixed-precision solve shared with the batched solver
void mixed_prepare(sem_handle* h, const sem_solve_opts& o, cudaStream_t s) {
  const int64_t n = h->nL;
  if (!h->f32.G.ptr) throw Error(SEM_ERR_STATE, "mixed solve needs FP32 geometry (SEM_PREC_F32)");
  ensure(h->r, n); ensure(h->w, n);
  ensure(h->r32, n); ensure(h->p32, n); ensure(h->w32, n); ensure(h->x32, n);
  ensure_dinv(h, o.h1, o.h2, o.h1_field, true, s);
}

void outer_norm_b(sem_handle* h, const double* b, cudaStream_t s) {
  k_norm_bb<<<kRedBlocks, kRedThreads, 0, s>>>(h->nL, b, h->imult.ptr, h->state.ptr,
                                               h->partials.ptr);
  SEM_CHECK_LAUNCH();
}

void outer_residual(sem_handle* h, const double* b, const double* x, const sem_solve_opts& o,
                    cudaStream_t s) {
  residual64(h, b, x, o.h1, o.h2, o.h1_field, h->r32.ptr, h->state.ptr, s);
}

void outer_residual_global(sem_handle* h, const double* b, const double* x,
                           const sem_solve_opts& o, cudaStream_t s) {
  residual64(h, b, x, o.h1, o.h2, o.h1_field, nullptr, h->state.ptr, s);
  to_global<double>(h, h->r.ptr, h->rg.ptr, s, h->rscale);
}

void inner_scale_from_b(sem_handle* h, cudaStream_t s) {
  const CGState hs = read_state(h->state.ptr, s);
  const double rms = std::sqrt(hs.bb / (double)std::max<int64_t>(1, h->nG));
  h->rscale = std::ldexp(1.0, -df_pick_exp(rms));
}

void outer_update(sem_handle* h, double* x, cudaStream_t s) {
  k_addx<<<ew_grid(h->nL), 256, 0, s>>>(h->nL, x, h->x32.ptr, 1.0 / h->rscale);
  SEM_CHECK_LAUNCH();
}

const double* jacobi_dinv64(sem_handle* h, double h1, double h2, cudaStream_t s) {
  ensure_dinv(h, h1, h2, nullptr, false, s);
  return h->f64.dinv.ptr;
}

void residual_f64(sem_handle* h, const double* b, const double* x, double h1, double h2,
                  double* w, double* r, CGState* st, cudaStream_t s) {
  launch_apply<double>(h, h->f64, x, w, h1, h2, nullptr, nullptr, SEM_APPLY_FULL, s);
  k_resid<<<kRedBlocks, kRedThreads, 0, s>>>(h->nL, b, w, r, nullptr, h->imult.ptr, st,
                                             h->partials.ptr, 1.0);
  SEM_CHECK_LAUNCH();
}

CGState state_to_host(const CGState* d, cudaStream_t s, int* dev_err) {
  return read_state(d, s, dev_err);
}

}  // namespace sem

using namespace sem;

extern "C" void sem_solve_opts_default(sem_solve_opts* o) {
  if (!o) return;
  o->h1 = 1.0;
  o->h2 = 0.0;
  o->h1_field = nullptr;
  o->tol = 1e-8;
  o->maxit = 20000;
  o->precision = SEM_SOLVE_F64;
  o->inner_tol = 1e-4;
  o->max_outer = 30;
  o->check_every = 16;
  o->use_graph = 1;
  o->x0_is_zero = 1;
  o->stream = nullptr;
}

extern "C" sem_status sem_cg_solve(sem_handle* h, const double* b_L, double* x_L,
                                   const sem_solve_opts* opts, sem_solve_info* info) {
  sem_solve_info local{};
  sem_status st = guarded("sem_cg_solve", [&] {
    SEM_REQUIRE(h && b_L && x_L, "sem_cg_solve: null handle or vector");
    sem_solve_opts o;
    if (opts) o = *opts; else sem_solve_opts_default(&o);
    SEM_REQUIRE(o.tol >= 0.0 && o.maxit >= 0, "sem_cg_solve: bad tol or maxit");
    SEM_REQUIRE(o.precision == SEM_SOLVE_F64 || o.precision == SEM_SOLVE_MIXED,
                "sem_cg_solve: bad precision");
    SEM_REQUIRE(o.precision == SEM_SOLVE_F64 || (o.inner_tol > 0.0 && o.inner_tol < 1.0),
                "sem_cg_solve: inner_tol must be in (0, 1)");
    StreamScope sc((cudaStream_t)o.stream);
    if (o.precision == SEM_SOLVE_F64 && h->cg_variant == SEM_CG_PIPELINED)
      solve_pipelined(h, b_L, x_L, o, local, sc.own);
    else if (o.precision == SEM_SOLVE_F64) solve_fp64(h, b_L, x_L, o, local, sc.own);
    else solve_mixed(h, b_L, x_L, o, local, sc.own);
  });
  if (info) *info = local;
  if (st != SEM_OK) {
    if (info) info->status = st;
    return st;
  }
  if (local.status != SEM_OK) {
    set_last_error(local.status == SEM_ERR_NOCONV ? "sem_cg_solve: no convergence within maxit"
                                                  : "sem_cg_solve: breakdown (<p,Hp> <= 0 or NaN)");
    return (sem_status)local.status;
  }
  return SEM_OK;
}

extern "C" sem_status sem_set_cg_variant(sem_handle* h, int kind) {
  return guarded("sem_set_cg_variant", [&] {
    SEM_REQUIRE(h, "sem_set_cg_variant: null handle");
    SEM_REQUIRE(kind == SEM_CG_STANDARD || kind == SEM_CG_PIPELINED,
                "sem_set_cg_variant: unknown kind");
    h->cg_variant = kind;
  });
}

extern "C" sem_status sem_set_inner_vectors(sem_handle* h, int kind) {
  return guarded("sem_set_inner_vectors", [&] {
    SEM_REQUIRE(h, "sem_set_inner_vectors: null handle");
    SEM_REQUIRE(kind == SEM_INNER_AUTO || kind == SEM_INNER_LOCAL || kind == SEM_INNER_GLOBAL,
                "sem_set_inner_vectors: unknown kind");
    h->inner_vectors = kind;
  });
}

extern "C" sem_status sem_rhs(sem_handle* h, const double* f_L, double* b_L, void* stream) {
  return guarded("sem_rhs", [&] {
    SEM_REQUIRE(h && f_L && b_L, "sem_rhs: null argument");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = h->nL;
    k_mul<<<ew_grid(n), 256, 0, s>>>(n, h->f64.B.ptr, f_L, b_L);
    SEM_CHECK_LAUNCH();
    launch_dssum<double>(h, b_L, true, nullptr, s);
  });
}

extern "C" sem_status sem_dot(sem_handle* h, const double* a, const double* b, double* out,
                              void* stream) {
  return guarded("sem_dot", [&] {
    SEM_REQUIRE(h && a && b && out, "sem_dot: null argument");
    cudaStream_t s = (cudaStream_t)stream;
    k_wdot<<<kRedBlocks, kRedThreads, 0, s>>>(h->nL, a, b, h->imult.ptr, out,
                                              h->partials.ptr + 2 * kRedBlocks,
                                              &h->state.ptr[2].counter);
    SEM_CHECK_LAUNCH();
  });
}

extern "C" sem_status sem_apply_host(sem_handle* h, const void* u_host, void* w_host, int dtype,
                                     void* stream) {
  return guarded("sem_apply_host", [&] {
    SEM_REQUIRE(h && u_host && w_host, "sem_apply_host: null argument");
    SEM_REQUIRE(dtype == SEM_F64 || dtype == SEM_F32, "sem_apply_host: bad dtype");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = h->nL;
    ensure(h->stage_in, n);
    ensure(h->stage_out, n);
    const size_t bytes = n * (dtype == SEM_F64 ? sizeof(double) : sizeof(float));
    if (dtype == SEM_F64 && host_pipeline_supported(h, h->stage_in.ptr, h->stage_out.ptr)) {
      apply_host_pipelined(h, (const double*)u_host, (double*)w_host, h->stage_in.ptr,
                           h->stage_out.ptr, s);
      int herr = 0;
      SEM_CUDA(cudaMemcpy(&herr, h->dev_err.ptr, sizeof(int), cudaMemcpyDeviceToHost));
      if (herr) {
        SEM_CUDA(cudaMemset(h->dev_err.ptr, 0, sizeof(int)));
        throw Error(SEM_ERR_TIMEOUT, "sem_apply_host: a bounded device wait timed out");
      }
      return;
    }
    SEM_CUDA(cudaMemcpyAsync(h->stage_in.ptr, u_host, bytes, cudaMemcpyHostToDevice, s));
    if (dtype == SEM_F64) {
      launch_apply<double>(h, h->f64, h->stage_in.ptr, h->stage_out.ptr, 1.0, 0.0, nullptr,
                           nullptr, SEM_APPLY_FULL, s);
    } else {
      if (!h->f32.G.ptr) throw Error(SEM_ERR_STATE, "sem_apply_host: no FP32 geometry");
      float* in = (float*)h->stage_in.ptr;
      float* out = (float*)h->stage_out.ptr;
      launch_apply<float>(h, h->f32, in, out, 1.0f, 0.0f, nullptr, nullptr, SEM_APPLY_FULL, s);
    }
    SEM_CUDA(cudaMemcpyAsync(w_host, h->stage_out.ptr, bytes, cudaMemcpyDeviceToHost, s));
    int herr = 0;
    SEM_CUDA(cudaMemcpyAsync(&herr, h->dev_err.ptr, sizeof(int), cudaMemcpyDeviceToHost, s));
    SEM_CUDA(cudaStreamSynchronize(s));
    if (herr) {
      SEM_CUDA(cudaMemsetAsync(h->dev_err.ptr, 0, sizeof(int), s));
      throw Error(SEM_ERR_TIMEOUT, "sem_apply_host: a bounded device wait timed out");
    }
  });
}
