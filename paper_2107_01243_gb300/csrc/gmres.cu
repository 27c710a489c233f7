// Flexible GMRES(m) with right preconditioning (arXiv 2107.01243 §4 and
// Table 2: Neko solves the pressure Poisson equation by preconditioned GMRES,
// the preconditioner being the two-level Schwarz method whose coarse level is
// solved only approximately, so the preconditioner varies between
// applications; the flexible form keeps the preconditioned directions).
//
// FP64 L-vectors, unique-dof inner product.  Per iteration j:
//   z_j = M^-1 v_j;  w = mask o QQ^T H z_j;
//   h = V^T w, w -= V h, twice (classical Gram-Schmidt repeated);
//   h_{j+1,j} = ||w||;  v_{j+1} = w / h_{j+1,j}
// The (m+1) x m Hessenberg matrix, its Givens rotations and the residual
// estimate live on the host (one synchronisation per iteration); x += Z y at
// the end of a cycle, and each cycle starts from the true residual.
//
// Mixed precision (gmres_solve_mixed): FP64 iterative refinement on
// L-vectors (residual r = b - Hx and update x += d in FP64, as the mixed CG
// does) around the same flexible GMRES in FP32 on global vectors: the
// operator of global.cu, the Schwarz preconditioner applied on global
// vectors, Gram-Schmidt dots accumulated per thread with Kahan compensation
// in FP32 and across threads in FP64.
#include <cmath>
#include <memory>
#include <vector>

#include "sem_internal.cuh"
#include "reduce.cuh"
#include "krylov.cuh"

namespace sem {
namespace {

constexpr int kMaxRestart = 32;         // vectors the Gram-Schmidt kernels hold (kGsMax)

// out = s v
__global__ void k_scale(int64_t n, const double* __restrict__ v, double sc,
                        double* __restrict__ out) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
       q += (int64_t)gridDim.x * blockDim.x)
    out[q] = sc * v[q];
}

// z = d o v
__global__ void k_hadamard(int64_t n, const double* __restrict__ d, const double* __restrict__ v,
                           double* __restrict__ z) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
       q += (int64_t)gridDim.x * blockDim.x)
    z[q] = d[q] * v[q];
}

constexpr int kGsMax = 32;            // vector pointers and coefficients an update kernel keeps

// Gram-Schmidt kernels.  Dots: blockIdx.y takes a chunk of kGsChunk vectors
// (eight accumulators per thread, full occupancy), each chunk reduced on its
// own counter and partials; updates loop over the vectors with the pointers
// and coefficients in shared memory.
constexpr int kGsChunk = 8;

// out[i] = <V_i, w>, i < cnt
__global__ void __launch_bounds__(kRedThreads)
k_gs_dots(int64_t n, const double* const* __restrict__ V, int cnt, const double* __restrict__ w,
          const float* __restrict__ imult, double* __restrict__ out, double* __restrict__ partials,
          unsigned* __restrict__ counters) {
  const int i0 = blockIdx.y * kGsChunk;
  const int c = min(kGsChunk, cnt - i0);
  const double* v[kGsChunk];
#pragma unroll
  for (int i = 0; i < kGsChunk; ++i) v[i] = i < c ? V[i0 + i] : nullptr;
  double acc[kGsChunk];
#pragma unroll
  for (int i = 0; i < kGsChunk; ++i) acc[i] = 0.0;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
       q += (int64_t)gridDim.x * blockDim.x) {
    const double wq = w[q] * (double)imult[q];
#pragma unroll
    for (int i = 0; i < kGsChunk; ++i)
      if (i < c) acc[i] = fma(v[i][q], wq, acc[i]);
  }
  double tot[kGsChunk];
  if (grid_sum<kGsChunk>(acc, partials + (size_t)blockIdx.y * kGsChunk * gridDim.x,
                         counters + blockIdx.y, tot) &&
      threadIdx.x == 0)
    for (int i = 0; i < c; ++i) out[i0 + i] = tot[i];
}

// w -= sum_{i < cnt} c_i V_i; with out, also out[0] = <w, w>
__global__ void __launch_bounds__(kRedThreads)
k_gs_update(int64_t n, const double* const* __restrict__ V, int cnt, const double* __restrict__ c,
            double* __restrict__ w, const float* __restrict__ imult, double* __restrict__ out,
            double* __restrict__ partials, unsigned* __restrict__ counter) {
  __shared__ const double* sv[kGsMax];
  __shared__ double sc[kGsMax];
  if (threadIdx.x < kGsMax) {
    sv[threadIdx.x] = threadIdx.x < cnt ? V[threadIdx.x] : nullptr;
    sc[threadIdx.x] = threadIdx.x < cnt ? c[threadIdx.x] : 0.0;
  }
  __syncthreads();
  double acc[1] = {0.0};
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
       q += (int64_t)gridDim.x * blockDim.x) {
    double wq = w[q];
#pragma unroll 4
    for (int i = 0; i < cnt; ++i) wq = fma(-sc[i], sv[i][q], wq);
    w[q] = wq;
    if (out) acc[0] = fma(wq * (double)imult[q], wq, acc[0]);
  }
  if (out) {
    double tot[1];
    if (grid_sum<1>(acc, partials, counter, tot) && threadIdx.x == 0) out[0] = tot[0];
  }
}

// h = c1 + c2 (the two Gram-Schmidt passes' coefficients), i < cnt
__global__ void k_hsum(int cnt, const double* __restrict__ c1, const double* __restrict__ c2,
                       double* __restrict__ h) {
  for (int i = threadIdx.x; i < cnt; i += blockDim.x) h[i] = c1[i] + c2[i];
}

}  // namespace

// Workspace of the GMRES solver, kept on the handle between solves.
struct GmresWork {
  sem_handle* h;
  int m;
  std::vector<std::unique_ptr<DevBuf<double>>> V, Z;
  DevBuf<double> w;
  DevBuf<const double*> vptr, zptr, one;
  DevBuf<double> coef, coef2, hcol, dots, partials;
  DevBuf<unsigned> counter;
  double* pin = nullptr;
  GmresWork(sem_handle* hh, int mm, cudaStream_t s) : h(hh), m(mm) {
    const int64_t n = h->nL;
    for (int i = 0; i <= m; ++i) {
      V.emplace_back(new DevBuf<double>());
      V.back()->alloc(n);
    }
    for (int i = 0; i < m; ++i) {
      Z.emplace_back(new DevBuf<double>());
      Z.back()->alloc(n);
    }
    w.alloc(n);
    std::vector<const double*> pv, pz;
    for (auto& b : V) pv.push_back(b->ptr);
    for (auto& b : Z) pz.push_back(b->ptr);
    vptr.alloc(m + 1);
    zptr.alloc(m);
    one.alloc(1);
    SEM_CUDA(cudaMemcpyAsync(vptr.ptr, pv.data(), pv.size() * sizeof(double*),
                             cudaMemcpyHostToDevice, s));
    SEM_CUDA(cudaMemcpyAsync(zptr.ptr, pz.data(), pz.size() * sizeof(double*),
                             cudaMemcpyHostToDevice, s));
    coef.alloc(m + 1);
    coef2.alloc(m + 1);
    hcol.alloc(m + 2);
    dots.alloc(1);
    partials.alloc((size_t)kGsMax * kRedBlocks);
    counter.alloc(kGsMax / kGsChunk + 1);      // one per dot chunk, one for the norm
    SEM_CUDA(cudaMemsetAsync(counter.ptr, 0, (kGsMax / kGsChunk + 1) * sizeof(unsigned), s));
    SEM_CUDA(cudaMallocHost(&pin, (m + 4) * sizeof(double)));
  }
  ~GmresWork() {
    if (pin) cudaFreeHost(pin);
  }
  // out[i] = <V_i, b>, i < cnt (device)
  void mdot(const double* const* Vp, int cnt, const double* b, double* out, cudaStream_t s) {
    for (int i0 = 0; i0 < cnt; i0 += kDotChunk) {
      const int c = std::min(kDotChunk, cnt - i0);
      k_mdot<kDotChunk><<<kRedBlocks, kRedThreads, 0, s>>>(h->nL, Vp, i0, c, b, h->imult.ptr,
                                                           out, partials.ptr, counter.ptr);
      SEM_CHECK_LAUNCH();
    }
  }
  double norm2_host(const double* a, cudaStream_t s) {
    const double* p[1] = {a};
    SEM_CUDA(cudaMemcpyAsync(one.ptr, p, sizeof(p), cudaMemcpyHostToDevice, s));
    mdot(one.ptr, 1, a, dots.ptr, s);
    SEM_CUDA(cudaMemcpyAsync(pin, dots.ptr, sizeof(double), cudaMemcpyDeviceToHost, s));
    SEM_CUDA(cudaStreamSynchronize(s));
    return pin[0];
  }
};

namespace {

// ---- FP32 FGMRES on global vectors (padded to a multiple of 4 with zeros):
// plain dots, Kahan-compensated per thread, FP64 across threads
struct KahanAcc {
  float s = 0.0f, c = 0.0f;
  __device__ __forceinline__ void add(float v) {
    const float y = __fsub_rn(v, c);
    const float t = __fadd_rn(s, y);
    c = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

// out[i] = <V_i, w>, i < cnt (blockIdx.y: chunk of kGsChunk vectors)
__global__ void __launch_bounds__(kRedThreads)
k_gsf_dots(int64_t n4, const float* const* __restrict__ V, int cnt, const float* __restrict__ w,
           double* __restrict__ out, double* __restrict__ partials,
           unsigned* __restrict__ counters) {
  const int i0 = blockIdx.y * kGsChunk;
  const int c = min(kGsChunk, cnt - i0);
  const float4* v[kGsChunk];
#pragma unroll
  for (int i = 0; i < kGsChunk; ++i)
    v[i] = i < c ? reinterpret_cast<const float4*>(V[i0 + i]) : nullptr;
  const float4* w4 = reinterpret_cast<const float4*>(w);
  KahanAcc acc[kGsChunk];
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n4;
       q += (int64_t)gridDim.x * blockDim.x) {
    const float4 wq = w4[q];
#pragma unroll
    for (int i = 0; i < kGsChunk; ++i)
      if (i < c) {
        const float4 a = v[i][q];
        acc[i].add(fmaf(a.x, wq.x, fmaf(a.y, wq.y, __fmul_rn(a.z, wq.z))) + a.w * wq.w);
      }
  }
  double tv[kGsChunk], tot[kGsChunk];
#pragma unroll
  for (int i = 0; i < kGsChunk; ++i) tv[i] = acc[i].value();
  if (grid_sum<kGsChunk>(tv, partials + (size_t)blockIdx.y * kGsChunk * gridDim.x,
                         counters + blockIdx.y, tot) &&
      threadIdx.x == 0)
    for (int i = 0; i < c; ++i) out[i0 + i] = tot[i];
}

// w -= sum_{i < cnt} c_i V_i (FP32); with out, also out[0] = <w, w>
__global__ void __launch_bounds__(kRedThreads)
k_gsf_update(int64_t n4, const float* const* __restrict__ V, int cnt, const double* __restrict__ c,
             float* __restrict__ w, double* __restrict__ out, double* __restrict__ partials,
             unsigned* __restrict__ counter) {
  __shared__ const float4* sv[kGsMax];
  __shared__ float sc[kGsMax];
  if (threadIdx.x < kGsMax) {
    sv[threadIdx.x] = threadIdx.x < cnt ? reinterpret_cast<const float4*>(V[threadIdx.x])
                                        : nullptr;
    sc[threadIdx.x] = threadIdx.x < cnt ? (float)c[threadIdx.x] : 0.0f;
  }
  __syncthreads();
  float4* w4 = reinterpret_cast<float4*>(w);
  KahanAcc acc;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n4;
       q += (int64_t)gridDim.x * blockDim.x) {
    float4 wq = w4[q];
#pragma unroll 4
    for (int i = 0; i < cnt; ++i) {
      const float4 a = sv[i][q];
      wq.x = fmaf(-sc[i], a.x, wq.x);
      wq.y = fmaf(-sc[i], a.y, wq.y);
      wq.z = fmaf(-sc[i], a.z, wq.z);
      wq.w = fmaf(-sc[i], a.w, wq.w);
    }
    w4[q] = wq;
    if (out) acc.add(fmaf(wq.x, wq.x, fmaf(wq.y, wq.y, __fmul_rn(wq.z, wq.z))) + wq.w * wq.w);
  }
  if (out) {
    double v[1] = {acc.value()}, tot[1];
    if (grid_sum<1>(v, partials, counter, tot) && threadIdx.x == 0) out[0] = tot[0];
  }
}

// out = s v (FP32)
__global__ void k_scalef(int64_t n4, const float* __restrict__ v, float sc, float* __restrict__ out) {
  const float4* v4 = reinterpret_cast<const float4*>(v);
  float4* o4 = reinterpret_cast<float4*>(out);
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n4;
       q += (int64_t)gridDim.x * blockDim.x) {
    const float4 a = v4[q];
    o4[q] = make_float4(sc * a.x, sc * a.y, sc * a.z, sc * a.w);
  }
}

// out = a - b (FP32)
__global__ void k_subf(int64_t n4, const float* __restrict__ a, const float* __restrict__ b,
                       float* __restrict__ out) {
  const float4* a4 = reinterpret_cast<const float4*>(a);
  const float4* b4 = reinterpret_cast<const float4*>(b);
  float4* o4 = reinterpret_cast<float4*>(out);
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n4;
       q += (int64_t)gridDim.x * blockDim.x) {
    const float4 x = a4[q], y = b4[q];
    o4[q] = make_float4(x.x - y.x, x.y - y.y, x.z - y.z, x.w - y.w);
  }
}

}  // namespace

// Workspace of the mixed-precision GMRES (FP32 global vectors), kept on the handle.
struct GmresWorkF {
  sem_handle* h;
  int m;
  int64_t n4;                              // padded global length / 4
  std::vector<std::unique_ptr<DevBuf<float>>> V, Z;
  DevBuf<float> w, r, d;                   // scratch, the inner residual, the correction
  DevBuf<const float*> vptr, zptr;
  DevBuf<double> coef, coef2, hcol, dots, partials;
  DevBuf<unsigned> counter;
  double* pin = nullptr;
  GmresWorkF(sem_handle* hh, int mm, cudaStream_t s) : h(hh), m(mm) {
    const int64_t n = glob_padded(h);
    n4 = n / 4;
    auto fresh = [&](DevBuf<float>& b) {
      b.alloc(n);
      SEM_CUDA(cudaMemsetAsync(b.ptr, 0, n * sizeof(float), s));
    };
    for (int i = 0; i <= m; ++i) {
      V.emplace_back(new DevBuf<float>());
      fresh(*V.back());
    }
    for (int i = 0; i < m; ++i) {
      Z.emplace_back(new DevBuf<float>());
      fresh(*Z.back());
    }
    fresh(w);
    fresh(r);
    fresh(d);
    std::vector<const float*> pv, pz;
    for (auto& b : V) pv.push_back(b->ptr);
    for (auto& b : Z) pz.push_back(b->ptr);
    vptr.alloc(m + 1);
    zptr.alloc(m);
    SEM_CUDA(cudaMemcpyAsync(vptr.ptr, pv.data(), pv.size() * sizeof(float*),
                             cudaMemcpyHostToDevice, s));
    SEM_CUDA(cudaMemcpyAsync(zptr.ptr, pz.data(), pz.size() * sizeof(float*),
                             cudaMemcpyHostToDevice, s));
    coef.alloc(m + 1);
    coef2.alloc(m + 1);
    hcol.alloc(m + 2);
    dots.alloc(1);
    partials.alloc((size_t)kGsMax * kRedBlocks);
    counter.alloc(kGsMax / kGsChunk + 1);
    SEM_CUDA(cudaMemsetAsync(counter.ptr, 0, (kGsMax / kGsChunk + 1) * sizeof(unsigned), s));
    SEM_CUDA(cudaMallocHost(&pin, (m + 4) * sizeof(double)));
  }
  ~GmresWorkF() {
    if (pin) cudaFreeHost(pin);
  }
  // <a, a> on the host (synchronises); the update kernel with no vectors
  // rewrites a unchanged and returns its norm
  double norm2_host(const float* a, cudaStream_t s) {
    k_gsf_update<<<kRedBlocks, kRedThreads, 0, s>>>(n4, vptr.ptr, 0, coef.ptr,
                                                    const_cast<float*>(a), dots.ptr, partials.ptr,
                                                    counter.ptr + kGsMax / kGsChunk);
    SEM_CHECK_LAUNCH();
    SEM_CUDA(cudaMemcpyAsync(pin, dots.ptr, sizeof(double), cudaMemcpyDeviceToHost, s));
    SEM_CUDA(cudaStreamSynchronize(s));
    return pin[0];
  }
};

namespace {

void check_timeout(sem_handle* h, cudaStream_t s) {
  int herr = 0;
  SEM_CUDA(cudaMemcpyAsync(&herr, h->dev_err.ptr, sizeof(int), cudaMemcpyDeviceToHost, s));
  SEM_CUDA(cudaStreamSynchronize(s));
  if (herr) {
    SEM_CUDA(cudaMemsetAsync(h->dev_err.ptr, 0, sizeof(int), s));
    throw Error(SEM_ERR_TIMEOUT, "a bounded device wait timed out during the solve");
  }
}

void gmres_solve(sem_handle* h, const double* b, double* x, const sem_solve_opts& o, int m,
                 sem_schwarz* M, sem_solve_info& info, cudaStream_t s) {
  const int64_t n = h->nL;
  if (!h->gmres || h->gmres->m < m) {
    h->gmres.reset();
    h->gmres = std::make_shared<GmresWork>(h, m, s);
  }
  GmresWork& g = *h->gmres;
  const double* dinv = M ? nullptr : jacobi_dinv64(h, o.h1, o.h2, s);
  const double bnorm = std::sqrt(g.norm2_host(b, s));
  if (o.x0_is_zero) SEM_CUDA(cudaMemsetAsync(x, 0, n * sizeof(double), s));
  info = sem_solve_info{0, 0, 0.0, SEM_OK};
  if (bnorm == 0.0) {
    SEM_CUDA(cudaMemsetAsync(x, 0, n * sizeof(double), s));
    SEM_CUDA(cudaStreamSynchronize(s));
    return;
  }
  CGState* st = h->state.ptr;
  std::vector<double> H((m + 1) * m), cs(m), sn(m), gv(m + 1), y(m);
  int total = 0, cycles = 0;
  for (;;) {
    // true residual into V_0
    residual_f64(h, b, x, o.h1, o.h2, g.w.ptr, g.V[0]->ptr, st, s);
    const CGState hs = state_to_host(st, s, h->dev_err.ptr);
    const double beta = std::sqrt(hs.rr);
    info.rel_res = beta / bnorm;
    if (!(beta == beta)) { info.status = SEM_ERR_BREAKDOWN; break; }
    if (beta <= o.tol * bnorm) { info.status = SEM_OK; break; }
    if (total >= o.maxit) { info.status = SEM_ERR_NOCONV; break; }
    ++cycles;
    k_scale<<<lin_grid(n), 256, 0, s>>>(n, g.V[0]->ptr, 1.0 / beta, g.V[0]->ptr);
    SEM_CHECK_LAUNCH();
    std::fill(H.begin(), H.end(), 0.0);
    std::fill(gv.begin(), gv.end(), 0.0);
    gv[0] = beta;
    int k = 0;
    for (int j = 0; j < m; ++j) {
      double* zj = g.Z[j]->ptr;
      if (M) {
        schwarz_apply(M, g.V[j]->ptr, zj, s);
      } else {
        k_hadamard<<<lin_grid(n), 256, 0, s>>>(n, dinv, g.V[j]->ptr, zj);
        SEM_CHECK_LAUNCH();
      }
      launch_apply<double>(h, h->f64, zj, g.w.ptr, o.h1, o.h2, nullptr, nullptr, SEM_APPLY_FULL,
                           s);
      // classical Gram-Schmidt twice: c1 = V^T w; w -= V c1, c2 = V^T w; w -= V c2, ||w||^2
      const int cnt = j + 1;
      const dim3 dgrid(kRedBlocks, (cnt + kGsChunk - 1) / kGsChunk);
      k_gs_dots<<<dgrid, kRedThreads, 0, s>>>(n, g.vptr.ptr, cnt, g.w.ptr, h->imult.ptr,
                                              g.coef.ptr, g.partials.ptr, g.counter.ptr);
      SEM_CHECK_LAUNCH();
      k_gs_update<<<kRedBlocks, kRedThreads, 0, s>>>(n, g.vptr.ptr, cnt, g.coef.ptr, g.w.ptr,
                                                     h->imult.ptr, nullptr, nullptr, nullptr);
      SEM_CHECK_LAUNCH();
      k_gs_dots<<<dgrid, kRedThreads, 0, s>>>(n, g.vptr.ptr, cnt, g.w.ptr, h->imult.ptr,
                                              g.coef2.ptr, g.partials.ptr, g.counter.ptr);
      SEM_CHECK_LAUNCH();
      k_gs_update<<<kRedBlocks, kRedThreads, 0, s>>>(n, g.vptr.ptr, cnt, g.coef2.ptr, g.w.ptr,
                                                     h->imult.ptr, g.dots.ptr, g.partials.ptr,
                                                     g.counter.ptr + kGsMax / kGsChunk);
      SEM_CHECK_LAUNCH();
      k_hsum<<<1, 64, 0, s>>>(cnt, g.coef.ptr, g.coef2.ptr, g.hcol.ptr);
      SEM_CHECK_LAUNCH();
      SEM_CUDA(cudaMemcpyAsync(g.pin, g.hcol.ptr, (j + 1) * sizeof(double),
                               cudaMemcpyDeviceToHost, s));
      SEM_CUDA(cudaMemcpyAsync(g.pin + m + 2, g.dots.ptr, sizeof(double), cudaMemcpyDeviceToHost,
                               s));
      check_timeout(h, s);                    // synchronises
      for (int i = 0; i <= j; ++i) H[i * m + j] = g.pin[i];
      const double hn = std::sqrt(std::max(0.0, g.pin[m + 2]));
      for (int i = 0; i < j; ++i) {
        const double t = cs[i] * H[i * m + j] + sn[i] * H[(i + 1) * m + j];
        H[(i + 1) * m + j] = -sn[i] * H[i * m + j] + cs[i] * H[(i + 1) * m + j];
        H[i * m + j] = t;
      }
      const double a = H[j * m + j];
      if (hn == 0.0) {
        cs[j] = 1.0;
        sn[j] = 0.0;
      } else {
        const double r = std::hypot(a, hn);
        cs[j] = a / r;
        sn[j] = hn / r;
      }
      H[j * m + j] = cs[j] * a + sn[j] * hn;
      gv[j + 1] = -sn[j] * gv[j];
      gv[j] = cs[j] * gv[j];
      k = j + 1;
      ++total;
      if (!(H[j * m + j] != 0.0) || !(hn == hn)) { info.status = SEM_ERR_BREAKDOWN; break; }
      if (std::fabs(gv[j + 1]) <= o.tol * bnorm || total >= o.maxit || hn == 0.0) break;
      k_scale<<<lin_grid(n), 256, 0, s>>>(n, g.w.ptr, 1.0 / hn, g.V[j + 1]->ptr);
      SEM_CHECK_LAUNCH();
    }
    if (info.status == SEM_ERR_BREAKDOWN) break;
    for (int i = k - 1; i >= 0; --i) {
      double acc = gv[i];
      for (int l = i + 1; l < k; ++l) acc -= H[i * m + l] * y[l];
      y[i] = acc / H[i * m + i];
    }
    SEM_CUDA(cudaMemcpyAsync(g.coef.ptr, y.data(), k * sizeof(double), cudaMemcpyHostToDevice, s));
    k_mcomb<<<lin_grid(n), 256, 0, s>>>(n, g.zptr.ptr, k, g.coef.ptr, 1.0, x, x);
    SEM_CHECK_LAUNCH();
  }
  info.iters = total;
  info.outer_iters = cycles;
  SEM_CUDA(cudaStreamSynchronize(s));
}

// Mixed precision: FP64 refinement on L-vectors around an FP32 flexible
// GMRES on global vectors (operator sem_apply_global, the Schwarz
// preconditioner on global vectors), each inner solve to the relative
// tolerance inner_target(inner_tol, tol, outer residual).
void gmres_solve_mixed(sem_handle* h, const double* b, double* x, const sem_solve_opts& o, int m,
                       sem_schwarz* M, sem_solve_info& info, cudaStream_t s) {
  const int64_t nL = h->nL;
  if (!h->gmres32 || h->gmres32->m < m) {
    h->gmres32.reset();
    h->gmres32 = std::make_shared<GmresWorkF>(h, m, s);
  }
  GmresWorkF& g = *h->gmres32;
  const int64_t n4 = g.n4;
  const size_t gbytes = (size_t)n4 * 4 * sizeof(float);
  for (DevBuf<double>* v : {&h->r, &h->w}) if (v->n < (size_t)nL) v->alloc(nL);
  if (h->rg.n < (size_t)(n4 * 4)) {                    // the residual's global copy
    h->rg.alloc(n4 * 4);
    SEM_CUDA(cudaMemsetAsync(h->rg.ptr, 0, gbytes, s));
  }
  CGState* st = h->state.ptr;
  outer_norm_b(h, b, s);
  inner_scale_from_b(h, s);
  if (o.x0_is_zero) SEM_CUDA(cudaMemsetAsync(x, 0, nL * sizeof(double), s));
  info = sem_solve_info{0, 0, 0.0, SEM_ERR_NOCONV};
  std::vector<double> H((m + 1) * m), cs(m), sn(m), gv(m + 1), y(m);
  int total = 0, outer = 0;
  const float* r_in = h->rg.ptr;
  for (;;) {
    outer_residual_global(h, b, x, o, s);               // r = b - H x (FP64), rg its copy
    const CGState hs = state_to_host(st, s, h->dev_err.ptr);
    const double rel = hs.bb > 0 ? std::sqrt(hs.rr / hs.bb) : 0.0;
    info.rel_res = rel;
    if (!(rel == rel)) { info.status = SEM_ERR_BREAKDOWN; break; }
    if (rel <= o.tol) { info.status = SEM_OK; break; }
    if (outer >= o.max_outer || total >= o.maxit) { info.status = SEM_ERR_NOCONV; break; }
    ++outer;
    const double itol = inner_target(o.inner_tol, o.tol, rel);
    SEM_CUDA(cudaMemsetAsync(g.d.ptr, 0, gbytes, s));
    const double beta0 = std::sqrt(g.norm2_host(r_in, s));
    bool breakdown = false;
    for (int cycle = 0; total < o.maxit; ++cycle) {
      // inner residual r_g - H d (d = 0 in the first cycle)
      if (cycle == 0) {
        SEM_CUDA(cudaMemcpyAsync(g.r.ptr, r_in, gbytes, cudaMemcpyDeviceToDevice, s));
      } else {
        SEM_CUDA(cudaMemsetAsync(g.w.ptr, 0, gbytes, s));
        launch_apply_global(h, g.d.ptr, g.w.ptr, (float)o.h1, (float)o.h2, nullptr, nullptr, s);
        k_subf<<<lin_grid(n4), 256, 0, s>>>(n4, r_in, g.w.ptr, g.r.ptr);
        SEM_CHECK_LAUNCH();
      }
      const double beta = std::sqrt(g.norm2_host(g.r.ptr, s));
      if (!(beta > itol * beta0)) break;
      k_scalef<<<lin_grid(n4), 256, 0, s>>>(n4, g.r.ptr, (float)(1.0 / beta), g.V[0]->ptr);
      SEM_CHECK_LAUNCH();
      std::fill(H.begin(), H.end(), 0.0);
      std::fill(gv.begin(), gv.end(), 0.0);
      gv[0] = beta;
      int k = 0;
      for (int j = 0; j < m; ++j) {
        schwarz_apply_global(M, g.V[j]->ptr, g.Z[j]->ptr, s);
        SEM_CUDA(cudaMemsetAsync(g.w.ptr, 0, gbytes, s));
        launch_apply_global(h, g.Z[j]->ptr, g.w.ptr, (float)o.h1, (float)o.h2, nullptr, nullptr,
                            s);
        const int cnt = j + 1;
        const dim3 dgrid(kRedBlocks, (cnt + kGsChunk - 1) / kGsChunk);
        k_gsf_dots<<<dgrid, kRedThreads, 0, s>>>(n4, g.vptr.ptr, cnt, g.w.ptr, g.coef.ptr,
                                                 g.partials.ptr, g.counter.ptr);
        SEM_CHECK_LAUNCH();
        k_gsf_update<<<kRedBlocks, kRedThreads, 0, s>>>(n4, g.vptr.ptr, cnt, g.coef.ptr, g.w.ptr,
                                                        nullptr, nullptr, nullptr);
        SEM_CHECK_LAUNCH();
        k_gsf_dots<<<dgrid, kRedThreads, 0, s>>>(n4, g.vptr.ptr, cnt, g.w.ptr, g.coef2.ptr,
                                                 g.partials.ptr, g.counter.ptr);
        SEM_CHECK_LAUNCH();
        k_gsf_update<<<kRedBlocks, kRedThreads, 0, s>>>(n4, g.vptr.ptr, cnt, g.coef2.ptr, g.w.ptr,
                                                        g.dots.ptr, g.partials.ptr,
                                                        g.counter.ptr + kGsMax / kGsChunk);
        SEM_CHECK_LAUNCH();
        k_hsum<<<1, 64, 0, s>>>(cnt, g.coef.ptr, g.coef2.ptr, g.hcol.ptr);
        SEM_CHECK_LAUNCH();
        SEM_CUDA(cudaMemcpyAsync(g.pin, g.hcol.ptr, cnt * sizeof(double), cudaMemcpyDeviceToHost,
                                 s));
        SEM_CUDA(cudaMemcpyAsync(g.pin + m + 2, g.dots.ptr, sizeof(double),
                                 cudaMemcpyDeviceToHost, s));
        check_timeout(h, s);
        for (int i = 0; i <= j; ++i) H[i * m + j] = g.pin[i];
        const double hn = std::sqrt(std::max(0.0, g.pin[m + 2]));
        for (int i = 0; i < j; ++i) {
          const double t = cs[i] * H[i * m + j] + sn[i] * H[(i + 1) * m + j];
          H[(i + 1) * m + j] = -sn[i] * H[i * m + j] + cs[i] * H[(i + 1) * m + j];
          H[i * m + j] = t;
        }
        const double a = H[j * m + j];
        if (hn == 0.0) {
          cs[j] = 1.0;
          sn[j] = 0.0;
        } else {
          const double r = std::hypot(a, hn);
          cs[j] = a / r;
          sn[j] = hn / r;
        }
        H[j * m + j] = cs[j] * a + sn[j] * hn;
        gv[j + 1] = -sn[j] * gv[j];
        gv[j] = cs[j] * gv[j];
        k = j + 1;
        ++total;
        if (!(H[j * m + j] != 0.0) || !(hn == hn)) { breakdown = true; break; }
        if (std::fabs(gv[j + 1]) <= itol * beta0 || total >= o.maxit || hn == 0.0) break;
        k_scalef<<<lin_grid(n4), 256, 0, s>>>(n4, g.w.ptr, (float)(1.0 / hn), g.V[j + 1]->ptr);
        SEM_CHECK_LAUNCH();
      }
      if (breakdown) break;
      for (int i = k - 1; i >= 0; --i) {
        double acc = gv[i];
        for (int l = i + 1; l < k; ++l) acc -= H[i * m + l] * y[l];
        y[i] = acc / H[i * m + i];
      }
      for (int i = 0; i < k; ++i) g.pin[i] = -y[i];   // d -= (-y) Z: the kernel subtracts
      SEM_CUDA(cudaMemcpyAsync(g.coef.ptr, g.pin, k * sizeof(double), cudaMemcpyHostToDevice, s));
      k_gsf_update<<<kRedBlocks, kRedThreads, 0, s>>>(n4, g.zptr.ptr, k, g.coef.ptr, g.d.ptr,
                                                      nullptr, nullptr, nullptr);
      SEM_CHECK_LAUNCH();
      if (std::fabs(gv[k]) <= itol * beta0) break;
    }
    if (breakdown) { info.status = SEM_ERR_BREAKDOWN; break; }
    add_from_global(h, x, g.d.ptr, s, 1.0 / h->rscale);
  }
  info.iters = total;
  info.outer_iters = outer;
  SEM_CUDA(cudaStreamSynchronize(s));
}

}  // namespace
}  // namespace sem

using namespace sem;

extern "C" sem_status sem_gmres_solve(sem_handle* h, const double* b_L, double* x_L,
                                      const sem_solve_opts* opts, int restart,
                                      sem_schwarz* precond, sem_solve_info* info) {
  sem_solve_info local{};
  sem_status st = guarded("sem_gmres_solve", [&] {
    SEM_REQUIRE(h && b_L && x_L, "sem_gmres_solve: null handle or vector");
    sem_solve_opts o;
    if (opts) o = *opts; else sem_solve_opts_default(&o);
    SEM_REQUIRE(o.tol >= 0.0 && o.maxit >= 0, "sem_gmres_solve: bad tol or maxit");
    SEM_REQUIRE(o.h1_field == nullptr, "sem_gmres_solve: a per-point h1 is not supported");
    SEM_REQUIRE(restart >= 1 && restart <= kMaxRestart, "sem_gmres_solve: restart in [1, 32]");
    SEM_REQUIRE(!precond || schwarz_handle(precond) == h,
                "sem_gmres_solve: the preconditioner belongs to another handle");
    SEM_REQUIRE(b_L != x_L, "sem_gmres_solve: b and x must not alias");
    cudaStream_t s = (cudaStream_t)o.stream;
    if (o.precision == SEM_SOLVE_MIXED && precond && glob_supported(h) &&
        h->inner_vectors != SEM_INNER_LOCAL) {
      SEM_REQUIRE(o.inner_tol > 0.0 && o.inner_tol < 1.0,
                  "sem_gmres_solve: inner_tol must be in (0, 1)");
      gmres_solve_mixed(h, b_L, x_L, o, restart, precond, local, s);
    } else {
      gmres_solve(h, b_L, x_L, o, restart, precond, local, s);
    }
  });
  if (info) *info = local;
  if (st != SEM_OK) {
    if (info) info->status = st;
    return st;
  }
  if (local.status != SEM_OK) {
    set_last_error(local.status == SEM_ERR_NOCONV ? "sem_gmres_solve: no convergence within maxit"
                                                  : "sem_gmres_solve: breakdown");
    return (sem_status)local.status;
  }
  return SEM_OK;
}
