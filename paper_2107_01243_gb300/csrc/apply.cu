// The assembled operator w = mask o QQ^T (h1 A_L + h2 B_L) u (arXiv 2107.01243
// §2, Eq. 9-10) with the gather-scatter split by direction.  On the box,
// QQ^T is the product of three commuting pair sums, one per direction: the
// copies of a point on an x-interface are the i = N value of element e and
// the i = 0 value of element e + 1, and so on for y (e + nelx) and z
// (e + nelx nely).  Summing the x-pairs, then the y-pairs, then the z-pairs
// gives every copy the sum of all its copies (2, 4 or 8).
//
//   local   the element kernel walks segments of kFuseSeg consecutive elements
//           per CTA and sums the x-pairs inside a segment itself (the upper
//           element reads back the copy the lower one stored just before);
//           masked points are written as zero
//   finish  k_sx_cut: x-pairs between segments;
//           k_sy, k_sz: the y- and z-pairs, each a coalesced sweep over the
//           j = N / k = N planes of the elements and their neighbours' j = 0 /
//           k = 0 planes
//
// The x-face copies are 8-byte values 64 bytes apart (P = 8), so a separate
// gather-scatter spends a 32-byte sector on each; here they never leave the
// element kernel.  Summation order: ((x-pairs) + (x-pairs)) + ..., i.e. the
// copies of an edge point are added as (w0 + w1) + (w2 + w3); sem_dssum keeps
// the increasing-index order instead.
#include "sem_internal.cuh"
#include <type_traits>

#include "ax_tile.cuh"

namespace sem {

bool launch_ax_tma_fused(const sem_handle* h, const float* u, float* w, float h1, float h2,
                         const float* h1f, const CGState* st, CGState* pwst, cudaStream_t s);
bool launch_ax_df_fused(const sem_handle* h, const double* u, double* w, double h1, double h2,
                        const CGState* st, CGState* pwst, cudaStream_t s);
void launch_ax_df_fused_slab(const sem_handle* h, const double* u, double* w, double h1,
                             double h2, int z0, int z1, cudaStream_t s);
bool df_ax_supported(const sem_handle* h, const void* u, const void* w, const void* h1f);

namespace {

// x-pairs at the segment starts of the element kernel: the first element
// e_b = g kFuseSeg of segment g >= 1 pairs its i = 0 face with the i = N face
// of the element before it, unless it starts an x-row.  One block per segment
// start.
template <int P, class T>
__global__ void __launch_bounds__(P * P)
k_sx_cut(T* __restrict__ w, int nelx, const CGState* __restrict__ st) {
  if (st && st->done) return;
  constexpr int P2 = P * P;
  constexpr long long P3 = (long long)P2 * P;
  const long long eb = (long long)(blockIdx.x + 1) * kFuseSeg;
  if (eb % nelx == 0) return;
  const int j = threadIdx.x % P, k = threadIdx.x / P;
  const long long hi = eb * P3 + (long long)k * P2 + j * P;    // (eb, 0, j, k)
  const long long lo = hi - P3 + (P - 1);                       // (eb - 1, N, j, k)
  const T sum = w[lo] + w[hi];
  w[lo] = sum;
  w[hi] = sum;
}

template <class T>
struct Vec2;
template <>
struct Vec2<float> {
  using V = float2;
};
template <>
struct Vec2<double> {
  using V = double2;
};

// y-pairs: (e, i, N, k) + (e + nelx, i, 0, k) for every element with
// ey < nely - 1; a thread takes two neighbouring i (P is even), threads run
// over (i pair, k, element) with the i pair fastest
template <int P, class T>
__global__ void __launch_bounds__(256)
k_sy(T* __restrict__ w, int nelx, int nely, uint32_t total, FastDiv dnx, FastDiv dny1,
     const CGState* __restrict__ st) {
  if (st && st->done) return;
  using V = typename Vec2<T>::V;
  constexpr int H = P / 2, P2 = P * P, P3 = P2 * P;
  V* wv = reinterpret_cast<V*>(w);
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += gridDim.x * blockDim.x) {
    const uint32_t ip = t % H, r = t / H;
    const uint32_t k = r % P, m = r / P;            // element among those with ey < nely - 1
    const uint32_t r2 = dnx.div(m);
    const uint32_t ex = m - r2 * (uint32_t)nelx;
    const uint32_t ez = dny1.div(r2);
    const uint32_t ey = r2 - ez * (uint32_t)(nely - 1);
    const uint32_t e = ex + (uint32_t)nelx * (ey + (uint32_t)nely * ez);
    const uint32_t lo = (e * P3 + k * P2 + (P - 1) * P) / 2 + ip;
    const uint32_t hi = ((e + nelx) * P3 + k * P2) / 2 + ip;
    const V a = wv[lo], b = wv[hi];
    const V sum = {a.x + b.x, a.y + b.y};
    wv[lo] = sum;
    wv[hi] = sum;
  }
}

// z-pairs: (e, i, j, N) + (e + nelx nely, i, j, 0) for every element with
// ez < nelz - 1 (the first nelx nely (nelz - 1) elements); 16 bytes per thread
template <int P, class T>
__global__ void __launch_bounds__(256)
k_sz(T* __restrict__ w, uint32_t layer, uint32_t total, const CGState* __restrict__ st) {
  if (st && st->done) return;
  constexpr int VW = 16 / (int)sizeof(T), P2 = P * P, P3 = P2 * P, Q = P2 / VW;
  static_assert(P2 % VW == 0, "plane not a whole number of 16-byte vectors");
  using V = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
  V* wv = reinterpret_cast<V*>(w);
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += gridDim.x * blockDim.x) {
    const uint32_t q = t % Q, e = t / Q;
    const uint32_t lo = (e * P3 + (P - 1) * P2) / VW + q;
    const uint32_t hi = ((e + layer) * P3) / VW + q;
    V a = wv[lo];
    const V b = wv[hi];
    T* ap = reinterpret_cast<T*>(&a);
    const T* bp = reinterpret_cast<const T*>(&b);
#pragma unroll
    for (int c = 0; c < VW; ++c) ap[c] = ap[c] + bp[c];
    wv[lo] = a;
    wv[hi] = a;
  }
}

int sweep_blocks(long long total) {
  return (int)std::max<long long>(1, std::min<long long>((total + 255) / 256, 16LL * sem_num_sms()));
}

// the finishing passes on a box of nelx x nely x nelz elements starting at w
template <int P, class T>
void finish_box(T* w, int nelx, int nely, int nelz, const CGState* st, cudaStream_t s) {
  const long long E = (long long)nelx * nely * nelz;
  const long long nseg = (E + kFuseSeg - 1) / kFuseSeg;
  if (nseg > 1 && nelx > 1) {
    k_sx_cut<P, T><<<(unsigned)(nseg - 1), P * P, 0, s>>>(w, nelx, st);
    SEM_CHECK_LAUNCH();
  }
  if (nely > 1) {
    const long long total = (long long)nelx * (nely - 1) * nelz * P * (P / 2);
    k_sy<P, T><<<sweep_blocks(total), 256, 0, s>>>(
        w, nelx, nely, (uint32_t)total, FastDiv((uint32_t)nelx), FastDiv((uint32_t)(nely - 1)),
        st);
    SEM_CHECK_LAUNCH();
  }
  if (nelz > 1) {
    const long long layer = (long long)nelx * nely;
    const long long total = layer * (nelz - 1) * P * P / (16 / (int)sizeof(T));
    k_sz<P, T><<<sweep_blocks(total), 256, 0, s>>>(w, (uint32_t)layer, (uint32_t)total, st);
    SEM_CHECK_LAUNCH();
  }
}

template <int P, class T>
void finish_p(const sem_handle* h, T* w, const CGState* st, cudaStream_t s) {
  finish_box<P, T>(w, h->nelx, h->nely, h->nelz, st, s);
}

// z-pairs between element planes z - 1 and z of the box (one plane of pairs)
template <int P, class T>
void zpairs_between(const sem_handle* h, T* w, int z, cudaStream_t s) {
  constexpr long long P3 = (long long)P * P * P;
  const long long layer = (long long)h->nelx * h->nely;
  const long long total = layer * P * P / (16 / (int)sizeof(T));
  k_sz<P, T><<<sweep_blocks(total), 256, 0, s>>>(w + (z - 1) * layer * P3, (uint32_t)layer,
                                                  (uint32_t)total, nullptr);
  SEM_CHECK_LAUNCH();
}

// the finishing passes of the slab of element planes [z0, z1), then (z0 > 0)
// the z-pairs between it and the slab below
template <int P>
void finish_slab(const sem_handle* h, double* w, int z0, int z1, cudaStream_t s) {
  constexpr long long P3 = (long long)P * P * P;
  finish_box<P, double>(w + (long long)z0 * h->nelx * h->nely * P3, h->nelx, h->nely, z1 - z0,
                        nullptr, s);
  if (z0 > 0) zpairs_between<P, double>(h, w, z0, s);
}

template <class T>
void finish(const sem_handle* h, T* w, const CGState* st, cudaStream_t s) {
  switch (h->P) {
    case 2: finish_p<2, T>(h, w, st, s); break;
    case 4: finish_p<4, T>(h, w, st, s); break;
    case 6: finish_p<6, T>(h, w, st, s); break;
    case 8: finish_p<8, T>(h, w, st, s); break;
    case 10: finish_p<10, T>(h, w, st, s); break;
    default: throw Error(SEM_ERR_ARG, "apply: unsupported order");
  }
}

}  // namespace

template <>
bool apply_fused_supported<float>(const sem_handle* h, const void* u, const void* w,
                                  const void* h1f) {
  return h->f32.G.ptr && tma_ax_supported<float>(h, u, w, h1f) && h->nL < (1LL << 31);
}

template <>
bool apply_fused_supported<double>(const sem_handle* h, const void* u, const void* w,
                                   const void* h1f) {
  return h->f64_kernel != SEM_F64_KERNEL_NATIVE && df_ax_supported(h, u, w, h1f) &&
         h->nL < (1LL << 31);
}

template <class T>
bool launch_apply(sem_handle* h, const OpData<T>& op, const T* u, T* w, T h1, T h2, const T* h1f,
                  const CGState* st, int phase, cudaStream_t s, CGState* pwst) {
  if (!apply_fused_supported<T>(h, u, w, h1f)) {
    // element kernel and the gather-scatter kernel, in the full phase
    if (phase & SEM_APPLY_LOCAL) launch_ax<T>(h, op, u, w, h1, h2, h1f, st, s);
    if (phase & SEM_APPLY_FINISH) launch_dssum<T>(h, w, true, st, s);
    return false;
  }
  bool pw = false;
  if (phase & SEM_APPLY_LOCAL) {
    if constexpr (std::is_same<T, float>::value)
      pw = launch_ax_tma_fused(h, u, w, h1, h2, h1f, st, pwst, s);
    else
      pw = launch_ax_df_fused(h, u, w, h1, h2, st, pwst, s);
  }
  if (phase & SEM_APPLY_FINISH) finish<T>(h, w, st, s);
  return pw;
}

// Streams and events of the pipelined host-buffer operator, kept per handle.
struct HostPipe {
  static constexpr int kSlabs = 8;
  cudaStream_t in = nullptr, comp = nullptr, out = nullptr;
  cudaEvent_t start = nullptr, arrived[kSlabs] = {}, final_[kSlabs] = {};
  HostPipe() {
    SEM_CUDA(cudaStreamCreateWithFlags(&in, cudaStreamNonBlocking));
    SEM_CUDA(cudaStreamCreateWithFlags(&comp, cudaStreamNonBlocking));
    SEM_CUDA(cudaStreamCreateWithFlags(&out, cudaStreamNonBlocking));
    SEM_CUDA(cudaEventCreateWithFlags(&start, cudaEventDisableTiming));
    for (int q = 0; q < kSlabs; ++q) {
      SEM_CUDA(cudaEventCreateWithFlags(&arrived[q], cudaEventDisableTiming));
      SEM_CUDA(cudaEventCreateWithFlags(&final_[q], cudaEventDisableTiming));
    }
  }
  ~HostPipe() {
    for (int q = 0; q < kSlabs; ++q) {
      if (arrived[q]) cudaEventDestroy(arrived[q]);
      if (final_[q]) cudaEventDestroy(final_[q]);
    }
    if (start) cudaEventDestroy(start);
    for (cudaStream_t t : {in, comp, out})
      if (t) cudaStreamDestroy(t);
  }
};

bool host_pipeline_supported(const sem_handle* h, const void* din, const void* dout) {
  return h->nelz >= 2 && apply_fused_supported<double>(h, din, dout, nullptr);
}

// w_host = mask o QQ^T A_L u_host (FP64) with the copies overlapped with the
// work: the box is cut into slabs of element planes; slab q is copied in on
// one stream, its element kernel and finishing passes (and the z-pairs with
// slab q - 1) run on a second, and the planes those passes made final are
// copied out on a third while later slabs are still arriving or being
// computed.  Every pair sum is the one the unsplit operator forms, so the
// result is the same.
void apply_host_pipelined(sem_handle* h, const double* u_host, double* w_host, double* din,
                          double* dout, cudaStream_t user) {
  if (!h->host_pipe) h->host_pipe = std::make_shared<HostPipe>();
  HostPipe& hp = *h->host_pipe;
  const int S = std::min(HostPipe::kSlabs, h->nelz);
  const long long P3 = h->P3, layer = (long long)h->nelx * h->nely;
  std::vector<int> z(S + 1);
  for (int q = 0; q <= S; ++q) z[q] = (int)((long long)q * h->nelz / S);
  SEM_CUDA(cudaEventRecord(hp.start, user));
  SEM_CUDA(cudaStreamWaitEvent(hp.in, hp.start, 0));
  SEM_CUDA(cudaStreamWaitEvent(hp.comp, hp.start, 0));
  SEM_CUDA(cudaStreamWaitEvent(hp.out, hp.start, 0));
  for (int q = 0; q < S; ++q) {
    const long long o = z[q] * layer * P3, n = (long long)(z[q + 1] - z[q]) * layer * P3;
    SEM_CUDA(cudaMemcpyAsync(din + o, u_host + o, n * sizeof(double), cudaMemcpyHostToDevice,
                             hp.in));
    SEM_CUDA(cudaEventRecord(hp.arrived[q], hp.in));
  }
  for (int q = 0; q < S; ++q) {
    SEM_CUDA(cudaStreamWaitEvent(hp.comp, hp.arrived[q], 0));
    launch_ax_df_fused_slab(h, din, dout, 1.0, 0.0, z[q], z[q + 1], hp.comp);
    switch (h->P) {
      case 6: finish_slab<6>(h, dout, z[q], z[q + 1], hp.comp); break;
      case 8: finish_slab<8>(h, dout, z[q], z[q + 1], hp.comp); break;
      case 10: finish_slab<10>(h, dout, z[q], z[q + 1], hp.comp); break;
      default: throw Error(SEM_ERR_ARG, "apply_host_pipelined: unsupported order");
    }
    SEM_CUDA(cudaEventRecord(hp.final_[q], hp.comp));
  }
  // after slab q's passes the planes from the last plane of slab q - 1 up to
  // (not including) slab q's last plane are final; the last slab's last
  // plane too
  for (int q = 0; q < S; ++q) {
    const long long p0 = q == 0 ? z[0] : z[q] - 1, p1 = q == S - 1 ? z[S] : z[q + 1] - 1;
    if (p1 <= p0) continue;
    const long long o = p0 * layer * P3, n = (p1 - p0) * layer * P3;
    SEM_CUDA(cudaStreamWaitEvent(hp.out, hp.final_[q], 0));
    SEM_CUDA(cudaMemcpyAsync(w_host + o, dout + o, n * sizeof(double), cudaMemcpyDeviceToHost,
                             hp.out));
  }
  SEM_CUDA(cudaStreamSynchronize(hp.out));
  SEM_CUDA(cudaStreamSynchronize(hp.comp));
}

template bool launch_apply<float>(sem_handle*, const OpData<float>&, const float*, float*, float,
                                  float, const float*, const CGState*, int, cudaStream_t,
                                  CGState*);
template bool launch_apply<double>(sem_handle*, const OpData<double>&, const double*, double*,
                                   double, double, const double*, const CGState*, int,
                                   cudaStream_t, CGState*);

}  // namespace sem

using namespace sem;

extern "C" sem_status sem_apply(sem_handle* h, const void* u_L, void* w_L, double h1, double h2,
                                const void* h1_field, int dtype, int phase, void* stream) {
  return guarded("sem_apply", [&] {
    SEM_REQUIRE(h && u_L && w_L, "sem_apply: null argument");
    SEM_REQUIRE(phase == SEM_APPLY_FULL || phase == SEM_APPLY_LOCAL || phase == SEM_APPLY_FINISH,
                "sem_apply: phase must be SEM_APPLY_FULL, _LOCAL or _FINISH");
    SEM_REQUIRE(u_L != w_L, "sem_apply: u and w must not alias");
    cudaStream_t s = (cudaStream_t)stream;
    if (dtype == SEM_F64) {
      SEM_REQUIRE(h->f64.G.ptr, "sem_apply: handle has no FP64 geometry");
      launch_apply<double>(h, h->f64, (const double*)u_L, (double*)w_L, h1, h2,
                           (const double*)h1_field, nullptr, phase, s);
    } else if (dtype == SEM_F32) {
      SEM_REQUIRE(h->f32.G.ptr, "sem_apply: handle has no FP32 geometry");
      launch_apply<float>(h, h->f32, (const float*)u_L, (float*)w_L, (float)h1, (float)h2,
                          (const float*)h1_field, nullptr, phase, s);
    } else {
      throw Error(SEM_ERR_ARG, "sem_apply: dtype must be SEM_F64 or SEM_F32");
    }
  });
}
