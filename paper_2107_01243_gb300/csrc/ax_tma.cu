// Element operator w_e = (h1 D^T G_e D + h2 B_e) u_e (arXiv 2107.01243 §2,
// Eq. 9) with bulk-copy staging: a persistent CTA of P x P threads walks its
// elements; thread 0 keeps STAGES elements in flight, each one copied into
// shared memory by cp.async.bulk (u_e, the 6 geometric factors, optionally B_e
// and h1_e: contiguous runs of P^3 values) and completed on an mbarrier.  D
// travels in the kernel parameters (constant bank); each thread keeps the
// D rows and columns of its (i, j) in registers.
//
// Per element (thread (i, j) owns the k-column):
//   u column -> registers, transposed plane copy -> sT;  sync
//   r, s, t derivatives (rows of u, rows of sT, the register column),
//   times G -> swr, swsT (transposed), wt in registers;  sync; stage released
//   w = D^T-contractions of swr rows, swsT rows and the wt column (+ h2 B u)
// Needs P^3 * sizeof(T) % 16 == 0 (even P) and 16-byte aligned vectors.
#include "sem_internal.cuh"
#include "tma.cuh"
#include "ax_tile.cuh"
#include "reduce.cuh"
#include "cg_state.cuh"

namespace sem {

// FUSE (K = 1 only): the CTA walks segments of kFuseSeg consecutive elements
// and writes the fused output of each (FusedStore: mask, x-neighbour pairs of
// the segment summed in the CTA), for the assembled operator of apply.cu.
template <int P, class T, int STAGES, int K, bool FUSE>
__global__ void __launch_bounds__(K * P * P)
ax_tma_kernel(const T* __restrict__ u, T* __restrict__ w, const T* __restrict__ G,
              const T* __restrict__ B, const T* __restrict__ h1f, T h1, T h2, DMat<P, T> D,
              int E, const CGState* __restrict__ st, int* __restrict__ err, uint64_t timeout_ns,
              uint32_t starve_bytes, FuseBox fb, CGState* __restrict__ pwst,
              double* __restrict__ partials) {
  static_assert(!FUSE || K == 1, "the fused output needs one element per CTA");
  constexpr int P2 = P * P, P3 = P2 * P;
  constexpr uint32_t FB = P3 * sizeof(T);          // bytes of one field of one element
  if (st && st->done) return;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);
  T* stage0 = reinterpret_cast<T*>(smem_raw + 128);
  const bool helm = h2 != T(0);
  const bool var = h1f != nullptr;
  const int nf = 7 + (helm ? 1 : 0) + (var ? 1 : 0);
  const int SE = nf * K * P3;                          // stage size in values
  const int tid = threadIdx.x;
  const int slot = tid / P2;                           // element slot of this thread
  T* sT = stage0 + STAGES * SE + slot * P3;
  T* swr = stage0 + STAGES * SE + K * P3 + slot * P3;
  T* swsT = stage0 + STAGES * SE + 2 * K * P3 + slot * P3;
  const int nitems = (E + K - 1) / K;
  const ItemSeq<FUSE> seq{nitems};     // this CTA's items in order
  BoxWalk bw;                          // thread 0 (FUSE)
  __shared__ unsigned s_fl;            // FusedStore flags of the current element
  auto Dm = [&](int r, int c) { return D.d[r * P + c]; };
  TileThread<P, T> t;
  t.init(tid - slot * P2, Dm);

  // item it = elements [it K, it K + cnt): one copy per field
  auto issue = [&](int it, int s) {
    const int e0 = it * K;
    const int cnt = min(K, E - e0);
    T* dst = stage0 + s * SE;
    const uint64_t pol = l2_policy_evict_first();   // G, B and h1 are read once
    mbar_arrive_expect_tx(&bar[s], nf * cnt * FB + starve_bytes);
    bulk_g2s(dst, u + (size_t)e0 * P3, cnt * FB, &bar[s]);
    bulk_g2s_hint(dst + K * P3, G + (size_t)e0 * 6 * P3, 6 * cnt * FB, &bar[s], pol);
    int off = 7 * K * P3;
    if (helm) {
      bulk_g2s_hint(dst + off, B + (size_t)e0 * P3, cnt * FB, &bar[s], pol);
      off += K * P3;
    }
    if (var) bulk_g2s_hint(dst + off, h1f + (size_t)e0 * P3, cnt * FB, &bar[s], pol);
  };

  if (tid == 0) {
#pragma unroll
    for (int s = 0; s < STAGES; ++s) mbar_init(&bar[s], 1);
    mbar_fence_init();
  }
  __syncthreads();
  int ahead = seq.first(), issued = 0;     // thread 0: next item to prefetch, copies issued
  if (tid == 0) {
#pragma unroll
    for (int s = 0; s < STAGES; ++s) {
      if (ahead < nitems) {
        issue(ahead, s);
        ahead = seq.next(ahead);
        ++issued;
      }
    }
  }

  // FUSE with pwst: <p, H p> = sum over local points of p (H_L p), which
  // equals the unique-dof product of p with the assembled, masked H p (p is
  // continuous and zero on Dirichlet points), accumulated here per thread
  float pw_s = 0.0f, pw_c = 0.0f;      // Kahan-compensated
  int n = 0;
  for (int it = seq.first(); it < nitems; it = seq.next(it), ++n) {
    const int s = n % STAGES;
    const uint32_t par = (uint32_t)(n / STAGES) & 1u;
    const bool ok = mbar_wait_bounded(&bar[s], par, err, timeout_ns);
    const int e0 = it * K;
    const bool act = slot < min(K, E - e0);
    const T* su = stage0 + s * SE + slot * P3;
    const T* sg = stage0 + s * SE + K * P3 + slot * 6 * P3;
    const T* sb = helm ? stage0 + s * SE + 7 * K * P3 + slot * P3 : nullptr;
    const T* sh = var ? stage0 + s * SE + (helm ? 8 : 7) * K * P3 + slot * P3 : nullptr;
    T uc[P], bk[P], ck[P], wt[P];
    if (act) tile_load<P, T>(t, su, sb, sh, h1, sT, uc, bk, ck);
    if (__syncthreads_or(!ok)) {
      // a copy never completed: wait (bounded) for what is in flight, then leave
      if (tid == 0) {
        for (int nn = n; nn < issued; ++nn)
          mbar_wait_bounded(&bar[nn % STAGES], (uint32_t)(nn / STAGES) & 1u, err, timeout_ns);
      }
      break;                           // the reduction below still counts this CTA
    }
    if (FUSE && tid == 0) {            // box position of e0, read back in the output phase
      if (e0 % kFuseSeg == 0) bw.start(e0, fb); else bw.step(fb);
      s_fl = fused_flags(e0, bw, fb);
    }
    if (act) tile_forward<P, T>(t, su, sT, sg, uc, ck, swr, swsT, wt, Dm);
    __syncthreads();
    if (tid == 0 && ahead < nitems) {           // stage s consumed
      fence_proxy_async_smem();
      issue(ahead, s);
      ahead = seq.next(ahead);
      ++issued;
    }
    if (!act) continue;
    if constexpr (FUSE) {
      FusedStore<P, T> fs;
      fs.we = w + (size_t)e0 * P3;
      fs.fl = s_fl;
      if (pwst) {
        tile_backward<P, T>(t, swr, swsT, wt, uc, bk, h2, helm, Dm, [&](int k, T v) {
          const float y = __fsub_rn(__fmul_rn((float)uc[k], (float)v), pw_c);
          const float tt = __fadd_rn(pw_s, y);
          pw_c = __fsub_rn(__fsub_rn(tt, pw_s), y);
          pw_s = tt;
          fs.store(t.i, t.j, k, v);
        });
      } else {
        tile_backward<P, T>(t, swr, swsT, wt, uc, bk, h2, helm, Dm,
                            [&](int k, T v) { fs.store(t.i, t.j, k, v); });
      }
    } else {
      T* we = w + (size_t)(e0 + slot) * P3;
      tile_backward<P, T>(t, swr, swsT, wt, uc, bk, h2, helm, Dm,
                          [&](int k, T v) { we[k * P2 + t.lt] = v; });
    }
  }
  if constexpr (FUSE && (K * P * P) % 32 == 0) {
    if (pwst) {
      double v[1] = {(double)pw_s - (double)pw_c};
      double tot[1];
      if (grid_sum<1>(v, partials, &pwst->counter, tot) && threadIdx.x == 0) {
        st_after_pw(pwst, tot[0]);
      }
    }
  }
}

// ---------------------------------------------------------------- launch
template <int P, class T, int STAGES, int K>
static size_t tma_smem_bytes(int nf) {
  return 128 + (size_t)(STAGES * nf + 3) * K * P * P * P * sizeof(T);
}

// returns the grid it launched (the fused operator's later passes need it)
template <int P, class T, int STAGES, int K, bool FUSE = false>
static int launch_tma_p(const sem_handle* h, const OpData<T>& op, const T* u, T* w, T h1, T h2,
                        const T* h1f, const CGState* st, int* err, uint64_t timeout_ns,
                        uint32_t starve, cudaStream_t s, CGState* pwst = nullptr) {
  const int nf = 7 + (h2 != T(0) ? 1 : 0) + (h1f ? 1 : 0);
  const size_t smem = tma_smem_bytes<P, T, STAGES, K>(nf);
  auto kern = ax_tma_kernel<P, T, STAGES, K, FUSE>;
  static int configured_smem = 0;
  static int occ[3] = {0, 0, 0};
  const int maxsmem = (int)tma_smem_bytes<P, T, STAGES, K>(9);
  if (configured_smem < maxsmem) {
    SEM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, maxsmem));
    configured_smem = maxsmem;
  }
  int& o = occ[nf - 7];
  if (!o) {
    SEM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, K * P * P, smem));
    if (o < 1) o = 1;
  }
  DMat<P, T> D;
  for (int a = 0; a < P * P; ++a) D.d[a] = (T)h->Dh[a];
  const int E = (int)h->E;
  const int nitems = (E + K - 1) / K;
  int grid = std::min<int64_t>(nitems, (int64_t)o * sem_num_sms());
  if (grid < 1) grid = 1;
  if (pwst) grid = std::min(grid, kFusedPartials);
  const FuseBox fb{h->nelx, h->nely, h->nelz, h->faces};
  kern<<<grid, K * P * P, smem, s>>>(u, w, op.G.ptr, op.B.ptr, h1f, h1, h2, D, E, st, err,
                                     timeout_ns, starve, fb, pwst,
                                     h->partials.ptr + 4 * kRedBlocks);
  SEM_CHECK_LAUNCH();
  return grid;
}

template <class T>
bool tma_ax_supported(const sem_handle* h, const void* u, const void* w, const void* h1f) {
  const int P = h->P;
  if (P != 2 && P != 4 && P != 6 && P != 8 && P != 10) return false;
  auto al = [](const void* p) { return p == nullptr || ((uintptr_t)p % 16) == 0; };
  return al(u) && al(w) && al(h1f);
}

// (stages, elements per CTA) variants the autotuner chooses from
constexpr int kTmaVariantStages[5] = {1, 2, 3, 1, 2};
template <int P, class T>
static void launch_tma_variant(int variant, const sem_handle* h, const OpData<T>& op, const T* u,
                               T* w, T h1, T h2, const T* h1f, const CGState* st, int* err,
                               uint64_t timeout_ns, uint32_t starve, cudaStream_t s) {
  switch (variant) {
    case 0: launch_tma_p<P, T, 1, 1>(h, op, u, w, h1, h2, h1f, st, err, timeout_ns, starve, s); break;
    case 1: launch_tma_p<P, T, 2, 1>(h, op, u, w, h1, h2, h1f, st, err, timeout_ns, starve, s); break;
    case 2: launch_tma_p<P, T, 3, 1>(h, op, u, w, h1, h2, h1f, st, err, timeout_ns, starve, s); break;
    case 3: launch_tma_p<P, T, 1, 2>(h, op, u, w, h1, h2, h1f, st, err, timeout_ns, starve, s); break;
    default: launch_tma_p<P, T, 2, 2>(h, op, u, w, h1, h2, h1f, st, err, timeout_ns, starve, s); break;
  }
}

template <class T>
void launch_ax_tma(const sem_handle* h, const OpData<T>& op, const T* u, T* w, T h1, T h2,
                   const T* h1f, const CGState* st, int* err, uint64_t timeout_ns,
                   uint32_t starve, cudaStream_t s) {
  const int v = h->tune.ax32_variant;
  switch (h->P) {
    case 2: launch_tma_variant<2, T>(v, h, op, u, w, h1, h2, h1f, st, err, timeout_ns, starve, s); break;
    case 4: launch_tma_variant<4, T>(v, h, op, u, w, h1, h2, h1f, st, err, timeout_ns, starve, s); break;
    case 6: launch_tma_variant<6, T>(v, h, op, u, w, h1, h2, h1f, st, err, timeout_ns, starve, s); break;
    case 8: launch_tma_variant<8, T>(v, h, op, u, w, h1, h2, h1f, st, err, timeout_ns, starve, s); break;
    case 10: launch_tma_variant<10, T>(v, h, op, u, w, h1, h2, h1f, st, err, timeout_ns, starve, s); break;
    default: throw Error(SEM_ERR_ARG, "launch_ax_tma: unsupported order");
  }
}

// The fused-output FP32 kernel (one element per CTA, the tuned stage count);
// faces = the Dirichlet faces to zero (0: none).  Returns the grid.
template <int P>
static int launch_tma_fused_p(const sem_handle* h, const float* u, float* w, float h1, float h2,
                              const float* h1f, const CGState* st, CGState* pwst,
                              cudaStream_t s) {
  const int stages = kTmaVariantStages[h->tune.ax32_variant];
  if (stages == 1)
    return launch_tma_p<P, float, 1, 1, true>(h, h->f32, u, w, h1, h2, h1f, st,
                                              h->dev_err.ptr, kWaitTimeoutNs, 0, s, pwst);
  if (stages == 2)
    return launch_tma_p<P, float, 2, 1, true>(h, h->f32, u, w, h1, h2, h1f, st,
                                              h->dev_err.ptr, kWaitTimeoutNs, 0, s, pwst);
  return launch_tma_p<P, float, 3, 1, true>(h, h->f32, u, w, h1, h2, h1f, st, h->dev_err.ptr,
                                            kWaitTimeoutNs, 0, s, pwst);
}

// pwst (may be NULL): state that receives <p, H p> and alpha, for orders whose
// CTAs are whole warps (P = 8); returns whether it was computed
bool launch_ax_tma_fused(const sem_handle* h, const float* u, float* w, float h1, float h2,
                         const float* h1f, const CGState* st, CGState* pwst, cudaStream_t s) {
  switch (h->P) {
    case 2: launch_tma_fused_p<2>(h, u, w, h1, h2, h1f, st, nullptr, s); return false;
    case 4: launch_tma_fused_p<4>(h, u, w, h1, h2, h1f, st, nullptr, s); return false;
    case 6: launch_tma_fused_p<6>(h, u, w, h1, h2, h1f, st, nullptr, s); return false;
    case 8: launch_tma_fused_p<8>(h, u, w, h1, h2, h1f, st, pwst, s); return pwst != nullptr;
    case 10: launch_tma_fused_p<10>(h, u, w, h1, h2, h1f, st, nullptr, s); return false;
    default: throw Error(SEM_ERR_ARG, "launch_ax_tma_fused: unsupported order");
  }
}

template bool tma_ax_supported<float>(const sem_handle*, const void*, const void*, const void*);
template void launch_ax_tma<float>(const sem_handle*, const OpData<float>&, const float*, float*,
                                   float, float, const float*, const CGState*, int*, uint64_t,
                                   uint32_t, cudaStream_t);

}  // namespace sem

using namespace sem;

extern "C" sem_status sem_selftest_timeout(sem_handle* h, double timeout_ms, void* stream) {
  sem_status result = SEM_OK;
  sem_status st = guarded("sem_selftest_timeout", [&] {
    SEM_REQUIRE(h, "sem_selftest_timeout: null handle");
    SEM_REQUIRE(timeout_ms > 0 && timeout_ms <= 2000, "sem_selftest_timeout: timeout in (0, 2000] ms");
    SEM_REQUIRE(h->f32.G.ptr, "sem_selftest_timeout: needs FP32 geometry");
    SEM_REQUIRE(tma_ax_supported<float>(h, nullptr, nullptr, nullptr),
                "sem_selftest_timeout: needs an even number of points per direction");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = h->nL;
    DevBuf<float> u, w;
    u.alloc(n);
    w.alloc(n);
    SEM_CUDA(cudaMemsetAsync(u.ptr, 0, n * sizeof(float), s));
    SEM_CUDA(cudaMemsetAsync(h->dev_err.ptr, 0, sizeof(int), s));
    // 16 bytes more than any copy delivers: the first stage barrier never completes
    launch_ax_tma<float>(h, h->f32, u.ptr, w.ptr, 1.0f, 0.0f, nullptr, nullptr, h->dev_err.ptr,
                         (uint64_t)(timeout_ms * 1e6), 16u, s);
    int herr = 0;
    SEM_CUDA(cudaMemcpyAsync(&herr, h->dev_err.ptr, sizeof(int), cudaMemcpyDeviceToHost, s));
    SEM_CUDA(cudaStreamSynchronize(s));
    SEM_CUDA(cudaMemsetAsync(h->dev_err.ptr, 0, sizeof(int), s));
    SEM_CUDA(cudaStreamSynchronize(s));
    result = (sem_status)herr;
  });
  return st != SEM_OK ? st : result;
}
