// FP64-accurate element operator w_e = (h1 D^T G_e D + h2 B_e) u_e (arXiv
// 2107.01243 §2, Eq. 9) evaluated in double-float arithmetic on the FP32
// pipes (df.cuh).  FP64 in, FP64 out; the geometric factors are stored as
// float pairs (8 bytes per value, the same traffic as FP64).
//
// A persistent CTA of P x P threads walks its elements; thread 0 keeps
// STAGES elements in flight with bulk copies (u_e as doubles, the 6 G pairs,
// B pairs for Helmholtz).  Every contraction is done by "line tasks": a
// thread reads one line of P pairs and produces the P outputs of that line,
// so every D index is a compile-time constant served from the constant bank.
//   phase 0  thread (i,j): u column -> pairs, kept in registers and stored U
//   F-r, F-s thread (j,k) / (i,k): lines of U -> UR, US  (D)
//   G        thread (i,j): F-t on its register column, then per point
//            (WR, WS, WT) = h1 G (UR, US, UT); WR, WS overwrite UR, US
//   B-r, B-s thread (j,k) / (i,k): lines of WR, WS -> CR, CS in place (D^T)
//   B-t      thread (i,j): w = CR + CS + sum_l D_lk WT_l (+ h2 B u) -> double
// Shared arrays use padded rows (P+2 pairs) and planes (stride = 8 mod 16
// pairs) so the line reads are free of bank conflicts at P = 8.
#include "sem_internal.cuh"
#include "tma.cuh"
#include "df.cuh"

namespace sem {

template <int P>
struct DFConst {
  float dh[P * P];   // D[i][l], high parts
  float dl[P * P];   // low parts
  float h1h, h1l, h2h, h2l;
};

template <int P>
struct DFLayout {
  static constexpr int RS = P + 2;                              // row stride (pairs)
  static constexpr int PL0 = P * RS;
  static constexpr int PL = PL0 + ((8 - (PL0 % 16)) + 16) % 16; // plane stride = 8 mod 16
  static constexpr int VOL = P * PL;                            // one padded array (pairs)
  __device__ static constexpr int at(int i, int j, int k) { return k * PL + j * RS + i; }
};

// y_i = sum_l M[i][l] x_l (TRANS: M = D^T), all outputs of one line
template <int P, bool TRANS>
__device__ __forceinline__ void line_df(const DFConst<P>& C, const float (&xh)[P],
                                        const float (&xl)[P], float (&yh)[P], float (&yl)[P]) {
#pragma unroll
  for (int i = 0; i < P; ++i) {
    float S, err;
    tmac0(C.dh[TRANS ? i : i * P], C.dl[TRANS ? i : i * P], xh[0], xl[0], S, err);
#pragma unroll
    for (int l = 1; l < P; ++l) {
      const int idx = TRANS ? l * P + i : i * P + l;
      tmac(C.dh[idx], C.dl[idx], xh[l], xl[l], S, err);
    }
    yh[i] = S;
    yl[i] = err;
  }
}

// sum of three products g_a * v_a
__device__ __forceinline__ void dot3_df(float g0h, float g0l, float g1h, float g1l, float g2h,
                                        float g2l, float v0h, float v0l, float v1h, float v1l,
                                        float v2h, float v2l, float& oh, float& ol) {
  float S, err;
  tmac0(g0h, g0l, v0h, v0l, S, err);
  tmac(g1h, g1l, v1h, v1l, S, err);
  tmac(g2h, g2l, v2h, v2l, S, err);
  oh = S;
  ol = err;
}

template <int P, int STAGES>
__global__ void __launch_bounds__(P * P)
ax_df_kernel(const double* __restrict__ u, double* __restrict__ w, const float2* __restrict__ G,
             const float2* __restrict__ B, DFConst<P> C, int E, const CGState* __restrict__ st,
             int* __restrict__ err, uint64_t timeout_ns) {
  using L = DFLayout<P>;
  constexpr int P2 = P * P, P3 = P2 * P;
  constexpr uint32_t UB = P3 * sizeof(double), GB = 6 * P3 * sizeof(float2),
                     BB = P3 * sizeof(float2);
  if (st && st->done) return;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);
  const bool helm = (C.h2h != 0.0f);
  const bool scale1 = !(C.h1h == 1.0f && C.h1l == 0.0f);
  const uint32_t SB = UB + GB + (helm ? BB : 0);          // stage bytes
  unsigned char* stage0 = smem_raw + 128;
  float2* U = reinterpret_cast<float2*>(stage0 + STAGES * SB);
  float2* UR = U + L::VOL;
  float2* US = UR + L::VOL;
  const int tid = threadIdx.x;
  const int a = tid % P, b = tid / P;     // line / column coordinates

  auto issue = [&](int e, int s) {
    unsigned char* dst = stage0 + s * SB;
    mbar_arrive_expect_tx(&bar[s], SB);
    bulk_g2s(dst, u + (size_t)e * P3, UB, &bar[s]);
    bulk_g2s(dst + UB, G + (size_t)e * 6 * P3, GB, &bar[s]);
    if (helm) bulk_g2s(dst + UB + GB, B + (size_t)e * P3, BB, &bar[s]);
  };
  if (tid == 0) {
#pragma unroll
    for (int s = 0; s < STAGES; ++s) mbar_init(&bar[s], 1);
    mbar_fence_init();
  }
  __syncthreads();
  if (tid == 0) {
#pragma unroll
    for (int s = 0; s < STAGES; ++s) {
      int e = blockIdx.x + s * gridDim.x;
      if (e < E) issue(e, s);
    }
  }

  int n = 0;
  for (int e = blockIdx.x; e < E; e += gridDim.x, ++n) {
    const int s = n % STAGES;
    const bool ok = mbar_wait_bounded(&bar[s], (uint32_t)(n / STAGES) & 1u, err, timeout_ns);
    const double* su = reinterpret_cast<const double*>(stage0 + s * SB);
    const float2* sg = reinterpret_cast<const float2*>(stage0 + s * SB + UB);
    const float2* sb = reinterpret_cast<const float2*>(stage0 + s * SB + UB + GB);
    // phase 0: thread (i=a, j=b) converts its column
    float uch[P], ucl[P];
#pragma unroll
    for (int k = 0; k < P; ++k) {
      d2df(su[k * P2 + tid], uch[k], ucl[k]);
      U[L::at(a, b, k)] = make_float2(uch[k], ucl[k]);
    }
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        for (int m = 0; m < STAGES; ++m) {
          int nn = n + m;
          if (blockIdx.x + nn * gridDim.x < E)
            mbar_wait_bounded(&bar[nn % STAGES], (uint32_t)(nn / STAGES) & 1u, err, timeout_ns);
        }
      }
      return;
    }
    // F-r: line over i at (j=a, k=b);  F-s: line over j at (i=a, k=b)
    {
      float xh[P], xl[P], yh[P], yl[P];
#pragma unroll
      for (int l = 0; l < P; ++l) {
        float2 v = U[L::at(l, a, b)];
        xh[l] = v.x; xl[l] = v.y;
      }
      line_df<P, false>(C, xh, xl, yh, yl);
#pragma unroll
      for (int l = 0; l < P; ++l) UR[L::at(l, a, b)] = make_float2(yh[l], yl[l]);
#pragma unroll
      for (int l = 0; l < P; ++l) {
        float2 v = U[L::at(a, l, b)];
        xh[l] = v.x; xl[l] = v.y;
      }
      line_df<P, false>(C, xh, xl, yh, yl);
#pragma unroll
      for (int l = 0; l < P; ++l) US[L::at(a, l, b)] = make_float2(yh[l], yl[l]);
    }
    __syncthreads();
    // G phase: thread (i=a, j=b); F-t on the register column first
    float wth[P], wtl[P];
    {
      float uth[P], utl[P];
      line_df<P, false>(C, uch, ucl, uth, utl);
#pragma unroll
      for (int k = 0; k < P; ++k) {
        const int q = k * P2 + tid;
        const float2 g11 = sg[q], g22 = sg[P3 + q], g33 = sg[2 * P3 + q];
        const float2 g12 = sg[3 * P3 + q], g13 = sg[4 * P3 + q], g23 = sg[5 * P3 + q];
        const float2 ur = UR[L::at(a, b, k)], us = US[L::at(a, b, k)];
        float rh, rl, sh, sl, th, tl;
        dot3_df(g11.x, g11.y, g12.x, g12.y, g13.x, g13.y, ur.x, ur.y, us.x, us.y, uth[k], utl[k],
                rh, rl);
        dot3_df(g12.x, g12.y, g22.x, g22.y, g23.x, g23.y, ur.x, ur.y, us.x, us.y, uth[k], utl[k],
                sh, sl);
        dot3_df(g13.x, g13.y, g23.x, g23.y, g33.x, g33.y, ur.x, ur.y, us.x, us.y, uth[k], utl[k],
                th, tl);
        if (scale1) {
          dfmul(C.h1h, C.h1l, rh, rl, rh, rl);
          dfmul(C.h1h, C.h1l, sh, sl, sh, sl);
          dfmul(C.h1h, C.h1l, th, tl, th, tl);
        }
        UR[L::at(a, b, k)] = make_float2(rh, rl);
        US[L::at(a, b, k)] = make_float2(sh, sl);
        wth[k] = th;
        wtl[k] = tl;
      }
    }
    float bh[P], bl[P];
#pragma unroll
    for (int k = 0; k < P; ++k) {
      if (helm) {
        const float2 bv = sb[k * P2 + tid];
        dfmul(C.h2h, C.h2l, bv.x, bv.y, bh[k], bl[k]);
      } else {
        bh[k] = 0.0f;
        bl[k] = 0.0f;
      }
    }
    __syncthreads();                          // stage s consumed; WR, WS complete
    if (tid == 0) {
      int en = e + STAGES * gridDim.x;
      if (en < E) {
        fence_proxy_async_smem();
        issue(en, s);
      }
    }
    // B-r: line over i at (j=a, k=b);  B-s: line over j at (i=a, k=b)  (D^T)
    {
      float xh[P], xl[P], yh[P], yl[P];
#pragma unroll
      for (int l = 0; l < P; ++l) {
        float2 v = UR[L::at(l, a, b)];
        xh[l] = v.x; xl[l] = v.y;
      }
      line_df<P, true>(C, xh, xl, yh, yl);
#pragma unroll
      for (int l = 0; l < P; ++l) UR[L::at(l, a, b)] = make_float2(yh[l], yl[l]);
#pragma unroll
      for (int l = 0; l < P; ++l) {
        float2 v = US[L::at(a, l, b)];
        xh[l] = v.x; xl[l] = v.y;
      }
      line_df<P, true>(C, xh, xl, yh, yl);
#pragma unroll
      for (int l = 0; l < P; ++l) US[L::at(a, l, b)] = make_float2(yh[l], yl[l]);
    }
    __syncthreads();
    // B-t: thread (i=a, j=b): w(i,j,k) = CR + CS + sum_l D_lk WT_l (+ h2 B u)
    {
      double* we = w + (size_t)e * P3;
#pragma unroll
      for (int k = 0; k < P; ++k) {
        const float2 cr = UR[L::at(a, b, k)], cs = US[L::at(a, b, k)];
        float S = cr.x, er = cr.y;
        tadd(cs.x, cs.y, S, er);
#pragma unroll
        for (int l = 0; l < P; ++l) tmac(C.dh[l * P + k], C.dl[l * P + k], wth[l], wtl[l], S, er);
        if (helm) tmac(bh[k], bl[k], uch[k], ucl[k], S, er);
        we[k * P2 + tid] = df2d(S, er);
      }
    }
  }
}

// ---------------------------------------------------------------- launch
template <int P>
static DFConst<P> make_consts(const sem_handle* h, double h1, double h2) {
  DFConst<P> c;
  for (int q = 0; q < P * P; ++q) {
    const double d = h->Dh[q];
    const float dh = (float)d;
    c.dh[q] = dh;
    c.dl[q] = (float)(d - (double)dh);
  }
  c.h1h = (float)h1;
  c.h1l = (float)(h1 - (double)c.h1h);
  c.h2h = (float)h2;
  c.h2l = (float)(h2 - (double)c.h2h);
  return c;
}

template <int P, int STAGES>
static size_t df_smem_bytes(bool helm) {
  using L = DFLayout<P>;
  const size_t P3 = (size_t)P * P * P;
  const size_t SB = P3 * 8 + 6 * P3 * 8 + (helm ? P3 * 8 : 0);
  return 128 + STAGES * SB + 3 * (size_t)L::VOL * sizeof(float2);
}

static int df_num_sms() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
      n = kNumSMs;
  }
  return n;
}

template <int P, int STAGES>
static void launch_df_p(const sem_handle* h, const double* u, double* w, double h1, double h2,
                        const CGState* st, cudaStream_t s) {
  const bool helm = (float)h2 != 0.0f;
  const size_t smem = df_smem_bytes<P, STAGES>(helm);
  auto kern = ax_df_kernel<P, STAGES>;
  static bool configured = false;
  static int occ[2] = {0, 0};
  if (!configured) {
    SEM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)df_smem_bytes<P, STAGES>(true)));
    configured = true;
  }
  int& o = occ[helm ? 1 : 0];
  if (!o) {
    SEM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, P * P, smem));
    if (o < 1) o = 1;
  }
  const int E = (int)h->E;
  int grid = (int)std::min<int64_t>(E, (int64_t)o * df_num_sms());
  if (grid < 1) grid = 1;
  kern<<<grid, P * P, smem, s>>>(u, w, h->gdf.ptr, h->bdf.ptr, make_consts<P>(h, h1, h2), E, st,
                                 h->dev_err.ptr, kWaitTimeoutNs);
  SEM_CHECK_LAUNCH();
}

bool df_ax_supported(const sem_handle* h, const void* u, const void* w, const void* h1f) {
  if (h1f != nullptr || !h->gdf.ptr) return false;
  const int P = h->P;
  if (P != 6 && P != 8 && P != 10) return false;
  return ((uintptr_t)u % 16) == 0 && ((uintptr_t)w % 16) == 0;
}

void launch_ax_df(const sem_handle* h, const double* u, double* w, double h1, double h2,
                  const CGState* st, cudaStream_t s) {
  switch (h->P) {
    case 6: launch_df_p<6, 2>(h, u, w, h1, h2, st, s); break;
    case 8: launch_df_p<8, 2>(h, u, w, h1, h2, st, s); break;
    case 10: launch_df_p<10, 1>(h, u, w, h1, h2, st, s); break;
    default: throw Error(SEM_ERR_ARG, "launch_ax_df: unsupported order");
  }
}

}  // namespace sem
