// Matrix-free element operator w_e = (h1 D^T G_e D + h2 B_e) u_e
// (arXiv 2107.01243 §2, Eq. 9; the ax_t compute of Listing 1).
//
// Layout: one CTA works on EPB elements at a time; inside an element a
// P x P thread plane owns the k-columns (i, j, 0..P-1).  The column of u
// stays in registers (t-derivative and its transpose in registers), the
// element is staged in shared memory for the r- and s-derivatives, rows are
// padded to P+1 to spread the banks.  The 6 geometric factors of an element
// are stored [6][P^3] so each factor streams coalesced along (i, j).
#include <type_traits>

#include "sem_internal.cuh"

namespace sem {

template <int P, class T>
struct AxCfg {
  static constexpr int P2 = P * P;
  static constexpr int PP = P + 1;
  static constexpr int VOL = P * P * PP;
  static constexpr int smem_per_el = 2 * VOL * (int)sizeof(T);
  static constexpr int by_threads = (256 / P2) < 1 ? 1 : (256 / P2);
  static constexpr int by_smem = (40 * 1024) / smem_per_el < 1 ? 1 : (40 * 1024) / smem_per_el;
  static constexpr int EPB0 = by_threads < by_smem ? by_threads : by_smem;
  static constexpr int EPB = EPB0 > 32 ? 32 : EPB0;
};

template <int P, class T>
__global__ void __launch_bounds__(AxCfg<P, T>::P2 * AxCfg<P, T>::EPB)
ax_kernel(const T* __restrict__ u, T* __restrict__ w, const T* __restrict__ G,
          const T* __restrict__ B, const T* __restrict__ h1f, T h1, T h2,
          const T* __restrict__ Dg, int E, const CGState* __restrict__ st) {
  using C = AxCfg<P, T>;
  constexpr int P2 = C::P2, P3 = P2 * P, PP = C::PP, PL = P * PP, EPB = C::EPB;
  if (st && st->done) return;
  __shared__ T sD[P][PP];    // sD[a][b]  = D[a][b]
  __shared__ T sDt[P][PP];   // sDt[a][b] = D[b][a]
  __shared__ T s1[EPB][C::VOL];
  __shared__ T s2[EPB][C::VOL];
  const int tid = threadIdx.x;
  const int el = threadIdx.y;
  const int i = tid % P, j = tid / P;
  for (int q = tid + el * P2; q < P2; q += P2 * EPB) {
    T d = Dg[q];
    sD[q / P][q % P] = d;
    sDt[q % P][q / P] = d;
  }
  __syncthreads();
  const bool helm = h2 != T(0);
  for (int e0 = blockIdx.x * EPB; e0 < E; e0 += gridDim.x * EPB) {
    const int e = e0 + el;
    const bool act = e < E;
    const size_t base = (size_t)(act ? e : 0) * P3 + tid;
    T uc[P];
#pragma unroll
    for (int k = 0; k < P; ++k) {
      uc[k] = act ? u[base + k * P2] : T(0);
      s1[el][k * PL + j * PP + i] = uc[k];
    }
    __syncthreads();
    T rr[P], rs[P], rt[P];
    const T* g = G + (size_t)(act ? e : 0) * 6 * P3 + tid;
#pragma unroll
    for (int k = 0; k < P; ++k) {
      T ur = T(0), us = T(0), ut = T(0);
#pragma unroll
      for (int l = 0; l < P; ++l) {
        ur += sD[i][l] * s1[el][k * PL + j * PP + l];
        us += sD[j][l] * s1[el][k * PL + l * PP + i];
        ut += sD[k][l] * uc[l];
      }
      T g11 = g[0 * P3 + k * P2], g22 = g[1 * P3 + k * P2], g33 = g[2 * P3 + k * P2];
      T g12 = g[3 * P3 + k * P2], g13 = g[4 * P3 + k * P2], g23 = g[5 * P3 + k * P2];
      T c = h1f ? h1f[base + k * P2] : h1;
      rr[k] = c * (g11 * ur + g12 * us + g13 * ut);
      rs[k] = c * (g12 * ur + g22 * us + g23 * ut);
      rt[k] = c * (g13 * ur + g23 * us + g33 * ut);
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < P; ++k) {
      s1[el][k * PL + j * PP + i] = rr[k];
      s2[el][k * PL + j * PP + i] = rs[k];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < P; ++k) {
      T acc = T(0);
#pragma unroll
      for (int l = 0; l < P; ++l) {
        acc += sDt[i][l] * s1[el][k * PL + j * PP + l];
        acc += sDt[j][l] * s2[el][k * PL + l * PP + i];
        acc += sDt[k][l] * rt[l];
      }
      if (helm) acc += h2 * B[base + k * P2] * uc[k];
      if (act) w[base + k * P2] = acc;
    }
    __syncthreads();
  }
}

// ------------------------------------------------- IEEE FP64, even P
// The same operator in IEEE FP64 arithmetic for even P, with the even-odd
// split of D: D is centro-antisymmetric on GLL nodes (D_{N-i,N-l} = -D_il),
// so with e_l = x_l + x_{N-l} and o_l = x_l - x_{N-l} (l < P/2) a line's
// outputs come in pairs y_i = A_i.o + S_i.e, y_{N-i} = A_i.o - S_i.e, where
// A_il = (M_il - M_{i,N-l}) / 2 and S_il = (M_il + M_{i,N-l}) / 2 (M = D or
// D^T): 2P^2 / 4 + 2P operations per line instead of P^2, about 20% fewer
// FP64 operations per point at P = 8 for a kernel that GB300's FP64 pipe
// bounds.  One element per CTA of 3 P^2 threads: group g runs the lines of
// direction g (forward derivatives, then transposed contractions, in
// place), and the geometric factors are applied point by point in between.
// Used at P = 8 and 10 (see launch_ax).

// even-odd halves of D in double: [P][trans][0: A, 1: S][i * (P/2) + l]
constexpr int kEoH = kMaxP / 2 + 1;
__constant__ double c_eo[kMaxP + 1][2][2][kEoH * kEoH];

// shared-memory position of (i, j, k) for 8-byte values: P = 8 uses unpadded
// 64-value planes with rows and columns XOR-swizzled by the plane parity (the
// lines of all three directions and the point phases are free of bank
// conflicts); other orders pad rows to P + 2 and planes to 8 mod 16 values
template <int P>
struct EoLayout {
  static constexpr int RS = P + 2;
  static constexpr int PL0 = P * RS;
  static constexpr int PL = PL0 + ((8 - (PL0 % 16)) + 16) % 16;
  static constexpr int VOL = P * PL;
  __device__ static int at(int i, int j, int k) { return k * PL + j * RS + i; }
};
template <>
struct EoLayout<8> {
  static constexpr int PL = 64;
  static constexpr int VOL = 8 * PL;
  __device__ static int at(int i, int j, int k) {
    return k * PL + 8 * (j ^ (k & 1)) + (i ^ (((j >> 1) + 4 * (k & 1)) & 7));
  }
};

// tab: the even-odd halves of M in shared memory, [0: A, 1: S][i * (P/2) + l]
// (read at every use: the compiler would otherwise keep all of them in
// registers across the element loop and halve the CTAs per SM)
template <int P>
__device__ __forceinline__ void eo_line(const double* in, double* out, const int (&off)[P],
                                        const double* tab) {
  constexpr int H = P / 2, N = P - 1;
  double x[P];
#pragma unroll
  for (int l = 0; l < P; ++l) x[l] = in[off[l]];
  double e[H], o[H];
#pragma unroll
  for (int l = 0; l < H; ++l) {
    e[l] = x[l] + x[N - l];
    o[l] = x[l] - x[N - l];
  }
#pragma unroll
  for (int i = 0; i < H; ++i) {
    double a = tab[i * H] * o[0];
    double s = tab[H * H + i * H] * e[0];
#pragma unroll
    for (int l = 1; l < H; ++l) {
      a = fma(tab[i * H + l], o[l], a);
      s = fma(tab[H * H + i * H + l], e[l], s);
    }
    out[off[i]] = a + s;
    out[off[N - i]] = a - s;
  }
}

template <int P>
__global__ void __launch_bounds__(3 * P * P)
ax_eo_kernel(const double* __restrict__ u, double* __restrict__ w, const double* __restrict__ G,
             const double* __restrict__ B, const double* __restrict__ h1f, double h1, double h2,
             int E, const CGState* __restrict__ st) {
  using L = EoLayout<P>;
  constexpr int P2 = P * P, P3 = P2 * P, NT = 3 * P2, NQ = (P3 + NT - 1) / NT;
  if (st && st->done) return;
  constexpr int H = P / 2;
  __shared__ double sU[L::VOL];
  __shared__ double sR[3][L::VOL];
  __shared__ double sTab[2][2 * H * H];        // [D, D^T][A, S][i * H + l]
  const int tid = threadIdx.x;
  for (int q = tid; q < 4 * H * H; q += NT)
    sTab[q / (2 * H * H)][q % (2 * H * H)] =
        c_eo[P][q / (2 * H * H)][(q / (H * H)) % 2][q % (H * H)];
  const int g = tid / P2, lam = tid % P2, c1 = lam % P, c2 = lam / P;
  int loff[P];
#pragma unroll
  for (int l = 0; l < P; ++l)
    loff[l] = g == 0 ? L::at(l, c1, c2) : (g == 1 ? L::at(c1, l, c2) : L::at(c1, c2, l));
  int qoff[NQ];
#pragma unroll
  for (int m = 0; m < NQ; ++m) {
    const int q = tid + m * NT;
    qoff[m] = q < P3 ? L::at(q % P, (q / P) % P, q / P2) : 0;
  }
  double* myR = sR[g];
  const bool helm = h2 != 0.0;
  for (int e = blockIdx.x; e < E; e += gridDim.x) {
    const size_t base = (size_t)e * P3;
#pragma unroll
    for (int m = 0; m < NQ; ++m) {
      const int q = tid + m * NT;
      if (q < P3) sU[qoff[m]] = u[base + q];
    }
    __syncthreads();
    eo_line<P>(sU, myR, loff, sTab[0]);          // forward derivatives along g
    __syncthreads();
    const double* ge = G + (size_t)e * 6 * P3;
#pragma unroll
    for (int m = 0; m < NQ; ++m) {
      const int q = tid + m * NT;
      if (q >= P3) break;
      const int at = qoff[m];
      const double ur = sR[0][at], us = sR[1][at], ut = sR[2][at];
      const double g11 = ge[q], g22 = ge[P3 + q], g33 = ge[2 * P3 + q];
      const double g12 = ge[3 * P3 + q], g13 = ge[4 * P3 + q], g23 = ge[5 * P3 + q];
      double wr = fma(g13, ut, fma(g12, us, g11 * ur));
      double ws = fma(g23, ut, fma(g22, us, g12 * ur));
      double wt = fma(g33, ut, fma(g23, us, g13 * ur));
      const double c = h1f ? h1f[base + q] : h1;
      if (h1f || c != 1.0) {
        wr *= c;
        ws *= c;
        wt *= c;
      }
      sR[0][at] = wr;
      sR[1][at] = ws;
      sR[2][at] = wt;
    }
    __syncthreads();
    eo_line<P>(myR, myR, loff, sTab[1]);         // transposed contractions, in place
    __syncthreads();
#pragma unroll
    for (int m = 0; m < NQ; ++m) {
      const int q = tid + m * NT;
      if (q >= P3) break;
      const int at = qoff[m];
      double acc = (sR[0][at] + sR[1][at]) + sR[2][at];
      if (helm) acc = fma(h2 * B[base + q], sU[at], acc);
      w[base + q] = acc;
    }
    // the next element's first phase rewrites sU (read above for Helmholtz)
    // and its forward phase sR (read above): all threads finish here first
    __syncthreads();
  }
}

// copies the even-odd halves of D for this order into constant memory (once
// per process: the library drives one device)
static void eo_upload_d(const sem_handle* h) {
  static bool done[kMaxP + 1] = {};
  const int P = h->P, N = P - 1, H = P / 2;
  if (done[P]) return;
  double eo[2][2][kEoH * kEoH] = {};
  for (int t = 0; t < 2; ++t) {
    auto M = [&](int i, int l) { return t ? h->Dh[l * P + i] : h->Dh[i * P + l]; };
    for (int i = 0; i < H; ++i)
      for (int l = 0; l < H; ++l) {
        eo[t][0][i * H + l] = 0.5 * (M(i, l) - M(i, N - l));
        eo[t][1][i * H + l] = 0.5 * (M(i, l) + M(i, N - l));
      }
  }
  SEM_CUDA(cudaMemcpyToSymbol(c_eo, eo, sizeof(eo), (size_t)P * sizeof(eo)));
  // a copy from pageable memory may still be in flight when the call returns
  // and only the legacy stream is ordered after it: wait once
  SEM_CUDA(cudaDeviceSynchronize());
  done[P] = true;
}

template <int P>
static int eo_occupancy() {
  static int occ = 0;
  if (!occ) {
    SEM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, ax_eo_kernel<P>, 3 * P * P, 0));
    if (occ < 1) occ = 1;
  }
  return occ;
}

// the once-per-process setup of the IEEE FP64 even-order kernel (constant
// tables, occupancy), run by sem_setup outside any stream capture
void eo_prepare(const sem_handle* h) {
  switch (h->P) {
    case 8: eo_occupancy<8>(); break;
    case 10: eo_occupancy<10>(); break;
    default: return;
  }
  eo_upload_d(h);
}

template <int P>
static void launch_eo_p(const sem_handle* h, const OpData<double>& op, const double* u, double* w,
                        double h1, double h2, const double* h1f, const CGState* st,
                        cudaStream_t s) {
  eo_upload_d(h);
  const int E = (int)h->E;
  int grid = (int)std::min<int64_t>(E, (int64_t)eo_occupancy<P>() * sem_num_sms());
  if (grid < 1) grid = 1;
  ax_eo_kernel<P><<<grid, 3 * P * P, 0, s>>>(u, w, op.G.ptr, op.B.ptr, h1f, h1, h2, E, st);
  SEM_CHECK_LAUNCH();
}

// diag(H^e) at every local point: the rr, ss, tt terms run along the line
// through the point, the mixed terms only see the point (D_ii D_jj ...).
template <class T>
__global__ void local_diag_kernel(int P, int64_t nL, const T* __restrict__ G,
                                  const T* __restrict__ B, const T* __restrict__ h1f, T h1,
                                  T h2, const T* __restrict__ Dg, T* __restrict__ d) {
  const int P2 = P * P, P3 = P2 * P;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nL;
       q += (int64_t)gridDim.x * blockDim.x) {
    int64_t e = q / P3;
    int r = (int)(q - e * P3);
    int i = r % P, j = (r / P) % P, k = r / P2;
    const T* g = G + e * 6 * P3;
    const T* c = h1f ? h1f + e * P3 : nullptr;
    auto cf = [&](int idx) { return c ? c[idx] : h1; };
    T acc = T(0);
    for (int l = 0; l < P; ++l) {
      int a = k * P2 + j * P + l, b = k * P2 + l * P + i, t = l * P2 + j * P + i;
      T dli = Dg[l * P + i], dlj = Dg[l * P + j], dlk = Dg[l * P + k];
      acc += dli * dli * cf(a) * g[0 * P3 + a];
      acc += dlj * dlj * cf(b) * g[1 * P3 + b];
      acc += dlk * dlk * cf(t) * g[2 * P3 + t];
    }
    T dii = Dg[i * P + i], djj = Dg[j * P + j], dkk = Dg[k * P + k];
    T cr = cf(r);
    acc += T(2) * cr * (dii * djj * g[3 * P3 + r] + dii * dkk * g[4 * P3 + r] +
                        djj * dkk * g[5 * P3 + r]);
    if (h2 != T(0)) acc += h2 * B[q];
    d[q] = acc;
  }
}

template <int P, class T>
static void launch_ax_p(const sem_handle* h, const OpData<T>& op, const T* u, T* w, T h1, T h2,
                        const T* h1f, const CGState* st, cudaStream_t s) {
  using C = AxCfg<P, T>;
  const int E = (int)h->E;
  int blocks = (E + C::EPB - 1) / C::EPB;
  dim3 block(C::P2, C::EPB);
  ax_kernel<P, T><<<blocks, block, 0, s>>>(u, w, op.G.ptr, op.B.ptr, h1f, h1, h2, op.D.ptr, E,
                                           st);
  SEM_CHECK_LAUNCH();
}

template <class T>
void launch_ax(const sem_handle* h, const OpData<T>& op, const T* u, T* w, T h1, T h2,
               const T* h1f, const CGState* st, cudaStream_t s) {
  if constexpr (std::is_same<T, float>::value) {
    if (!h->tune.ax32_ldg && tma_ax_supported<float>(h, u, w, h1f)) {
      launch_ax_tma<float>(h, op, u, w, h1, h2, h1f, st, h->dev_err.ptr, kWaitTimeoutNs, 0u, s);
      return;
    }
  } else {
    if (h->f64_kernel != SEM_F64_KERNEL_NATIVE && df_ax_supported(h, u, w, h1f)) {
      launch_ax_df(h, u, w, h1, h2, st, s);
      return;
    }
    if (h->f64_kernel == SEM_F64_KERNEL_DOUBLEFLOAT)
      throw Error(SEM_ERR_STATE, "double-float Ax needs N in {5, 7, 9}, constant h1 and "
                                 "16-byte aligned vectors");
    // IEEE FP64: the even-odd kernel at P = 8 and 10 (measured on 32^3-size
    // meshes: 2.6% and 17% faster than the column kernel below; at P = 6 its
    // 108-thread CTAs idle a fifth of their lanes and it was 18% slower)
    switch (h->P) {
      case 8: launch_eo_p<8>(h, op, u, w, h1, h2, h1f, st, s); return;
      case 10: launch_eo_p<10>(h, op, u, w, h1, h2, h1f, st, s); return;
      default: break;
    }
  }
  switch (h->P) {
    case 2: launch_ax_p<2, T>(h, op, u, w, h1, h2, h1f, st, s); break;
    case 3: launch_ax_p<3, T>(h, op, u, w, h1, h2, h1f, st, s); break;
    case 4: launch_ax_p<4, T>(h, op, u, w, h1, h2, h1f, st, s); break;
    case 5: launch_ax_p<5, T>(h, op, u, w, h1, h2, h1f, st, s); break;
    case 6: launch_ax_p<6, T>(h, op, u, w, h1, h2, h1f, st, s); break;
    case 7: launch_ax_p<7, T>(h, op, u, w, h1, h2, h1f, st, s); break;
    case 8: launch_ax_p<8, T>(h, op, u, w, h1, h2, h1f, st, s); break;
    case 9: launch_ax_p<9, T>(h, op, u, w, h1, h2, h1f, st, s); break;
    case 10: launch_ax_p<10, T>(h, op, u, w, h1, h2, h1f, st, s); break;
    case 11: launch_ax_p<11, T>(h, op, u, w, h1, h2, h1f, st, s); break;
    default: throw Error(SEM_ERR_ARG, "launch_ax: unsupported order");
  }
}

template <class T>
void launch_local_diag(const sem_handle* h, const OpData<T>& op, T* d, T h1, T h2, const T* h1f,
                       cudaStream_t s) {
  int64_t nL = h->nL;
  int blocks = (int)std::min<int64_t>((nL + 255) / 256, 16 * sem_num_sms());
  local_diag_kernel<T><<<blocks, 256, 0, s>>>(h->P, nL, op.G.ptr, op.B.ptr, h1f, h1, h2,
                                              op.D.ptr, d);
  SEM_CHECK_LAUNCH();
}

template void launch_ax<double>(const sem_handle*, const OpData<double>&, const double*, double*,
                                double, double, const double*, const CGState*, cudaStream_t);
template void launch_ax<float>(const sem_handle*, const OpData<float>&, const float*, float*,
                               float, float, const float*, const CGState*, cudaStream_t);
template void launch_local_diag<double>(const sem_handle*, const OpData<double>&, double*, double,
                                        double, const double*, cudaStream_t);
template void launch_local_diag<float>(const sem_handle*, const OpData<float>&, float*, float,
                                       float, const float*, cudaStream_t);

}  // namespace sem

using namespace sem;

extern "C" sem_status sem_ax(sem_handle* h, const void* u_L, void* w_L, double h1, double h2,
                             const void* h1_field, int dtype, void* stream) {
  return guarded("sem_ax", [&] {
    SEM_REQUIRE(h && u_L && w_L, "sem_ax: null handle or vector");
    SEM_REQUIRE(u_L != w_L, "sem_ax: u_L and w_L must be distinct");
    cudaStream_t s = (cudaStream_t)stream;
    if (dtype == SEM_F64) {
      launch_ax<double>(h, h->f64, (const double*)u_L, (double*)w_L, h1, h2,
                        (const double*)h1_field, nullptr, s);
    } else if (dtype == SEM_F32) {
      if (!h->f32.G.ptr) throw Error(SEM_ERR_STATE, "sem_ax: handle keeps no FP32 geometry");
      launch_ax<float>(h, h->f32, (const float*)u_L, (float*)w_L, (float)h1, (float)h2,
                       (const float*)h1_field, nullptr, s);
    } else {
      throw Error(SEM_ERR_ARG, "sem_ax: bad dtype");
    }
  });
}
