// Two-level additive overlapping Schwarz preconditioner (arXiv 2107.01243 §4:
// Neko's pressure preconditioner, M^-1 = R_0^T A_0^-1 R_0 + sum_k R_k^T
// A~_k^-1 R_k, after Nek5000), applied in FP32:
//
// local level   subdomain = element grown by one GLL point into each
//               neighbour, (N + 3)^3 lattice points without points outside
//               the box and without Dirichlet points.  A~_e is the separable
//               Kronecker sum of 1D spectral-element stiffness and mass
//               matrices of the element and its neighbours (undeformed box
//               spacing), inverted by fast diagonalisation: per direction
//               A S = B S diag(lam), S^T B S = I, computed once on the host.
//               One CTA per element (persistent): gather the grown box of
//               r from the global vector, five line phases (S^T along x, y;
//               along z with the diagonal scaling and S back; S along y, x),
//               scatter-add to z by L2 reductions.  The same kernel forms the
//               coarse restriction from the element's own points.
// coarse level  trilinear vertex functions; A_0 = R_0 H R_0^T assembled from
//               8 x 8 element matrices Phi^T H_e Phi (computed at setup with
//               the FP64 element operator, stored packed in FP32); a fixed
//               number of Jacobi-PCG iterations from zero (the FP32 CG steps
//               of cg.cu with an element-by-element coarse matvec).
// output        z_L = mask o (z_local[g(L)] + R_0^T c) as FP64 L-vector.
#include <cmath>
#include <memory>
#include <vector>

#include "sem_internal.cuh"
#include "reduce.cuh"
#include "tma.cuh"

namespace sem {
namespace {

// threads of the local-solve CTA: one per z-column of the grown box, whole warps
template <int PE>
struct SwCfg {
  static constexpr int THREADS = PE * PE <= 128 ? 128 : (PE * PE + 31) / 32 * 32;
  static constexpr int MINB = PE * PE <= 128 ? 4 : 2;
};
constexpr int kNbr = 0, kDir = 1, kFree = 2;

// ------------------------------------------------------------------ host setup
// Symmetric eigen-decomposition by cyclic Jacobi rotations (n <= 13):
// A = V diag(lam) V^T, V orthogonal (columns are eigenvectors).
void jacobi_eigen(int n, std::vector<double> A, std::vector<double>& V, std::vector<double>& lam) {
  V.assign(n * n, 0.0);
  for (int i = 0; i < n; ++i) V[i * n + i] = 1.0;
  double scale = 0.0;
  for (double a : A) scale = std::max(scale, std::fabs(a));
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) off = std::max(off, std::fabs(A[p * n + q]));
    if (off <= 1e-16 * scale) break;
    for (int p = 0; p < n; ++p) {
      for (int q = p + 1; q < n; ++q) {
        const double apq = A[p * n + q];
        if (std::fabs(apq) <= 1e-300) continue;
        const double theta = (A[q * n + q] - A[p * n + p]) / (2.0 * apq);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {           // columns p, q
          const double akp = A[k * n + p], akq = A[k * n + q];
          A[k * n + p] = c * akp - s * akq;
          A[k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {           // rows p, q
          const double apk = A[p * n + k], aqk = A[q * n + k];
          A[p * n + k] = c * apk - s * aqk;
          A[q * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          const double vkp = V[k * n + p], vkq = V[k * n + q];
          V[k * n + p] = c * vkp - s * vkq;
          V[k * n + q] = s * vkp + c * vkq;
        }
      }
    }
  }
  lam.resize(n);
  for (int i = 0; i < n; ++i) lam[i] = A[i * n + i];
}

// 1D stiffness and lumped mass on the N + 3 points of a grown element
// (position a = lattice point N e - 1 + a), from the element and its
// neighbours of length L; positions not kept are decoupled (unit diagonal).
void extended_1d(const sem_handle* h, double L, int lo, int hi, std::vector<double>& A,
                 std::vector<double>& B, unsigned& keep) {
  const int N = h->N, P = h->P, Pe = N + 3, n3 = 3 * N + 1;
  std::vector<double> ae(P * P, 0.0);
  for (int i = 0; i < P; ++i)
    for (int j = 0; j < P; ++j) {
      double acc = 0.0;
      for (int k = 0; k < P; ++k) acc += h->Dh[k * P + i] * h->wq[k] * h->Dh[k * P + j];
      ae[i * P + j] = (2.0 / L) * acc;
    }
  std::vector<double> A3(n3 * n3, 0.0), B3(n3, 0.0);
  for (int m = 0; m < 3; ++m) {
    if ((m == 0 && lo != kNbr) || (m == 2 && hi != kNbr)) continue;
    const int s0 = m * N;
    for (int i = 0; i < P; ++i) {
      B3[s0 + i] += 0.5 * L * h->wq[i];
      for (int j = 0; j < P; ++j) A3[(s0 + i) * n3 + s0 + j] += ae[i * P + j];
    }
  }
  keep = (1u << Pe) - 1u;
  if (lo != kNbr) {
    keep &= ~1u;
    if (lo == kDir) keep &= ~2u;
  }
  if (hi != kNbr) {
    keep &= ~(1u << (N + 2));
    if (hi == kDir) keep &= ~(1u << (N + 1));
  }
  A.assign(Pe * Pe, 0.0);
  B.assign(Pe, 0.0);
  for (int a = 0; a < Pe; ++a) {
    const int ga = N - 1 + a;
    B[a] = B3[ga];
    for (int b = 0; b < Pe; ++b) A[a * Pe + b] = A3[ga * n3 + N - 1 + b];
  }
  for (int a = 0; a < Pe; ++a) {
    if (keep & (1u << a)) continue;
    for (int b = 0; b < Pe; ++b) {
      A[a * Pe + b] = 0.0;
      A[b * Pe + a] = 0.0;
    }
    A[a * Pe + a] = 1.0;
    B[a] = 1.0;
  }
}

// ------------------------------------------------------------------ device tables
// Per direction d and element kind v (bit 0: first along d, bit 1: last),
// rows padded to R floats: ST[a'][a] = S[a][a'], then S[a][a'], then lam[a].
template <int PE>
struct SwLayout {
  static constexpr int R = (PE + 3) / 4 * 4;
  static constexpr int TAB = 2 * PE * R + R;         // one (d, v) table
  static constexpr int ALL = 12 * TAB;
};

struct SwParams {
  int N, nelx, nely, nelz, gx, gy;
  long long sk;
  FastDiv dnx, dny;
  unsigned keep[3][4];
  float h1, h2;
  int do_local, do_coarse;
  float phi[2][kMaxP];                 // trilinear vertex functions at the GLL nodes
};

template <int R>
__device__ __forceinline__ float dot_row(const float* __restrict__ row, const float (&x)[R], int n) {
  float acc = 0.0f;
#pragma unroll
  for (int a = 0; a < R; a += 4) {
    const float4 v = *reinterpret_cast<const float4*>(row + a);
    if (a + 0 < n) acc = fmaf(v.x, x[a + 0], acc);
    if (a + 1 < n) acc = fmaf(v.y, x[a + 1], acc);
    if (a + 2 < n) acc = fmaf(v.z, x[a + 2], acc);
    if (a + 3 < n) acc = fmaf(v.w, x[a + 3], acc);
  }
  return acc;
}

// One element at a time per CTA.  Thread (a, b) < PE^2 owns the z-column of
// the grown box: it gathers the column, applies S^T along z in registers and
// writes box[c][b][a] (rows padded to R); the x- and y-directions run as line
// tasks through shared memory (S^T along x; along y S^T, the diagonal scaling
// and S; S along x); the thread then reads its column back, applies S along
// z in registers and adds the kept points to z.  Factors along different
// directions commute, so this order gives the same A~^-1 as x, y, z first.
// The coarse restriction is taken from the gathered columns of the element's
// own points (a, b, c in 1 .. P).
template <int PE>
__global__ void __launch_bounds__(SwCfg<PE>::THREADS, SwCfg<PE>::MINB)
schwarz_local_kernel(const float* __restrict__ rg, float* __restrict__ zg,
                     float* __restrict__ rc, const float* __restrict__ tab_g, SwParams prm,
                     int E) {
  using L = SwLayout<PE>;
  constexpr int R = L::R, P = PE - 2, N = PE - 3;
  __shared__ __align__(16) float tab[L::ALL];
  __shared__ __align__(16) float box[PE * PE * R];
  constexpr int NW = SwCfg<PE>::THREADS / 32;
  __shared__ float red[8][NW];
  for (int q = threadIdx.x; q < L::ALL; q += blockDim.x) tab[q] = tab_g[q];
  __syncthreads();
  const int tid = threadIdx.x;
  const bool owner = tid < PE * PE;
  const int ca = tid % PE, cb = tid / PE;          // this thread's column (a, b)
  for (int e = blockIdx.x; e < E; e += gridDim.x) {
    const uint32_t r1 = prm.dnx.div((uint32_t)e);
    const int ex = e - (int)r1 * prm.nelx;
    const uint32_t q1 = prm.dny.div(r1);
    const int ey = (int)(r1 - q1 * (uint32_t)prm.nely), ez = (int)q1;
    const int vx = (ex == 0 ? 1 : 0) | (ex == prm.nelx - 1 ? 2 : 0);
    const int vy = (ey == 0 ? 1 : 0) | (ey == prm.nely - 1 ? 2 : 0);
    const int vz = (ez == 0 ? 1 : 0) | (ez == prm.nelz - 1 ? 2 : 0);
    const unsigned kx = prm.keep[0][vx], ky = prm.keep[1][vy], kz = prm.keep[2][vz];
    const float* tx = tab + (0 * 4 + vx) * L::TAB;
    const float* ty = tab + (1 * 4 + vy) * L::TAB;
    const float* tz = tab + (2 * 4 + vz) * L::TAB;
    const bool colkeep = owner && ((kx >> ca) & 1u) && ((ky >> cb) & 1u);
    // lattice index of (a, b, 0) of this thread's column
    const long long cbase = (long long)(N * ex - 1 + ca) + (long long)prm.gx * (N * ey - 1 + cb) +
                            prm.sk * (long long)(N * ez - 1);
    float col[R];
#pragma unroll
    for (int c = 0; c < R; ++c)
      col[c] = (c < PE && colkeep && ((kz >> c) & 1u)) ? rg[cbase + prm.sk * c] : 0.0f;
    if (prm.do_coarse) {
      // restriction: sum over own points of phi_v r / mult
      float acc[8];
#pragma unroll
      for (int v = 0; v < 8; ++v) acc[v] = 0.0f;
      if (owner && ca >= 1 && ca <= P && cb >= 1 && cb <= P) {
        const int i = ca - 1, j = cb - 1;
        const float mij = ((i == 0 && ex > 0) || (i == N && ex < prm.nelx - 1) ? 0.5f : 1.0f) *
                          ((j == 0 && ey > 0) || (j == N && ey < prm.nely - 1) ? 0.5f : 1.0f);
        float s0 = 0.0f, s1 = 0.0f;
#pragma unroll
        for (int k = 0; k < P; ++k) {
          const float mk = (k == 0 && ez > 0) || (k == N && ez < prm.nelz - 1) ? 0.5f : 1.0f;
          const float rv = mk * col[k + 1];
          s0 = fmaf(prm.phi[0][k], rv, s0);
          s1 = fmaf(prm.phi[1][k], rv, s1);
        }
#pragma unroll
        for (int v = 0; v < 8; ++v)
          acc[v] = mij * prm.phi[v & 1][i] * prm.phi[(v >> 1) & 1][j] * ((v >> 2) ? s1 : s0);
      }
#pragma unroll
      for (int v = 0; v < 8; ++v)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc[v] += __shfl_down_sync(0xffffffffu, acc[v], o);
      if ((tid & 31) == 0)
#pragma unroll
        for (int v = 0; v < 8; ++v) red[v][tid >> 5] = acc[v];
      __syncthreads();
      if (tid < 8) {
        float t = 0.0f;
        for (int w = 0; w < NW; ++w) t += red[tid][w];
        const int v = tid;
        const long long vi = (long long)(ex + (v & 1)) +
                             (long long)(prm.nelx + 1) *
                                 ((ey + ((v >> 1) & 1)) + (long long)(prm.nely + 1) * (ez + (v >> 2)));
        red_add(rc + vi, t);
      }
    }
    if (prm.do_local) {
      // S^T along z in registers, to the box
      if (owner) {
#pragma unroll 2
        for (int c = 0; c < PE; ++c) box[(c * PE + cb) * R + ca] = dot_row<R>(tz + c * R, col, PE);
      }
      __syncthreads();
      // S^T along x on lines (b, c)
      for (int ln = tid; ln < PE * PE; ln += blockDim.x) {
        float* row = box + ln * R;
        float x[R];
#pragma unroll
        for (int a = 0; a < R; a += 4) {
          const float4 v = *reinterpret_cast<const float4*>(row + a);
          x[a] = v.x; x[a + 1] = v.y; x[a + 2] = v.z; x[a + 3] = v.w;
        }
#pragma unroll 2
        for (int a = 0; a < PE; ++a) row[a] = dot_row<R>(tx + a * R, x, PE);
      }
      __syncthreads();
      // along y on lines (a, c): S^T, the diagonal scaling, S
      for (int ln = tid; ln < PE * PE; ln += blockDim.x) {
        const int a = ln % PE, c = ln / PE;
        float* yl = box + c * PE * R + a;
        float x[R];
#pragma unroll
        for (int b = 0; b < R; ++b) x[b] = b < PE ? yl[b * R] : 0.0f;
        const float lac = tx[2 * PE * R + a] + tz[2 * PE * R + c];
        float t[R];
#pragma unroll
        for (int b = 0; b < R; ++b) {
          if (b < PE) {
            const float d = prm.h1 * (lac + ty[2 * PE * R + b]) + prm.h2;
            t[b] = dot_row<R>(ty + b * R, x, PE) / d;
          } else {
            t[b] = 0.0f;
          }
        }
#pragma unroll 2
        for (int b = 0; b < PE; ++b) yl[b * R] = dot_row<R>(ty + PE * R + b * R, t, PE);
      }
      __syncthreads();
      // S along x
      for (int ln = tid; ln < PE * PE; ln += blockDim.x) {
        float* row = box + ln * R;
        float x[R];
#pragma unroll
        for (int a = 0; a < R; a += 4) {
          const float4 v = *reinterpret_cast<const float4*>(row + a);
          x[a] = v.x; x[a + 1] = v.y; x[a + 2] = v.z; x[a + 3] = v.w;
        }
#pragma unroll 2
        for (int a = 0; a < PE; ++a) row[a] = dot_row<R>(tx + PE * R + a * R, x, PE);
      }
      __syncthreads();
      // S along z in registers, add the kept points
      if (colkeep) {
#pragma unroll
        for (int c = 0; c < R; ++c) col[c] = c < PE ? box[(c * PE + cb) * R + ca] : 0.0f;
#pragma unroll 2
        for (int c = 0; c < PE; ++c)
          if ((kz >> c) & 1u) red_add(zg + cbase + prm.sk * c, dot_row<R>(tz + PE * R + c * R, col, PE));
      }
    }
    __syncthreads();                         // box and red are reused by the next element
  }
}

// packed index of (r, c), r <= c, in the upper triangle of an 8 x 8 matrix
__host__ __device__ constexpr int pk(int r, int c) { return r * 8 - r * (r - 1) / 2 + (c - r); }

// w += A_0 p element by element (K packed symmetric, FP32)
__global__ void k_coarse_matvec(int E, const float* __restrict__ K, const float* __restrict__ p,
                                float* __restrict__ w, int nelx, int nely, FastDiv dnx,
                                FastDiv dny) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < E; e += gridDim.x * blockDim.x) {
    const uint32_t r1 = dnx.div((uint32_t)e);
    const int ex = e - (int)r1 * nelx;
    const uint32_t q1 = dny.div(r1);
    const int ey = (int)(r1 - q1 * (uint32_t)nely), ez = (int)q1;
    int vi[8];
    float pv[8];
#pragma unroll
    for (int v = 0; v < 8; ++v) {
      vi[v] = (ex + (v & 1)) + (nelx + 1) * ((ey + ((v >> 1) & 1)) + (nely + 1) * (ez + (v >> 2)));
      pv[v] = p[vi[v]];
    }
    const float* Ke = K + (size_t)e * 36;
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      float acc = 0.0f;
#pragma unroll
      for (int c = 0; c < 8; ++c) acc = fmaf(Ke[r <= c ? pk(r, c) : pk(c, r)], pv[c], acc);
      red_add(w + vi[r], acc);
    }
  }
}

// L-vector of vertex function v (all elements), FP64
__global__ void k_vertex_field(int64_t nL, int P, int v, const double* __restrict__ xi,
                               double* __restrict__ out) {
  const int P3 = P * P * P;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nL;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int lq = (int)(q % P3);
    const int i = lq % P, j = (lq / P) % P, k = lq / (P * P);
    const double fa = (v & 1) ? 0.5 * (1.0 + xi[i]) : 0.5 * (1.0 - xi[i]);
    const double fb = ((v >> 1) & 1) ? 0.5 * (1.0 + xi[j]) : 0.5 * (1.0 - xi[j]);
    const double fc = (v >> 2) ? 0.5 * (1.0 + xi[k]) : 0.5 * (1.0 - xi[k]);
    out[q] = fa * fb * fc;
  }
}

// K[e][pk(r, v)] = phi_r^T (H_e phi_v) for r <= v (one CTA per element)
__global__ void k_coarse_entries(int E, int P, int v, const double* __restrict__ hv,
                                 const double* __restrict__ xi, float* __restrict__ K,
                                 double* __restrict__ diag) {
  __shared__ double red[8][8];
  const int P3 = P * P * P;
  for (int e = blockIdx.x; e < E; e += gridDim.x) {
    double acc[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) acc[r] = 0.0;
    for (int q = threadIdx.x; q < P3; q += blockDim.x) {
      const int i = q % P, j = (q / P) % P, k = q / (P * P);
      const double hq = hv[(size_t)e * P3 + q];
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        const double fa = (r & 1) ? 0.5 * (1.0 + xi[i]) : 0.5 * (1.0 - xi[i]);
        const double fb = ((r >> 1) & 1) ? 0.5 * (1.0 + xi[j]) : 0.5 * (1.0 - xi[j]);
        const double fc = (r >> 2) ? 0.5 * (1.0 + xi[k]) : 0.5 * (1.0 - xi[k]);
        acc[r] += fa * fb * fc * hq;
      }
    }
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc[r] += __shfl_down_sync(0xffffffffu, acc[r], o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0)
#pragma unroll
      for (int r = 0; r < 8; ++r) red[r][wid] = acc[r];
    __syncthreads();
    if (threadIdx.x < 8) {
      const int r = threadIdx.x;
      double t = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[r][w];
      if (r <= v) K[(size_t)e * 36 + pk(r, v)] = (float)t;
      if (r == v) diag[(size_t)e * 8 + v] = t;
    }
    __syncthreads();
  }
}

// cdinv[v] = mask_v / sum over elements of the vertex's diagonal entries
__global__ void k_coarse_dinv(int E, const double* __restrict__ diag, float* __restrict__ cdinv,
                              double* __restrict__ acc, int nelx, int nely, int nelz, int faces,
                              int phase) {
  const int nvx = nelx + 1, nvy = nely + 1, nvz = nelz + 1;
  if (phase == 0) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < E; e += gridDim.x * blockDim.x) {
      const int ex = e % nelx, ey = (e / nelx) % nely, ez = e / (nelx * nely);
      for (int v = 0; v < 8; ++v) {
        const int vi = (ex + (v & 1)) + nvx * ((ey + ((v >> 1) & 1)) + nvy * (ez + (v >> 2)));
        atomicAdd(acc + vi, diag[(size_t)e * 8 + v]);
      }
    }
  } else {
    const int nv = nvx * nvy * nvz;
    for (int vi = blockIdx.x * blockDim.x + threadIdx.x; vi < nv; vi += gridDim.x * blockDim.x) {
      const int x = vi % nvx, y = (vi / nvx) % nvy, z = vi / (nvx * nvy);
      const bool masked = ((faces & SEM_FACE_XMIN) && x == 0) || ((faces & SEM_FACE_XMAX) && x == nelx) ||
                          ((faces & SEM_FACE_YMIN) && y == 0) || ((faces & SEM_FACE_YMAX) && y == nely) ||
                          ((faces & SEM_FACE_ZMIN) && z == 0) || ((faces & SEM_FACE_ZMAX) && z == nelz);
      cdinv[vi] = masked || !(acc[vi] > 0.0) ? 0.0f : (float)(1.0 / acc[vi]);
    }
  }
}

// z_L = mask o (z_local[g(L)] + sum_v phi_v c_v) at every local point
template <int P>
__global__ void k_sw_combine(int64_t nL, const float* __restrict__ zg, const float* __restrict__ xc,
                             double* __restrict__ z, SwParams prm, int faces) {
  constexpr int N = P - 1, P3 = P * P * P;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nL;
       q += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t e = (uint32_t)q / (uint32_t)P3;    // n_L < 2^31
    const int lq = (int)((uint32_t)q - e * (uint32_t)P3);
    const int i = lq % P, j = (lq / P) % P, k = lq / (P * P);
    const uint32_t re = prm.dnx.div(e);
    const int ex = (int)(e - re * (uint32_t)prm.nelx);
    const uint32_t ezu = prm.dny.div(re);
    const int ey = (int)(re - ezu * (uint32_t)prm.nely), ez = (int)ezu;
    const int ix = ex * N + i, iy = ey * N + j, iz = ez * N + k;
    const bool masked = ((faces & SEM_FACE_XMIN) && ix == 0) ||
                        ((faces & SEM_FACE_XMAX) && ix == prm.gx - 1) ||
                        ((faces & SEM_FACE_YMIN) && iy == 0) ||
                        ((faces & SEM_FACE_YMAX) && iy == prm.gy - 1) ||
                        ((faces & SEM_FACE_ZMIN) && iz == 0) ||
                        ((faces & SEM_FACE_ZMAX) && iz == N * prm.nelz);
    double v = 0.0;
    if (!masked) {
      v = (double)zg[(long long)ix + (long long)prm.gx * iy + prm.sk * iz];
      if (xc) {
        const int v0 = ex + (prm.nelx + 1) * (ey + (prm.nely + 1) * ez);
        const int sy = prm.nelx + 1, sz = (prm.nelx + 1) * (prm.nely + 1);
        const float fx0 = prm.phi[0][i], fx1 = prm.phi[1][i];
        const float fy0 = prm.phi[0][j], fy1 = prm.phi[1][j];
        const float fz0 = prm.phi[0][k], fz1 = prm.phi[1][k];
        const float c00 = fmaf(fx1, xc[v0 + 1], fx0 * xc[v0]);
        const float c10 = fmaf(fx1, xc[v0 + sy + 1], fx0 * xc[v0 + sy]);
        const float c01 = fmaf(fx1, xc[v0 + sz + 1], fx0 * xc[v0 + sz]);
        const float c11 = fmaf(fx1, xc[v0 + sz + sy + 1], fx0 * xc[v0 + sz + sy]);
        v += (double)fmaf(fz1, fmaf(fy1, c11, fy0 * c01), fz0 * fmaf(fy1, c10, fy0 * c00));
      }
    }
    z[q] = v;
  }
}

int ew_blocks(int64_t n) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 8 * sem_num_sms()));
}

}  // namespace
}  // namespace sem

using namespace sem;

struct sem_schwarz {
  sem_handle* h = nullptr;
  int levels = 3, coarse_iters = 10;
  double h1 = 1.0, h2 = 0.0;
  int Pe = 0;
  SwParams prm{};
  DevBuf<float> tab;                       // FDM tables
  int64_t nv = 0, nv4 = 0;                 // coarse vertices, padded
  DevBuf<float> K, cdinv, rc, xc, pc, wc;
  DevBuf<float> rg, zg;                    // fine global vectors
  DevBuf<CGState> st;
  DevBuf<double> partials;
};

namespace sem {
namespace {

template <int PE>
void launch_local(sem_schwarz* sw, const float* rg, float* zg, cudaStream_t s) {
  const sem_handle* h = sw->h;
  auto kern = schwarz_local_kernel<PE>;
  constexpr int T = SwCfg<PE>::THREADS;
  static int occ = 0;
  if (!occ) {
    SEM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, T, 0));
    if (occ < 1) occ = 1;
  }
  const int grid = (int)std::min<int64_t>(h->E, (int64_t)occ * sem_num_sms());
  kern<<<grid, T, 0, s>>>(rg, zg, sw->rc.ptr, sw->tab.ptr, sw->prm, (int)h->E);
  SEM_CHECK_LAUNCH();
}

void launch_local_any(sem_schwarz* sw, const float* rg, float* zg, cudaStream_t s) {
  switch (sw->Pe) {
    case 4: launch_local<4>(sw, rg, zg, s); break;
    case 5: launch_local<5>(sw, rg, zg, s); break;
    case 6: launch_local<6>(sw, rg, zg, s); break;
    case 7: launch_local<7>(sw, rg, zg, s); break;
    case 8: launch_local<8>(sw, rg, zg, s); break;
    case 9: launch_local<9>(sw, rg, zg, s); break;
    case 10: launch_local<10>(sw, rg, zg, s); break;
    case 11: launch_local<11>(sw, rg, zg, s); break;
    case 12: launch_local<12>(sw, rg, zg, s); break;
    case 13: launch_local<13>(sw, rg, zg, s); break;
    default: throw Error(SEM_ERR_ARG, "schwarz: unsupported order");
  }
}

// fills the host FDM tables in the layout of SwLayout<Pe>
void build_tables(sem_schwarz* sw, std::vector<float>& out) {
  const sem_handle* h = sw->h;
  const int N = h->N, Pe = N + 3, R = (Pe + 3) / 4 * 4, TAB = 2 * Pe * R + R;
  out.assign(12 * TAB, 0.0f);
  const int nel[3] = {h->nelx, h->nely, h->nelz};
  const int flo[3] = {SEM_FACE_XMIN, SEM_FACE_YMIN, SEM_FACE_ZMIN};
  const int fhi[3] = {SEM_FACE_XMAX, SEM_FACE_YMAX, SEM_FACE_ZMAX};
  for (int d = 0; d < 3; ++d) {
    const double L = h->len[d] / nel[d];
    for (int v = 0; v < 4; ++v) {
      const int bkind_lo = (h->faces & flo[d]) ? kDir : kFree;
      const int bkind_hi = (h->faces & fhi[d]) ? kDir : kFree;
      const int lo = (v & 1) ? bkind_lo : kNbr;
      const int hi = (v & 2) ? bkind_hi : kNbr;
      std::vector<double> A, B, V, lam;
      unsigned keep = 0;
      extended_1d(h, L, lo, hi, A, B, keep);
      sw->prm.keep[d][v] = keep;
      std::vector<double> C(Pe * Pe), bh(Pe);
      for (int a = 0; a < Pe; ++a) bh[a] = 1.0 / std::sqrt(B[a]);
      for (int a = 0; a < Pe; ++a)
        for (int b = 0; b < Pe; ++b) C[a * Pe + b] = bh[a] * A[a * Pe + b] * bh[b];
      for (int a = 0; a < Pe; ++a)           // symmetrise against rounding
        for (int b = a + 1; b < Pe; ++b) {
          const double m = 0.5 * (C[a * Pe + b] + C[b * Pe + a]);
          C[a * Pe + b] = C[b * Pe + a] = m;
        }
      jacobi_eigen(Pe, C, V, lam);
      float* t = out.data() + (d * 4 + v) * TAB;
      for (int a = 0; a < Pe; ++a)
        for (int ap = 0; ap < Pe; ++ap) {
          const double S = bh[a] * V[a * Pe + ap];     // S[a][a']
          t[ap * R + a] = (float)S;                    // ST[a'][a]
          t[Pe * R + a * R + ap] = (float)S;           // S[a][a']
        }
      for (int a = 0; a < Pe; ++a) t[2 * Pe * R + a] = (float)lam[a];
    }
  }
}

// coarse element matrices from the FP64 element operator
void build_coarse(sem_schwarz* sw, cudaStream_t s) {
  sem_handle* h = sw->h;
  const int64_t nL = h->nL, E = h->E;
  sw->K.alloc((size_t)E * 36);
  DevBuf<double> phi, hphi, dg, acc, xi;
  phi.alloc(nL);
  hphi.alloc(nL);
  dg.alloc((size_t)E * 8);
  xi.alloc(h->P);
  xi.upload(h->xi.data(), h->P, s);
  for (int v = 0; v < 8; ++v) {
    k_vertex_field<<<ew_blocks(nL), 256, 0, s>>>(nL, h->P, v, xi.ptr, phi.ptr);
    SEM_CHECK_LAUNCH();
    launch_ax<double>(h, h->f64, phi.ptr, hphi.ptr, sw->h1, sw->h2, nullptr, nullptr, s);
    k_coarse_entries<<<(int)std::min<int64_t>(E, 8 * sem_num_sms()), 128, 0, s>>>(
        (int)E, h->P, v, hphi.ptr, xi.ptr, sw->K.ptr, dg.ptr);
    SEM_CHECK_LAUNCH();
  }
  acc.alloc(sw->nv);
  SEM_CUDA(cudaMemsetAsync(acc.ptr, 0, sw->nv * sizeof(double), s));
  SEM_CUDA(cudaMemsetAsync(sw->cdinv.ptr, 0, sw->nv4 * 4 * sizeof(float), s));
  k_coarse_dinv<<<ew_blocks(E), 256, 0, s>>>((int)E, dg.ptr, sw->cdinv.ptr, acc.ptr, h->nelx,
                                            h->nely, h->nelz, h->faces, 0);
  SEM_CHECK_LAUNCH();
  k_coarse_dinv<<<ew_blocks(sw->nv), 256, 0, s>>>((int)E, dg.ptr, sw->cdinv.ptr, acc.ptr,
                                                 h->nelx, h->nely, h->nelz, h->faces, 1);
  SEM_CHECK_LAUNCH();
  SEM_CUDA(cudaStreamSynchronize(s));      // the scratch buffers are freed on return
}

}  // namespace

sem_handle* schwarz_handle(const sem_schwarz* sw) { return sw->h; }

namespace {

// the local solves of rg added into zg (zeroed here), the coarse restriction
// and the coarse CG; returns the coarse solution or NULL (no coarse level)
const float* schwarz_levels(sem_schwarz* sw, const float* rg, float* zg, cudaStream_t s) {
  sem_handle* h = sw->h;
  SEM_CUDA(cudaMemsetAsync(zg, 0, h->nG * sizeof(float), s));
  const bool coarse = (sw->levels & SEM_SCHWARZ_COARSE) != 0;
  if (coarse) SEM_CUDA(cudaMemsetAsync(sw->rc.ptr, 0, sw->nv4 * 4 * sizeof(float), s));
  launch_local_any(sw, rg, zg, s);
  if (coarse) {
    CGState* st = sw->st.ptr;
    vcg_init(sw->nv4, sw->rc.ptr, sw->cdinv.ptr, sw->pc.ptr, sw->xc.ptr, sw->wc.ptr, st,
             sw->partials.ptr, 0.0, sw->coarse_iters, s);
    const FastDiv dnx((uint32_t)h->nelx), dny((uint32_t)h->nely);
    for (int it = 0; it < sw->coarse_iters; ++it) {
      k_coarse_matvec<<<ew_blocks(h->E), 256, 0, s>>>((int)h->E, sw->K.ptr, sw->pc.ptr,
                                                      sw->wc.ptr, h->nelx, h->nely, dnx, dny);
      SEM_CHECK_LAUNCH();
      vcg_pw(sw->nv4, sw->pc.ptr, sw->wc.ptr, st, sw->partials.ptr, s);
      vcg_update(sw->nv4, sw->xc.ptr, sw->rc.ptr, sw->pc.ptr, sw->wc.ptr, sw->cdinv.ptr, st,
                 sw->partials.ptr, s);
      vcg_pupd(sw->nv4, sw->pc.ptr, sw->rc.ptr, sw->cdinv.ptr, st, s);
    }
  }
  return coarse ? sw->xc.ptr : nullptr;
}

// z_g = mask o (z_g + R_0^T c) at every global point, c read in the element
// that holds the point at (i, j, k) with i, j, k < N where possible
__global__ void k_sw_combine_global(int64_t nG, float* __restrict__ z, const float* __restrict__ xc,
                                    SwParams prm, int faces, FastDiv dgx, FastDiv dgy,
                                    FastDiv dN) {
  const int N = prm.N;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < nG;
       g += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t r = dgx.div((uint32_t)g);
    const int ix = (int)((uint32_t)g - r * dgx.d);
    const uint32_t izu = dgy.div(r);
    const int iy = (int)(r - izu * dgy.d), iz = (int)izu;
    const bool masked = ((faces & SEM_FACE_XMIN) && ix == 0) ||
                        ((faces & SEM_FACE_XMAX) && ix == prm.gx - 1) ||
                        ((faces & SEM_FACE_YMIN) && iy == 0) ||
                        ((faces & SEM_FACE_YMAX) && iy == prm.gy - 1) ||
                        ((faces & SEM_FACE_ZMIN) && iz == 0) ||
                        ((faces & SEM_FACE_ZMAX) && iz == N * prm.nelz);
    if (masked) {
      z[g] = 0.0f;
      continue;
    }
    if (!xc) continue;
    const int ex = min((int)dN.div((uint32_t)ix), prm.nelx - 1);
    const int ey = min((int)dN.div((uint32_t)iy), prm.nely - 1);
    const int ez = min((int)dN.div((uint32_t)iz), prm.nelz - 1);
    const int i = ix - ex * N, j = iy - ey * N, k = iz - ez * N;
    const int v0 = ex + (prm.nelx + 1) * (ey + (prm.nely + 1) * ez);
    const int sy = prm.nelx + 1, sz = (prm.nelx + 1) * (prm.nely + 1);
    const float fx0 = prm.phi[0][i], fx1 = prm.phi[1][i];
    const float fy0 = prm.phi[0][j], fy1 = prm.phi[1][j];
    const float fz0 = prm.phi[0][k], fz1 = prm.phi[1][k];
    const float c00 = fmaf(fx1, xc[v0 + 1], fx0 * xc[v0]);
    const float c10 = fmaf(fx1, xc[v0 + sy + 1], fx0 * xc[v0 + sy]);
    const float c01 = fmaf(fx1, xc[v0 + sz + 1], fx0 * xc[v0 + sz]);
    const float c11 = fmaf(fx1, xc[v0 + sz + sy + 1], fx0 * xc[v0 + sz + sy]);
    z[g] += fmaf(fz1, fmaf(fy1, c11, fy0 * c01), fz0 * fmaf(fy1, c10, fy0 * c00));
  }
}

}  // namespace

void schwarz_apply_global(sem_schwarz* sw, const float* r_g, float* z_g, cudaStream_t s) {
  sem_handle* h = sw->h;
  const float* xcp = schwarz_levels(sw, r_g, z_g, s);
  k_sw_combine_global<<<ew_blocks(h->nG), 256, 0, s>>>(
      h->nG, z_g, xcp, sw->prm, h->faces, FastDiv((uint32_t)(h->N * h->nelx + 1)),
      FastDiv((uint32_t)(h->N * h->nely + 1)), FastDiv((uint32_t)h->N));
  SEM_CHECK_LAUNCH();
}

void schwarz_apply(sem_schwarz* sw, const double* r, double* z, cudaStream_t s) {
  sem_handle* h = sw->h;
  to_global<double>(h, r, sw->rg.ptr, s);
  const float* xcp = schwarz_levels(sw, sw->rg.ptr, sw->zg.ptr, s);
  const int cg = ew_blocks(h->nL);
  switch (h->P) {
    case 3: k_sw_combine<3><<<cg, 256, 0, s>>>(h->nL, sw->zg.ptr, xcp, z, sw->prm, h->faces); break;
    case 4: k_sw_combine<4><<<cg, 256, 0, s>>>(h->nL, sw->zg.ptr, xcp, z, sw->prm, h->faces); break;
    case 5: k_sw_combine<5><<<cg, 256, 0, s>>>(h->nL, sw->zg.ptr, xcp, z, sw->prm, h->faces); break;
    case 6: k_sw_combine<6><<<cg, 256, 0, s>>>(h->nL, sw->zg.ptr, xcp, z, sw->prm, h->faces); break;
    case 7: k_sw_combine<7><<<cg, 256, 0, s>>>(h->nL, sw->zg.ptr, xcp, z, sw->prm, h->faces); break;
    case 8: k_sw_combine<8><<<cg, 256, 0, s>>>(h->nL, sw->zg.ptr, xcp, z, sw->prm, h->faces); break;
    case 9: k_sw_combine<9><<<cg, 256, 0, s>>>(h->nL, sw->zg.ptr, xcp, z, sw->prm, h->faces); break;
    case 10: k_sw_combine<10><<<cg, 256, 0, s>>>(h->nL, sw->zg.ptr, xcp, z, sw->prm, h->faces); break;
    case 11: k_sw_combine<11><<<cg, 256, 0, s>>>(h->nL, sw->zg.ptr, xcp, z, sw->prm, h->faces); break;
    default: throw Error(SEM_ERR_ARG, "schwarz: unsupported order");
  }
  SEM_CHECK_LAUNCH();
}

}  // namespace sem

extern "C" sem_status sem_schwarz_create(sem_handle* h, double h1, double h2, int levels,
                                         int coarse_iters, void* stream, sem_schwarz** out) {
  return guarded("sem_schwarz_create", [&] {
    SEM_REQUIRE(h && out, "sem_schwarz_create: null argument");
    *out = nullptr;
    SEM_REQUIRE(levels >= 1 && levels <= 3, "sem_schwarz_create: levels must be 1, 2 or 3");
    SEM_REQUIRE(coarse_iters >= 0 && coarse_iters <= 1000,
                "sem_schwarz_create: coarse_iters must be in [0, 1000]");
    SEM_REQUIRE(h1 > 0.0 && h2 >= 0.0, "sem_schwarz_create: needs h1 > 0 and h2 >= 0");
    SEM_REQUIRE(h->N >= 2, "sem_schwarz_create: needs N >= 2 (the point a subdomain takes from "
                           "a neighbour must lie inside it)");
    cudaStream_t s = (cudaStream_t)stream;
    std::unique_ptr<sem_schwarz> sw(new sem_schwarz());
    sw->h = h;
    sw->levels = levels;
    sw->coarse_iters = coarse_iters;
    sw->h1 = h1;
    sw->h2 = h2;
    sw->Pe = h->N + 3;
    SwParams& p = sw->prm;
    p.N = h->N;
    p.nelx = h->nelx; p.nely = h->nely; p.nelz = h->nelz;
    p.gx = h->N * h->nelx + 1;
    p.gy = h->N * h->nely + 1;
    p.sk = (long long)p.gx * p.gy;
    p.dnx = FastDiv((uint32_t)h->nelx);
    p.dny = FastDiv((uint32_t)h->nely);
    p.h1 = (float)h1;
    p.h2 = (float)h2;
    p.do_local = (levels & SEM_SCHWARZ_LOCAL) ? 1 : 0;
    p.do_coarse = (levels & SEM_SCHWARZ_COARSE) ? 1 : 0;
    for (int i = 0; i < h->P; ++i) {
      p.phi[0][i] = (float)(0.5 * (1.0 - h->xi[i]));
      p.phi[1][i] = (float)(0.5 * (1.0 + h->xi[i]));
    }
    std::vector<float> t;
    build_tables(sw.get(), t);
    sw->tab.alloc(t.size());
    sw->tab.upload(t.data(), t.size(), s);
    sw->rg.alloc(h->nG);
    sw->zg.alloc(h->nG);
    sw->nv = (int64_t)(h->nelx + 1) * (h->nely + 1) * (h->nelz + 1);
    sw->nv4 = (sw->nv + 3) / 4;
    for (DevBuf<float>* b : {&sw->cdinv, &sw->rc, &sw->xc, &sw->pc, &sw->wc}) {
      b->alloc(sw->nv4 * 4);
      SEM_CUDA(cudaMemsetAsync(b->ptr, 0, sw->nv4 * 4 * sizeof(float), s));
    }
    sw->st.alloc(1);
    SEM_CUDA(cudaMemsetAsync(sw->st.ptr, 0, sizeof(CGState), s));
    sw->partials.alloc(2 * kRedBlocks);
    if (levels & SEM_SCHWARZ_COARSE) build_coarse(sw.get(), s);
    SEM_CUDA(cudaStreamSynchronize(s));
    *out = sw.release();
  });
}

extern "C" sem_status sem_schwarz_apply(sem_schwarz* sw, const double* r_L, double* z_L,
                                        void* stream) {
  return guarded("sem_schwarz_apply", [&] {
    SEM_REQUIRE(sw && r_L && z_L, "sem_schwarz_apply: null argument");
    SEM_REQUIRE(r_L != z_L, "sem_schwarz_apply: r and z must not alias");
    schwarz_apply(sw, r_L, z_L, (cudaStream_t)stream);
  });
}

extern "C" sem_status sem_schwarz_destroy(sem_schwarz* sw) {
  return guarded("sem_schwarz_destroy", [&] {
    if (sw) cudaDeviceSynchronize();
    delete sw;
  });
}
