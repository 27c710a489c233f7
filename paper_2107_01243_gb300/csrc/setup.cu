// Handle setup: GLL basis, box topology, gather-scatter lists, coordinates and
// geometric factors (arXiv 2107.01243 §2, Eq. 7-10; §3.2).  sem_setup also
// binds the process to its device and runs the once-per-process kernel setup
// of the handle's order, outside any stream capture.
#include <cmath>
#include <cstring>
#include <algorithm>
#include <atomic>
#include <numeric>
#include <memory>

#include "sem_internal.cuh"
#include "df.cuh"

namespace sem {

static thread_local std::string g_last_error;
void set_last_error(const std::string& msg) { g_last_error = msg; }

// ------------------------------------------------------------------ GLL basis
// L_N(x) and L_N'(x) by the three-term recurrence and L'_{n+1} = L'_{n-1} + (2n+1) L_n.
static void legendre_and_deriv(int N, double x, double& L, double& dL) {
  double L0 = 1.0, L1 = x, d0 = 0.0, d1 = 1.0;
  if (N == 0) { L = 1.0; dL = 0.0; return; }
  for (int n = 1; n < N; ++n) {
    double L2 = ((2.0 * n + 1.0) * x * L1 - n * L0) / (n + 1.0);
    double d2 = d0 + (2.0 * n + 1.0) * L1;
    L0 = L1; L1 = L2; d0 = d1; d1 = d2;
  }
  L = L1;
  dL = d1;
}

// GLL nodes (-1, 1 and the roots of L_N'), weights 2 / (N (N+1) L_N^2) and the
// nodal derivative matrix D[i][j] = l_j'(x_i) (§2, Eq. 7-9).
void gll_host(int N, std::vector<double>& xi, std::vector<double>& w, std::vector<double>& D) {
  const int p = N + 1;
  xi.assign(p, 0.0);
  w.assign(p, 0.0);
  D.assign(p * p, 0.0);
  xi[0] = -1.0;
  xi[N] = 1.0;
  const double pi = 3.14159265358979323846;
  for (int j = 1; j <= (N - 1) / 2 + ((N - 1) % 2); ++j) {
    // Newton on q = L_N', q' = L_N'' from the Legendre equation
    double x = -std::cos(pi * j / N);
    for (int it = 0; it < 100; ++it) {
      double L, dL;
      legendre_and_deriv(N, x, L, dL);
      double d2L = (2.0 * x * dL - N * (N + 1.0) * L) / (1.0 - x * x);
      double dx = dL / d2L;
      x -= dx;
      if (std::fabs(dx) < 1e-17) break;
    }
    xi[j] = x;
    xi[N - j] = -x;
  }
  if (N % 2 == 0) xi[N / 2] = 0.0;
  std::vector<double> LN(p);
  for (int i = 0; i < p; ++i) {
    double L, dL;
    legendre_and_deriv(N, xi[i], L, dL);
    LN[i] = L;
    w[i] = 2.0 / (N * (N + 1.0) * L * L);
  }
  for (int i = 0; i < p; ++i)
    for (int j = 0; j < p; ++j)
      if (i != j) D[i * p + j] = LN[i] / (LN[j] * (xi[i] - xi[j]));
  D[0] = -N * (N + 1.0) / 4.0;
  D[N * p + N] = N * (N + 1.0) / 4.0;
}

// ------------------------------------------------------------------ device kernels
struct BoxParams {
  int nelx, nely, P;
  double x0, y0, z0, hx, hy, hz, amp;
};

__global__ void box_coords_kernel(BoxParams bp, const double* __restrict__ xi, int64_t nL,
                                  double* __restrict__ X, double* __restrict__ Y,
                                  double* __restrict__ Z) {
  const int P = bp.P, P3 = P * P * P;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nL;
       q += (int64_t)gridDim.x * blockDim.x) {
    int64_t e = q / P3;
    int r = (int)(q - e * P3);
    int i = r % P, j = (r / P) % P, k = r / (P * P);
    int ex = (int)(e % bp.nelx);
    int ey = (int)((e / bp.nelx) % bp.nely);
    int ez = (int)(e / ((int64_t)bp.nelx * bp.nely));
    double x = bp.x0 + (ex + 0.5 * (xi[i] + 1.0)) * bp.hx;
    double y = bp.y0 + (ey + 0.5 * (xi[j] + 1.0)) * bp.hy;
    double z = bp.z0 + (ez + 0.5 * (xi[k] + 1.0)) * bp.hz;
    if (bp.amp != 0.0) {
      double xd = x + bp.amp * sin(y) * sin(z);
      double yd = y + bp.amp * sin(z) * sin(x);
      double zd = z + bp.amp * sin(x) * sin(y);
      x = xd; y = yd; z = zd;
    }
    X[q] = x; Y[q] = y; Z[q] = z;
  }
}

// Jacobian, geometric factors and mass at every local point (§2, Eq. 9):
// G_bc = W detJ sum_a (dr_b/dx_a)(dr_c/dx_a), B = W detJ.
__global__ void geom_kernel(int P, int64_t nL, const double* __restrict__ Dm,
                            const double* __restrict__ wq, const double* __restrict__ X,
                            const double* __restrict__ Y, const double* __restrict__ Z,
                            double* __restrict__ G, double* __restrict__ Bm,
                            float* __restrict__ G32, float* __restrict__ B32,
                            int* __restrict__ bad) {
  const int P2 = P * P, P3 = P2 * P;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nL;
       q += (int64_t)gridDim.x * blockDim.x) {
    int64_t e = q / P3;
    int r = (int)(q - e * P3);
    int i = r % P, j = (r / P) % P, k = r / P2;
    const int64_t base = e * P3;
    const double* c3[3] = {X, Y, Z};
    double J[3][3];
    for (int a = 0; a < 3; ++a) {
      const double* c = c3[a] + base;
      double dr = 0.0, ds = 0.0, dt = 0.0;
      for (int l = 0; l < P; ++l) {
        dr += Dm[i * P + l] * c[k * P2 + j * P + l];
        ds += Dm[j * P + l] * c[k * P2 + l * P + i];
        dt += Dm[k * P + l] * c[l * P2 + j * P + i];
      }
      J[a][0] = dr; J[a][1] = ds; J[a][2] = dt;
    }
    // cofactors: inv[b][a] = cof[a][b] / det
    double c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
    double c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
    double c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
    double c10 = J[0][2] * J[2][1] - J[0][1] * J[2][2];
    double c11 = J[0][0] * J[2][2] - J[0][2] * J[2][0];
    double c12 = J[0][1] * J[2][0] - J[0][0] * J[2][1];
    double c20 = J[0][1] * J[1][2] - J[0][2] * J[1][1];
    double c21 = J[0][2] * J[1][0] - J[0][0] * J[1][2];
    double c22 = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    double det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
    if (!(det > 0.0)) atomicExch(bad, 1);
    double id = 1.0 / det;
    // inv[b][a] = d r_b / d x_a
    double inv[3][3] = {{c00 * id, c10 * id, c20 * id},
                        {c01 * id, c11 * id, c21 * id},
                        {c02 * id, c12 * id, c22 * id}};
    double W = wq[i] * wq[j] * wq[k];
    double s = W * det;
    double g[6];
    const int bi[6] = {0, 1, 2, 0, 0, 1};
    const int ci[6] = {0, 1, 2, 1, 2, 2};
    for (int m = 0; m < 6; ++m) {
      int b = bi[m], c = ci[m];
      g[m] = s * (inv[b][0] * inv[c][0] + inv[b][1] * inv[c][1] + inv[b][2] * inv[c][2]);
    }
    double* Ge = G + e * 6 * P3 + r;
    for (int m = 0; m < 6; ++m) Ge[m * P3] = g[m];
    Bm[q] = s;
    if (G32) {
      float* G32e = G32 + e * 6 * P3 + r;
      for (int m = 0; m < 6; ++m) G32e[m * P3] = (float)g[m];
      B32[q] = (float)s;
    }
  }
}

// Global number, 1/multiplicity and Dirichlet mask of every local point of
// the box (the lattice index of (e, i, j, k) is (N ex + i, N ey + j, N ez + k)).
__global__ void topo_kernel(int N, int nelx, int nely, int nelz, int faces, int64_t nL,
                            int64_t* __restrict__ gid, float* __restrict__ imult,
                            uint8_t* __restrict__ mask) {
  const int P = N + 1, P3 = P * P * P;
  const int64_t gx = (int64_t)N * nelx + 1, gy = (int64_t)N * nely + 1, gz = (int64_t)N * nelz + 1;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nL;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = q / P3;
    const int r = (int)(q - e * P3);
    const int i = r % P, j = (r / P) % P, k = r / (P * P);
    const int64_t ix = (int64_t)N * (e % nelx) + i;
    const int64_t iy = (int64_t)N * ((e / nelx) % nely) + j;
    const int64_t iz = (int64_t)N * (e / ((int64_t)nelx * nely)) + k;
    gid[q] = ix + gx * (iy + gy * iz);
    const int m = ((ix % N == 0 && ix > 0 && ix < gx - 1) ? 2 : 1) *
                  ((iy % N == 0 && iy > 0 && iy < gy - 1) ? 2 : 1) *
                  ((iz % N == 0 && iz > 0 && iz < gz - 1) ? 2 : 1);
    imult[q] = 1.0f / (float)m;
    const bool d = ((faces & SEM_FACE_XMIN) && ix == 0) || ((faces & SEM_FACE_XMAX) && ix == gx - 1) ||
                   ((faces & SEM_FACE_YMIN) && iy == 0) || ((faces & SEM_FACE_YMAX) && iy == gy - 1) ||
                   ((faces & SEM_FACE_ZMIN) && iz == 0) || ((faces & SEM_FACE_ZMAX) && iz == gz - 1);
    mask[q] = d ? 0 : 1;
  }
}

template <class S, class D>
__global__ void convert_kernel(const S* __restrict__ src, D* __restrict__ dst, int64_t n) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
       q += (int64_t)gridDim.x * blockDim.x)
    dst[q] = (D)src[q];
}

// Per-element power-of-two exponents of the double-float kernel's geometric
// factors (df.cuh): bits 0-15 the exponent sG of G, bits 16-31 that of B
// (both signed), 0 while the element's largest magnitude lies in
// [2^-16, 2^16).  One warp per element.
__global__ void df_escale_kernel(const double* __restrict__ G, const double* __restrict__ B,
                                 int P3, int64_t E, int* __restrict__ esc) {
  const int64_t e = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (e >= E) return;                  // whole warps leave together
  double gm = 0.0, bm = 0.0;
  for (int q = lane; q < 6 * P3; q += 32) gm = fmax(gm, fabs(G[e * 6 * P3 + q]));
  for (int q = lane; q < P3; q += 32) bm = fmax(bm, fabs(B[e * P3 + q]));
  for (int o = 16; o > 0; o >>= 1) {
    gm = fmax(gm, __shfl_xor_sync(0xffffffffu, gm, o));
    bm = fmax(bm, __shfl_xor_sync(0xffffffffu, bm, o));
  }
  if (lane == 0) esc[e] = (df_pick_exp(gm) & 0xFFFF) | (df_pick_exp(bm) << 16);
}

// float pairs (hi = RN(x), lo = RN(x - hi), FP64 arithmetic at setup) of
// x = src 2^-s, s the element's exponent in esc (bits 0-15 when shift = 0,
// bits 16-31 when shift = 16), per = values per element
__global__ void split_scaled_kernel(const double* __restrict__ src, float2* __restrict__ dst,
                                    int64_t n, int per, const int* __restrict__ esc, int shift) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int w = esc[q / per];
    const int sc = shift ? (w >> 16) : (int)(short)(w & 0xFFFF);
    const double x = sc ? scalbn(src[q], -sc) : src[q];
    const float hi = __double2float_rn(x);
    dst[q] = make_float2(hi, __double2float_rn(x - (double)hi));
  }
}

template <class D>
__global__ void recip_kernel(const float* __restrict__ src, D* __restrict__ dst, int64_t n) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
       q += (int64_t)gridDim.x * blockDim.x)
    dst[q] = (D)(1.0f / src[q]);
}

template <class S, class D>
static void convert(const S* src, D* dst, int64_t n, cudaStream_t s) {
  int blocks = (int)std::min<int64_t>((n + 255) / 256, 8 * sem_num_sms());
  if (blocks < 1) blocks = 1;
  convert_kernel<S, D><<<blocks, 256, 0, s>>>(src, dst, n);
  SEM_CHECK_LAUNCH();
}

static int grid_for(int64_t n, int threads = 256) {
  int64_t b = (n + threads - 1) / threads;
  return (int)std::max<int64_t>(1, std::min<int64_t>(b, 16 * sem_num_sms()));
}

// ------------------------------------------------------------------ topology (host)
// Multiplicity factor of one lattice coordinate (2 on an interior interface)
static inline int mult1(int64_t ind, int N, int nel) {
  return (ind % N == 0 && ind > 0 && ind < (int64_t)N * nel) ? 2 : 1;
}

static bool masked_at(const sem_handle* h, int64_t ix, int64_t iy, int64_t iz) {
  const int64_t gx = (int64_t)h->N * h->nelx + 1, gy = (int64_t)h->N * h->nely + 1;
  const int64_t gz = (int64_t)h->N * h->nelz + 1;
  const int f = h->faces;
  return ((f & SEM_FACE_XMIN) && ix == 0) || ((f & SEM_FACE_XMAX) && ix == gx - 1) ||
         ((f & SEM_FACE_YMIN) && iy == 0) || ((f & SEM_FACE_YMAX) && iy == gy - 1) ||
         ((f & SEM_FACE_ZMIN) && iz == 0) || ((f & SEM_FACE_ZMAX) && iz == gz - 1);
}

// Dirichlet points owned by a single element: only boundary elements can hold one.
static void build_masked_free(sem_handle* h, cudaStream_t s) {
  const int N = h->N, P = h->P, P3 = h->P3;
  std::vector<int> idx;
  for (int ez = 0; ez < h->nelz; ++ez)
    for (int ey = 0; ey < h->nely; ++ey)
      for (int ex = 0; ex < h->nelx; ++ex) {
        if (ex > 0 && ex < h->nelx - 1 && ey > 0 && ey < h->nely - 1 && ez > 0 && ez < h->nelz - 1)
          continue;
        const int64_t e = ex + (int64_t)h->nelx * (ey + (int64_t)h->nely * ez);
        for (int k = 0; k < P; ++k)
          for (int j = 0; j < P; ++j)
            for (int i = 0; i < P; ++i) {
              const int64_t ix = (int64_t)N * ex + i, iy = (int64_t)N * ey + j;
              const int64_t iz = (int64_t)N * ez + k;
              if (!masked_at(h, ix, iy, iz)) continue;
              if (mult1(ix, N, h->nelx) * mult1(iy, N, h->nely) * mult1(iz, N, h->nelz) != 1)
                continue;
              idx.push_back((int)(e * P3 + (k * P + j) * P + i));
            }
      }
  std::sort(idx.begin(), idx.end());
  h->nmasked_free = (int64_t)idx.size();
  if (!idx.empty()) {
    h->masked_free_idx.alloc(idx.size());
    h->masked_free_idx.upload(idx.data(), idx.size(), s);
    SEM_CUDA(cudaStreamSynchronize(s));
  }
}

}  // namespace sem

// Segments of local points sharing a global number (§3.2: local indices grouped
// per global id), ordered by global number, local indices ascending inside a
// segment, unmasked segments first; plus the list of all Dirichlet points.
// Built on first use of the segment-list gather-scatter.
void sem_build_segments(sem_handle* h, cudaStream_t s) {
  using namespace sem;
  if (h->segments_built) return;
  const int N = h->N, P = h->P, P3 = h->P3;
  const int64_t gx = (int64_t)N * h->nelx + 1, gy = (int64_t)N * h->nely + 1;
  const int64_t nL = h->nL, nG = h->nG;
  std::vector<int64_t> gid(nL);
  std::vector<uint8_t> mask(nL);
  for (int64_t e = 0; e < h->E; ++e) {
    const int ex = (int)(e % h->nelx), ey = (int)((e / h->nelx) % h->nely);
    const int ez = (int)(e / ((int64_t)h->nelx * h->nely));
    for (int k = 0; k < P; ++k)
      for (int j = 0; j < P; ++j)
        for (int i = 0; i < P; ++i) {
          const int64_t q = e * P3 + (k * P + j) * P + i;
          const int64_t ix = (int64_t)N * ex + i, iy = (int64_t)N * ey + j, iz = (int64_t)N * ez + k;
          gid[q] = ix + gx * (iy + gy * iz);
          mask[q] = masked_at(h, ix, iy, iz) ? 0 : 1;
        }
  }
  std::vector<int> count(nG, 0);
  std::vector<uint8_t> gmask(nG, 1);
  for (int64_t q = 0; q < nL; ++q) {
    count[gid[q]]++;
    if (!mask[q]) gmask[gid[q]] = 0;
  }
  std::vector<int> segid(nG, -1);
  int64_t nseg = 0;
  for (int pass = 0; pass < 2; ++pass) {
    for (int64_t g = 0; g < nG; ++g) {
      if (count[g] < 2) continue;
      const bool masked = gmask[g] == 0;
      if ((pass == 0) == masked) continue;
      segid[g] = (int)nseg++;
    }
    if (pass == 0) h->nseg_free = nseg;
  }
  h->nseg_all = nseg;
  std::vector<int> seg_ptr(nseg + 1, 0);
  for (int64_t g = 0; g < nG; ++g)
    if (segid[g] >= 0) seg_ptr[segid[g] + 1] = count[g];
  for (int64_t q = 0; q < nseg; ++q) seg_ptr[q + 1] += seg_ptr[q];
  std::vector<int> seg_idx(seg_ptr[nseg], 0);
  std::vector<int> fill(seg_ptr.begin(), seg_ptr.end() - 1);
  std::vector<int> masked_idx;
  for (int64_t q = 0; q < nL; ++q) {
    const int sg = segid[gid[q]];
    if (sg >= 0) seg_idx[fill[sg]++] = (int)q;
    if (!mask[q]) masked_idx.push_back((int)q);
  }
  h->nmasked = (int64_t)masked_idx.size();
  h->seg_ptr.alloc(seg_ptr.size());
  h->seg_ptr.upload(seg_ptr.data(), seg_ptr.size(), s);
  if (!seg_idx.empty()) {
    h->seg_idx.alloc(seg_idx.size());
    h->seg_idx.upload(seg_idx.data(), seg_idx.size(), s);
  }
  if (!masked_idx.empty()) {
    h->masked_idx.alloc(masked_idx.size());
    h->masked_idx.upload(masked_idx.data(), masked_idx.size(), s);
  }
  SEM_CUDA(cudaStreamSynchronize(s));
  h->segments_built = 1;
}

namespace sem {
}  // namespace sem

using namespace sem;

extern "C" const char* sem_last_error(void) { return g_last_error.c_str(); }

// The library drives one CUDA device per process: per-order constant tables
// and kernel attributes are set up once.  The first sem_setup binds the
// device current at that call; a later one on another device is refused.
static std::atomic<int> g_bound_device{-1};
static std::atomic<int> g_num_sms{0};

int sem::sem_num_sms() { return g_num_sms.load(std::memory_order_relaxed); }

extern "C" sem_status sem_setup(const sem_mesh_desc* mesh, int N, int precision_flags,
                                void* stream, sem_handle** out) {
  return guarded("sem_setup", [&] {
    SEM_REQUIRE(mesh && out, "sem_setup: null mesh or out");
    *out = nullptr;
    SEM_REQUIRE(N >= 1 && N <= kMaxN, "sem_setup: N must be in [1, 10]");
    SEM_REQUIRE(mesh->nelx >= 1 && mesh->nely >= 1 && mesh->nelz >= 1,
                "sem_setup: element counts must be >= 1");
    SEM_REQUIRE((precision_flags & (SEM_PREC_F64 | SEM_PREC_F32)) != 0,
                "sem_setup: precision_flags selects no precision");
    SEM_REQUIRE(mesh->len[0] > 0 && mesh->len[1] > 0 && mesh->len[2] > 0,
                "sem_setup: box lengths must be positive");
    SEM_REQUIRE((double)mesh->nelx * mesh->nely * mesh->nelz * (N + 1) * (N + 1) * (N + 1) <
                    (double)INT32_MAX,
                "sem_setup: more than 2^31 local points");
    // arguments first (no CUDA call above this line), then the device
    int dev = -1;
    SEM_CUDA(cudaGetDevice(&dev));
    int bound = -1;
    if (!g_bound_device.compare_exchange_strong(bound, dev) && bound != dev)
      throw Error(SEM_ERR_STATE, "sem_setup: the library drives one CUDA device per process "
                                 "(bound to device " + std::to_string(bound) + ", current " +
                                 std::to_string(dev) + ")");
    if (g_num_sms.load(std::memory_order_relaxed) == 0) {
      int sms = 0;
      SEM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
      SEM_REQUIRE(sms > 0, "sem_setup: the device reports no SMs");
      g_num_sms.store(sms, std::memory_order_relaxed);
    }
    cudaStream_t s = (cudaStream_t)stream;
    std::unique_ptr<sem_handle> h(new sem_handle());
    h->N = N;
    h->P = N + 1;
    h->P3 = h->P * h->P * h->P;
    h->nelx = mesh->nelx; h->nely = mesh->nely; h->nelz = mesh->nelz;
    h->E = (int64_t)mesh->nelx * mesh->nely * mesh->nelz;
    h->nL = h->E * h->P3;
    SEM_REQUIRE(h->nL < (int64_t)INT32_MAX, "sem_setup: more than 2^31 local points");
    h->prec_flags = precision_flags | SEM_PREC_F64;   // FP64 geometry is always kept
    h->faces = mesh->dirichlet_faces & SEM_FACE_ALL;
    for (int d = 0; d < 3; ++d) h->len[d] = mesh->len[d];
    h->tune.ax32_variant = h->P <= 4 ? 2 : 1;     // 3 stages for small elements, else 2
    gll_host(N, h->xi, h->wq, h->Dh);

    const int64_t nL = h->nL;
    const int P = h->P;
    h->nG = ((int64_t)N * h->nelx + 1) * ((int64_t)N * h->nely + 1) * ((int64_t)N * h->nelz + 1);
    h->gid.alloc(nL);
    h->imult.alloc(nL);
    h->mask.alloc(nL);
    topo_kernel<<<grid_for(nL), 256, 0, s>>>(N, h->nelx, h->nely, h->nelz, h->faces, nL,
                                            h->gid.ptr, h->imult.ptr, h->mask.ptr);
    SEM_CHECK_LAUNCH();
    build_masked_free(h.get(), s);

    DevBuf<double> dxi, dwq;
    dxi.alloc(P); dxi.upload(h->xi.data(), P, s);
    dwq.alloc(P); dwq.upload(h->wq.data(), P, s);
    h->f64.D.alloc(P * P); h->f64.D.upload(h->Dh.data(), P * P, s);
    std::vector<float> D32(h->Dh.begin(), h->Dh.end());
    h->f32.D.alloc(P * P); h->f32.D.upload(D32.data(), P * P, s);

    h->coords.alloc(3 * nL);
    double* X = h->coords.ptr;
    double* Y = X + nL;
    double* Z = Y + nL;
    if (mesh->xyz_gll) {
      h->coords.upload(mesh->xyz_gll, 3 * nL, s);
    } else {
      BoxParams bp{mesh->nelx, mesh->nely, P, mesh->x0[0], mesh->x0[1], mesh->x0[2],
                   mesh->len[0] / mesh->nelx, mesh->len[1] / mesh->nely,
                   mesh->len[2] / mesh->nelz, mesh->deform_amp};
      box_coords_kernel<<<grid_for(nL), 256, 0, s>>>(bp, dxi.ptr, nL, X, Y, Z);
      SEM_CHECK_LAUNCH();
    }
    h->f64.G.alloc(6 * nL);
    h->f64.B.alloc(nL);
    const bool keep32 = (h->prec_flags & SEM_PREC_F32) != 0;
    if (keep32) { h->f32.G.alloc(6 * nL); h->f32.B.alloc(nL); }
    DevBuf<int> bad;
    bad.alloc(1);
    SEM_CUDA(cudaMemsetAsync(bad.ptr, 0, sizeof(int), s));
    geom_kernel<<<grid_for(nL), 256, 0, s>>>(P, nL, h->f64.D.ptr, dwq.ptr, X, Y, Z,
                                             h->f64.G.ptr, h->f64.B.ptr,
                                             keep32 ? h->f32.G.ptr : nullptr,
                                             keep32 ? h->f32.B.ptr : nullptr, bad.ptr);
    SEM_CHECK_LAUNCH();
    int hbad = 0;
    SEM_CUDA(cudaMemcpyAsync(&hbad, bad.ptr, sizeof(int), cudaMemcpyDeviceToHost, s));
    SEM_CUDA(cudaStreamSynchronize(s));
    SEM_REQUIRE(!hbad, "sem_setup: element map has detJ <= 0 at some GLL point");
    if (P == 6 || P == 8 || P == 10) {
      // float-pair copies of G and B for the double-float FP64 kernel
      // (normalised per element where needed, see df.cuh)
      h->gdf.alloc(6 * nL);
      h->bdf.alloc(nL);
      h->escale.alloc(h->E);
      df_escale_kernel<<<(unsigned)((h->E + 7) / 8), 256, 0, s>>>(h->f64.G.ptr, h->f64.B.ptr,
                                                                  h->P3, h->E, h->escale.ptr);
      SEM_CHECK_LAUNCH();
      split_scaled_kernel<<<grid_for(6 * nL), 256, 0, s>>>(h->f64.G.ptr, h->gdf.ptr, 6 * nL,
                                                            6 * h->P3, h->escale.ptr, 0);
      SEM_CHECK_LAUNCH();
      split_scaled_kernel<<<grid_for(nL), 256, 0, s>>>(h->f64.B.ptr, h->bdf.ptr, nL, h->P3,
                                                        h->escale.ptr, 16);
      SEM_CHECK_LAUNCH();
      df_prepare(h.get());
    }
    if (h->f64.G.ptr) eo_prepare(h.get());
    noalloc_prepare();
    h->dev_err.alloc(1);
    SEM_CUDA(cudaMemsetAsync(h->dev_err.ptr, 0, sizeof(int), s));
    h->state.alloc(4);
    SEM_CUDA(cudaMemsetAsync(h->state.ptr, 0, 4 * sizeof(CGState), s));
    h->partials.alloc(6 * kRedBlocks + kFusedPartials);
    SEM_CUDA(cudaStreamSynchronize(s));
    *out = h.release();
  });
}

extern "C" sem_status sem_destroy(sem_handle* h) {
  return guarded("sem_destroy", [&] {
    if (!h) return;
    cudaDeviceSynchronize();
    delete h;
  });
}

extern "C" sem_status sem_get_sizes(const sem_handle* h, int64_t* n_local, int64_t* n_global,
                                    int* N, int64_t* E) {
  return guarded("sem_get_sizes", [&] {
    SEM_REQUIRE(h, "sem_get_sizes: null handle");
    if (n_local) *n_local = h->nL;
    if (n_global) *n_global = h->nG;
    if (N) *N = h->N;
    if (E) *E = h->E;
  });
}

extern "C" sem_status sem_get_field(sem_handle* h, int which, void* dst, int dtype,
                                    void* stream) {
  return guarded("sem_get_field", [&] {
    SEM_REQUIRE(h && dst, "sem_get_field: null handle or dst");
    SEM_REQUIRE(dtype == SEM_F64 || dtype == SEM_F32, "sem_get_field: bad dtype");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t nL = h->nL;
    auto put_d = [&](const double* src, int64_t n) {
      if (dtype == SEM_F64)
        SEM_CUDA(cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
      else
        convert(src, (float*)dst, n, s);
    };
    auto put_f = [&](const float* src, int64_t n) {
      if (dtype == SEM_F32)
        SEM_CUDA(cudaMemcpyAsync(dst, src, n * sizeof(float), cudaMemcpyDeviceToDevice, s));
      else
        convert(src, (double*)dst, n, s);
    };
    switch (which) {
      case SEM_FIELD_X: put_d(h->coords.ptr, nL); break;
      case SEM_FIELD_Y: put_d(h->coords.ptr + nL, nL); break;
      case SEM_FIELD_Z: put_d(h->coords.ptr + 2 * nL, nL); break;
      case SEM_FIELD_G:
        if (dtype == SEM_F32 && h->f32.G.ptr) put_f(h->f32.G.ptr, 6 * nL);
        else put_d(h->f64.G.ptr, 6 * nL);
        break;
      case SEM_FIELD_B:
        if (dtype == SEM_F32 && h->f32.B.ptr) put_f(h->f32.B.ptr, nL);
        else put_d(h->f64.B.ptr, nL);
        break;
      case SEM_FIELD_MULT:
        // multiplicity = 1 / imult, exact for powers of two
        if (dtype == SEM_F64) recip_kernel<double><<<grid_for(nL), 256, 0, s>>>(h->imult.ptr, (double*)dst, nL);
        else recip_kernel<float><<<grid_for(nL), 256, 0, s>>>(h->imult.ptr, (float*)dst, nL);
        SEM_CHECK_LAUNCH();
        break;
      case SEM_FIELD_MASK: {
        DevBuf<float> tmp;
        tmp.alloc(nL);
        convert(h->mask.ptr, tmp.ptr, nL, s);
        put_f(tmp.ptr, nL);
        SEM_CUDA(cudaStreamSynchronize(s));
        break;
      }
      case SEM_FIELD_GID:
        SEM_CUDA(cudaMemcpyAsync(dst, h->gid.ptr, nL * sizeof(int64_t),
                                 cudaMemcpyDeviceToDevice, s));
        break;
      case SEM_FIELD_DINV:
        if (!h->dinv_valid) throw Error(SEM_ERR_STATE, "sem_get_field: no solve has run yet");
        if (dtype == SEM_F32 && h->f32.dinv.ptr) put_f(h->f32.dinv.ptr, nL);
        else put_d(h->f64.dinv.ptr, nL);
        break;
      default:
        throw Error(SEM_ERR_ARG, "sem_get_field: unknown field");
    }
  });
}

extern "C" sem_status sem_sync(sem_handle* h, void* stream) {
  return guarded("sem_sync", [&] {
    SEM_REQUIRE(h, "sem_sync: null handle");
    cudaStream_t s = (cudaStream_t)stream;
    int herr = 0;
    SEM_CUDA(cudaMemcpyAsync(&herr, h->dev_err.ptr, sizeof(int), cudaMemcpyDeviceToHost, s));
    SEM_CUDA(cudaStreamSynchronize(s));
    if (herr) {
      SEM_CUDA(cudaMemsetAsync(h->dev_err.ptr, 0, sizeof(int), s));
      SEM_CUDA(cudaStreamSynchronize(s));
      throw Error((sem_status)herr,
                  herr == SEM_ERR_TIMEOUT
                      ? "sem_sync: a device wait timed out in an earlier call"
                      : "sem_sync: an earlier call found an index outside its vector");
    }
  });
}

extern "C" sem_status sem_set_f64_kernel(sem_handle* h, int kind) {
  return guarded("sem_set_f64_kernel", [&] {
    SEM_REQUIRE(h, "sem_set_f64_kernel: null handle");
    SEM_REQUIRE(kind == SEM_F64_KERNEL_AUTO || kind == SEM_F64_KERNEL_NATIVE ||
                    kind == SEM_F64_KERNEL_DOUBLEFLOAT,
                "sem_set_f64_kernel: unknown kind");
    if (kind == SEM_F64_KERNEL_DOUBLEFLOAT && !h->gdf.ptr)
      throw Error(SEM_ERR_STATE, "sem_set_f64_kernel: double-float needs N in {5, 7, 9}");
    h->f64_kernel = kind;
  });
}
