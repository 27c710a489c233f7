// Index-free gather-scatter QQ^T for the structured box (arXiv 2107.01243
// §2, Eq. 10; §3.2).  The box topology fixes every shared global point's
// copies, so no index lists are read: one thread per shared lattice point
// computes the local indices of its 2, 4 or 8 copies, sums them in increasing
// local index (increasing element number: owner, +x, +y, +x+y, +z, ...),
// exactly the order of the segment-list kernel, and writes the sum back.
//
// Shared lattice points are split into three disjoint sets enumerated so that
// consecutive threads touch consecutive memory where the layout allows it:
//   SX  x-interface points (any y, z), y fastest
//   SY  y-interface points with non-interface x (any z), x fastest
//   SZ  z-interface points with non-interface x and y, x fastest
// With the mask applied, shared Dirichlet points are zeroed instead of summed
// and the unshared Dirichlet points (a short precomputed list) are zeroed.
#include "sem_internal.cuh"

namespace sem {

struct BoxDims {
  int nelx, nely, nelz;
  int gx, gy, gz;            // lattice extents N nel + 1
  int nix, niy;              // non-interface lattice coordinates in x, y
  int faces;                 // Dirichlet faces (mask applied) or 0
  uint32_t nSX, nSY, nSZ;    // set sizes
  FastDiv dgy, dnx1, dny1, dnix, dniy;
};

// lattice coordinate -> (element coordinate, local index); for interface
// coordinates this is the lower element (local index N)
template <int N>
__device__ __forceinline__ void lat2el(int c, int nel, int& ec, int& lc) {
  ec = c / N;
  if (ec >= nel) ec = nel - 1;
  lc = c - ec * N;
  if (lc == 0 && ec > 0) {
    --ec;
    lc = N;
  }
}

__device__ __forceinline__ bool on_mask(const BoxDims& d, int ix, int iy, int iz) {
  return ((d.faces & SEM_FACE_XMIN) && ix == 0) || ((d.faces & SEM_FACE_XMAX) && ix == d.gx - 1) ||
         ((d.faces & SEM_FACE_YMIN) && iy == 0) || ((d.faces & SEM_FACE_YMAX) && iy == d.gy - 1) ||
         ((d.faces & SEM_FACE_ZMIN) && iz == 0) || ((d.faces & SEM_FACE_ZMAX) && iz == d.gz - 1);
}

template <int N, class T>
__device__ __forceinline__ void sum_point(T* __restrict__ w, const BoxDims& d, int ix, int iy,
                                          int iz) {
  constexpr int P = N + 1;
  constexpr long long P3 = (long long)P * P * P;
  int ex, i, ey, j, ez, k;
  lat2el<N>(ix, d.nelx, ex, i);
  lat2el<N>(iy, d.nely, ey, j);
  lat2el<N>(iz, d.nelz, ez, k);
  // interface directions: the copy on the + side has local index 0
  const bool fx = (i == N) && (ex < d.nelx - 1);
  const bool fy = (j == N) && (ey < d.nely - 1);
  const bool fz = (k == N) && (ez < d.nelz - 1);
  const long long e0 = (long long)ex + (long long)d.nelx * (ey + (long long)d.nely * ez);
  const long long sx = P3, sy = (long long)d.nelx * P3, sz = (long long)d.nelx * d.nely * P3;
  // the (up to) eight copies c = cx + 2 cy + 4 cz in increasing element order,
  // all loaded before any is added (one memory round trip per point)
  long long idx[8];
  bool has[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const int cx = c & 1, cy = (c >> 1) & 1, cz = c >> 2;
    has[c] = (!cx || fx) && (!cy || fy) && (!cz || fz);
    const int li = cx ? 0 : i, lj = cy ? 0 : j, lk = cz ? 0 : k;
    idx[c] = e0 * P3 + cx * sx + cy * sy + cz * sz + (lk * P + lj) * P + li;
  }
  if (d.faces && on_mask(d, ix, iy, iz)) {
#pragma unroll
    for (int c = 0; c < 8; ++c)
      if (has[c]) w[idx[c]] = T(0);
    return;
  }
  T v[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) v[c] = has[c] ? w[idx[c]] : T(0);
  // FP64: the adds of copies that no lane of the warp has are skipped as a
  // whole (warp-uniform branches): FP64 adds run at 1/64 of the FP32 rate on
  // this GPU, and a predicated add still occupies the pipe (FP32 adds are
  // cheaper than the votes)
  bool ax = true, ay = true, az = true;
  if constexpr (sizeof(T) == 8) {
    const unsigned am = __activemask();
    ax = __any_sync(am, fx);
    ay = __any_sync(am, fy);
    az = __any_sync(am, fz);
  }
  T s = v[0];
  if (ax && has[1]) s += v[1];
  if (ay) {
    if (has[2]) s += v[2];
    if (ax && has[3]) s += v[3];
  }
  if (az) {
#pragma unroll
    for (int c = 4; c < 8; ++c)
      if (has[c]) s += v[c];
  }
#pragma unroll
  for (int c = 0; c < 8; ++c)
    if (has[c]) w[idx[c]] = s;
}

// m-th lattice coordinate that is not an interior element interface:
// 0, then 1..N-1, N+1..2N-1, ... inside the elements, then the last one
template <int N>
__device__ __forceinline__ int free_coord(int m, int nfree, int g) {
  if (m == 0) return 0;
  if (m == nfree - 1) return g - 1;
  constexpr int M = N > 1 ? N - 1 : 1;      // N = 1 has no interior coordinates
  const int q = m - 1;
  return q / M * N + 1 + q % M;
}

template <int N, class T>
__global__ void __launch_bounds__(256)
dssum_box_kernel(T* __restrict__ w, BoxDims d, const int* __restrict__ masked, int nmasked,
                 const CGState* __restrict__ st) {
  if (st && st->done) return;
  const uint32_t total = d.nSX + d.nSY + d.nSZ + (uint32_t)nmasked;
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += gridDim.x * blockDim.x) {
    uint32_t r = t;
    if (r < d.nSX) {
      // (iz, a, iy) with iy fastest
      const uint32_t r1 = d.dgy.div(r);
      const int iy = (int)(r - r1 * d.gy);
      const uint32_t r2 = d.dnx1.div(r1);
      const int a = (int)(r1 - r2 * (uint32_t)(d.nelx - 1));
      sum_point<N, T>(w, d, (a + 1) * N, iy, (int)r2);
      continue;
    }
    r -= d.nSX;
    if (r < d.nSY) {
      // (iz, b, x') with x' over non-interface x coordinates, fastest
      const uint32_t r1 = d.dnix.div(r);
      const int xp = (int)(r - r1 * d.nix);
      const uint32_t r2 = d.dny1.div(r1);
      const int b = (int)(r1 - r2 * (uint32_t)(d.nely - 1));
      sum_point<N, T>(w, d, free_coord<N>(xp, d.nix, d.gx), (b + 1) * N, (int)r2);
      continue;
    }
    r -= d.nSY;
    if (r < d.nSZ) {
      const uint32_t r1 = d.dnix.div(r);
      const int xp = (int)(r - r1 * d.nix);
      const uint32_t r2 = d.dniy.div(r1);
      const int yp = (int)(r1 - r2 * d.niy);
      sum_point<N, T>(w, d, free_coord<N>(xp, d.nix, d.gx), free_coord<N>(yp, d.niy, d.gy),
                      ((int)r2 + 1) * N);
      continue;
    }
    r -= d.nSZ;
    w[masked[r]] = T(0);
  }
}

template <int N, class T>
static void launch_box_n(const BoxDims& d, T* w, const int* masked, int nm, const CGState* st,
                         cudaStream_t s) {
  const uint32_t total = d.nSX + d.nSY + d.nSZ + (uint32_t)nm;
  const int blocks = (int)std::min<long long>((total + 255) / 256, 32LL * sem_num_sms());
  dssum_box_kernel<N, T><<<blocks, 256, 0, s>>>(w, d, masked, nm, st);
  SEM_CHECK_LAUNCH();
}

template <class T>
void launch_dssum_box(const sem_handle* h, T* w, bool apply_mask, const CGState* st,
                      cudaStream_t s) {
  BoxDims d;
  const int N = h->N;
  d.nelx = h->nelx;
  d.nely = h->nely;
  d.nelz = h->nelz;
  d.gx = N * d.nelx + 1;
  d.gy = N * d.nely + 1;
  d.gz = N * d.nelz + 1;
  d.nix = d.gx - (d.nelx - 1);
  d.niy = d.gy - (d.nely - 1);
  d.faces = apply_mask ? h->faces : 0;
  const long long nSX = (long long)(d.nelx - 1) * d.gy * d.gz;
  const long long nSY = (long long)(d.nely - 1) * d.nix * d.gz;
  const long long nSZ = (long long)(d.nelz - 1) * d.nix * d.niy;
  const int nm = apply_mask ? (int)h->nmasked_free : 0;
  if (nSX + nSY + nSZ + nm >= (1LL << 31))
    throw Error(SEM_ERR_ARG, "box gather-scatter: more than 2^31 shared points");
  d.nSX = (uint32_t)nSX;
  d.nSY = (uint32_t)nSY;
  d.nSZ = (uint32_t)nSZ;
  d.dgy = FastDiv((uint32_t)d.gy);
  d.dnx1 = FastDiv((uint32_t)std::max(1, d.nelx - 1));
  d.dny1 = FastDiv((uint32_t)std::max(1, d.nely - 1));
  d.dnix = FastDiv((uint32_t)d.nix);
  d.dniy = FastDiv((uint32_t)d.niy);
  if (nSX + nSY + nSZ + nm == 0) return;
  const int* mk = h->masked_free_idx.ptr;
  switch (N) {
    case 1: launch_box_n<1, T>(d, w, mk, nm, st, s); break;
    case 2: launch_box_n<2, T>(d, w, mk, nm, st, s); break;
    case 3: launch_box_n<3, T>(d, w, mk, nm, st, s); break;
    case 4: launch_box_n<4, T>(d, w, mk, nm, st, s); break;
    case 5: launch_box_n<5, T>(d, w, mk, nm, st, s); break;
    case 6: launch_box_n<6, T>(d, w, mk, nm, st, s); break;
    case 7: launch_box_n<7, T>(d, w, mk, nm, st, s); break;
    case 8: launch_box_n<8, T>(d, w, mk, nm, st, s); break;
    case 9: launch_box_n<9, T>(d, w, mk, nm, st, s); break;
    case 10: launch_box_n<10, T>(d, w, mk, nm, st, s); break;
    default: throw Error(SEM_ERR_ARG, "box gather-scatter: unsupported order");
  }
}

template void launch_dssum_box<double>(const sem_handle*, double*, bool, const CGState*,
                                       cudaStream_t);
template void launch_dssum_box<float>(const sem_handle*, float*, bool, const CGState*,
                                      cudaStream_t);

}  // namespace sem
