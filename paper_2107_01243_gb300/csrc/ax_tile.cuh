// One element of the operator w_e = (h1 D^T G_e D + h2 B_e) u_e (arXiv
// 2107.01243 §2, Eq. 9) on P x P threads from a shared-memory stage, shared
// by the single-problem bulk-copy kernel (ax_tma.cu) and the batched kernel
// (batch.cu).  Thread (i, j) owns the k-column of its (i, j):
//   tile_load      u column -> registers, transposed plane copy -> sT
//   (barrier)
//   tile_forward   r, s, t derivatives (rows of u, rows of sT, the register
//                  column), times G -> swr, swsT (transposed), wt (registers)
//   (barrier; the stage may be refilled)
//   tile_backward  w = D^T-contractions of swr rows, swsT rows and the wt
//                  column (+ h2 B u), stored to global memory
// The transposed planes hold row r = i, column c = j.  For P = 8 floats the
// two 16-byte halves of rows 4-7 are stored swapped and read back in swapped
// order: the row loads of 8 threads (rows 0-7) and the column stores of a
// warp then hit distinct banks, and the values arrive in natural order.
#pragma once
#include "sem_internal.cuh"

namespace sem {

template <int P, class T>
struct DMat {
  T d[P * P];
};

template <int P, class T>
__device__ __forceinline__ void load_row(const T* __restrict__ p, T (&v)[P]) {
  constexpr int bytes = P * (int)sizeof(T);
  if constexpr (bytes % 16 == 0) {
    constexpr int nv = bytes / 16;
    const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
    for (int a = 0; a < nv; ++a) {
      float4 f = q[a];
      const T* t = reinterpret_cast<const T*>(&f);
#pragma unroll
      for (int b = 0; b < 16 / (int)sizeof(T); ++b) v[a * (16 / (int)sizeof(T)) + b] = t[b];
    }
  } else if constexpr (bytes % 8 == 0) {
    constexpr int nv = bytes / 8;
    const float2* q = reinterpret_cast<const float2*>(p);
#pragma unroll
    for (int a = 0; a < nv; ++a) {
      float2 f = q[a];
      const T* t = reinterpret_cast<const T*>(&f);
#pragma unroll
      for (int b = 0; b < 8 / (int)sizeof(T); ++b) v[a * (8 / (int)sizeof(T)) + b] = t[b];
    }
  } else {
#pragma unroll
    for (int a = 0; a < P; ++a) v[a] = p[a];
  }
}

// a row of a transposed plane whose 16-byte halves are stored swapped when
// hs = 4 (P = 8 floats only; hs = 0 otherwise): read back in natural order
template <int P, class T>
__device__ __forceinline__ void load_trow(const T* __restrict__ p, T (&v)[P], int hs) {
  if constexpr (P == 8 && sizeof(T) == 4) {
    const float4 a = *reinterpret_cast<const float4*>(p + hs);
    const float4 b = *reinterpret_cast<const float4*>(p + (hs ^ 4));
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
  } else {
    load_row<P, T>(p, v);
  }
}

template <int P, class T>
struct TileThread {
  int i, j, lt, hs, tpos;
  T Di[P], Dj[P], DiT[P], DjT[P];     // rows i, j of D and of D^T
  // DF: (row, column) -> D entry
  template <class DF>
  __device__ __forceinline__ void init(int lt_, DF D) {
    constexpr bool SWZ = (P == 8 && sizeof(T) == 4);
    lt = lt_;
    i = lt % P;
    j = lt / P;
    hs = SWZ ? 4 * ((i >> 2) & 1) : 0;
    tpos = i * P + (j ^ hs);
#pragma unroll
    for (int l = 0; l < P; ++l) {
      Di[l] = D(i, l);
      Dj[l] = D(j, l);
      DiT[l] = D(l, i);
      DjT[l] = D(l, j);
    }
  }
};

// column of u (and of B, h1 when present) into registers; transposed copy
template <int P, class T>
__device__ __forceinline__ void tile_load(const TileThread<P, T>& t, const T* su, const T* sb,
                                          const T* sh, T h1, T* sT, T (&uc)[P], T (&bk)[P],
                                          T (&ck)[P]) {
  constexpr int P2 = P * P;
#pragma unroll
  for (int k = 0; k < P; ++k) {
    uc[k] = su[k * P2 + t.lt];
    sT[k * P2 + t.tpos] = uc[k];
    bk[k] = sb ? sb[k * P2 + t.lt] : T(0);
    ck[k] = sh ? sh[k * P2 + t.lt] : h1;
  }
}

// derivatives, geometric factors: (swr, swsT, wt) = ck G (ur, us, ut)
template <int P, class T, class DF>
__device__ __forceinline__ void tile_forward(const TileThread<P, T>& t, const T* su, const T* sT,
                                             const T* sg, const T (&uc)[P], const T (&ck)[P],
                                             T* swr, T* swsT, T (&wt)[P], DF D) {
  constexpr int P2 = P * P, P3 = P2 * P;
#pragma unroll
  for (int k = 0; k < P; ++k) {
    T row[P], col[P];
    load_row<P, T>(su + k * P2 + t.j * P, row);
    load_trow<P, T>(sT + k * P2 + t.i * P, col, t.hs);
    T ur = T(0), us = T(0), ut = T(0);
#pragma unroll
    for (int l = 0; l < P; ++l) {
      ur = fma(t.Di[l], row[l], ur);
      us = fma(t.Dj[l], col[l], us);
      ut = fma(D(k, l), uc[l], ut);
    }
    const int q = k * P2 + t.lt;
    const T g11 = sg[q], g22 = sg[P3 + q], g33 = sg[2 * P3 + q];
    const T g12 = sg[3 * P3 + q], g13 = sg[4 * P3 + q], g23 = sg[5 * P3 + q];
    const T c = ck[k];
    swr[k * P2 + t.j * P + t.i] = c * (g11 * ur + g12 * us + g13 * ut);
    swsT[k * P2 + t.tpos] = c * (g12 * ur + g22 * us + g23 * ut);
    wt[k] = c * (g13 * ur + g23 * us + g33 * ut);
  }
}

// transposed contractions (+ h2 B u); store(k, value) receives the output of
// point (i, j, k)
template <int P, class T, class DF, class ST>
__device__ __forceinline__ void tile_backward(const TileThread<P, T>& t, const T* swr,
                                              const T* swsT, const T (&wt)[P], const T (&uc)[P],
                                              const T (&bk)[P], T h2, bool helm, DF D,
                                              ST store) {
  constexpr int P2 = P * P;
#pragma unroll
  for (int k = 0; k < P; ++k) {
    T row[P], col[P];
    load_row<P, T>(swr + k * P2 + t.j * P, row);
    load_trow<P, T>(swsT + k * P2 + t.i * P, col, t.hs);
    T acc = T(0);
#pragma unroll
    for (int l = 0; l < P; ++l) {
      acc = fma(t.DiT[l], row[l], acc);
      acc = fma(t.DjT[l], col[l], acc);
      acc = fma(D(l, k), wt[l], acc);
    }
    if (helm) acc = fma(h2 * bk[k], uc[k], acc);
    store(k, acc);
  }
}

// Box position of element e and the Dirichlet faces, for the operator kernels
// that apply the mask and sum x-neighbour pairs themselves (apply.cu).
struct FuseBox {
  int nelx, nely, nelz, faces;
};

// Elements per segment of the fused operator: a CTA takes segments of
// kFuseSeg consecutive elements, segment g = blockIdx.x + m gridDim.x, so
// that the x-neighbour pairs inside a segment are summed in the CTA while all
// CTAs together stream one contiguous window of memory (whole per-CTA ranges
// spread the streams over the address space and ran 25-45% slower).
constexpr int kFuseSeg = 4;

// The items a persistent CTA walks: blockIdx.x + m gridDim.x, or (SEG) the
// items of its segments in order
template <bool SEG>
struct ItemSeq {
  int n;   // number of items
  __device__ __forceinline__ int first() const {
    return SEG ? (int)blockIdx.x * kFuseSeg : (int)blockIdx.x;
  }
  __device__ __forceinline__ int next(int it) const {
    if (!SEG) return it + (int)gridDim.x;
    const int nx = it + 1;
    if (nx % kFuseSeg != 0 && nx < n) return nx;
    return (it / kFuseSeg + (int)gridDim.x) * kFuseSeg;
  }
};

// box position of the elements a CTA walks in order: set at the start of a
// segment, then stepped (no divisions per element)
struct BoxWalk {
  int ex, ey, ez;
  __device__ __forceinline__ void start(int e, const FuseBox& b) {
    ex = e % b.nelx;
    const int r = e / b.nelx;
    ey = r % b.nely;
    ez = r / b.nely;
  }
  __device__ __forceinline__ void step(const FuseBox& b) {
    if (++ex == b.nelx) {
      ex = 0;
      if (++ey == b.nely) {
        ey = 0;
        ++ez;
      }
    }
  }
};

// The fused output of one element e: masked points are zeroed, and when the
// element before it (e - 1, the -x neighbour) came just before in the same
// segment of the same CTA, each point of the i = 0 face is summed with e - 1's
// copy at i = N (lower element first), read back from w where e - 1's threads
// stored it before the CTA's last barrier, and the sum goes to both copies.
// FusedStore flags of element e at the walk's box position: bit 0 pairs it
// with e - 1 (same segment, not the first of an x-row), bits 2-7 its faces on
// Dirichlet boundaries (XMIN, XMAX, YMIN, YMAX, ZMIN, ZMAX)
__device__ __forceinline__ unsigned fused_flags(int e, const BoxWalk& bw, const FuseBox& b) {
  unsigned fl = (bw.ex > 0 && e % kFuseSeg != 0) ? 1u : 0u;
  if (b.faces) {
    fl |= ((b.faces & SEM_FACE_XMIN) && bw.ex == 0 ? 4u : 0u) |
          ((b.faces & SEM_FACE_XMAX) && bw.ex == b.nelx - 1 ? 8u : 0u) |
          ((b.faces & SEM_FACE_YMIN) && bw.ey == 0 ? 16u : 0u) |
          ((b.faces & SEM_FACE_YMAX) && bw.ey == b.nely - 1 ? 32u : 0u) |
          ((b.faces & SEM_FACE_ZMIN) && bw.ez == 0 ? 64u : 0u) |
          ((b.faces & SEM_FACE_ZMAX) && bw.ez == b.nelz - 1 ? 128u : 0u);
  }
  return fl;
}

template <int P, class T>
struct FusedStore {
  T* we;             // this element's output
  unsigned fl;       // fused_flags of the element
  __device__ __forceinline__ void store(int i, int j, int k, T v) const {
    constexpr int P2 = P * P, P3 = P2 * P, N = P - 1;
    if (fl & 0xFCu) {                 // element on a Dirichlet face (uniform branch)
      const unsigned pf = (i == 0 ? 4u : 0u) | (i == N ? 8u : 0u) | (j == 0 ? 16u : 0u) |
                          (j == N ? 32u : 0u) | (k == 0 ? 64u : 0u) | (k == N ? 128u : 0u);
      if (pf & fl) v = T(0);
    }
    const int idx = k * P2 + j * P + i;
    if ((fl & 1u) && i == 0) {
      const T sum = we[idx - P3 + N] + v;
      we[idx - P3 + N] = sum;
      v = sum;
    }
    we[idx] = v;
  }
};

}  // namespace sem
