// Batched solves: many independent Helmholtz problems of uneven element count
// and order N advance together, FP32-inner PCG inside FP64 refinement per
// problem (the solver of cg.cu, arXiv 2107.01243 §2 end and §4, applied to a
// batch).  Every stage of an inner CG iteration is one launch over all
// problems (per order class for the element kernels).  By default (every
// handle allows global vectors) the inner PCG runs on global vectors:
//   bglob   per order class, a persistent element kernel that gathers u from
//           each problem's lattice and adds face values to its w by L2
//           reductions (batch_glob.cuh), forming <p, H p> at P = 8
//   bginit, bgpw, bgupdate, bgpupd  per-problem-chunk vector kernels
// On L-vectors (SEM_INNER_LOCAL on a handle) the stages are:
//   bax     persistent bulk-copy (TMA) Ax over all elements of the problems of
//           one order (one launch per order present, each with the tile and
//           shared-memory stages of its own order)
//   bdssum  index-free gather-scatter over all problems' shared points
// or, when every order runs one element per CTA (N = 5, 7, 9), the assembled
// operator with the gather-scatter split by direction (batch_apply.cuh):
//   bapply  per order class, the element kernel summing x-neighbour pairs
//           inside segments of four elements and zeroing masked points
//   bcut, bsy, bsz  per class, x-pairs between segments, y- and z-pairs
//   bpw, bupdate, bpupd  vector updates over fixed-size chunks; the chunk
//           partial sums of one problem are reduced, in a fixed order, by the
//           last chunk block to finish (a ticket per problem)
// Converged problems are skipped by every stage.  A batch of iterations is
// captured in a CUDA graph; after each graph launch the host reads the
// problems' states and, for every problem whose inner solve finished, applies
// the correction, computes the FP64 residual and restarts its inner solve,
// so problems move through their refinement steps independently.
#include <cmath>
#include <memory>
#include <vector>

#include "sem_internal.cuh"
#include "tma.cuh"
#include "reduce.cuh"
#include "cg_state.cuh"
#include "ax_tile.cuh"

namespace sem {

constexpr int kMaxBatch = 256;
constexpr int kChunk = 65536;          // points per vector work item
constexpr int kGChunk = 16384;         // values per global-vector work item

// batched Ax tile per order: K elements of P^2 threads each per work item
template <int P>
struct BaxCfg {
  static constexpr int K = (64 / (P * P)) > 1 ? (64 / (P * P)) : 1;
  static constexpr int THREADS = K * P * P;
  static constexpr int STAGES = P >= 10 ? 1 : 2;     // P = 10: more CTAs per SM
  // stages, work arrays, then one ClsProb per problem of the class
  static constexpr size_t smem(int ncls) {
    return 128 + (size_t)(STAGES * 8 + 3) * K * P * P * P * sizeof(float) +
           (size_t)ncls * 48;
  }
};

// what the batched Ax reads of one problem, copied to shared memory per CTA
struct ClsProb {
  const float* p;
  const float* G;
  const float* B;
  float* w;
  int E;
  float h1, h2;
  int pad;
};
static_assert(sizeof(ClsProb) == 48, "ClsProb layout");

__constant__ float c_b32_D[kMaxP + 1][kMaxP * kMaxP];   // FP32 D of every order

struct BProb {
  const float* G;
  const float* B;
  const float* dinv;
  const float* imult;
  float* x;
  float* r;
  float* p;
  float* w;
  float h1, h2;
  int N, P, E, nelx, nely, nelz, faces;
  long long nL;
  CGState* st;
  long long e_off;       // first flat element
  int cls;               // index of the problem's order class
  long long d_off;       // first flat gather-scatter item
  int v_off, v_cnt;      // vector chunk items
  int gx, gy, gz, nix, niy;
  unsigned nSX, nSY, nSZ, nmf;
  const int* mfree;
  FastDiv dN, dN1, dgy, dnx1, dny1, dnix, dniy;
  // inner solve on global vectors (n_G padded to nGp, items of kChunk values)
  float *xg, *rg, *pg, *wg;
  const float* dinvg;
  long long nGp;
  int g_off, g_cnt;
  FastDiv dnx, dny;
  double* pwacc;         // <p, H p> accumulated by the element kernel (fused_pw)
  int fused_pw;          // P = 8: the element kernel forms <p, H p>
};

__device__ __forceinline__ int find_prob(const long long* off, int n, long long g) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= g) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Per-block view of the vector work items for one launch: the first item of
// every problem and whether the problem's inner solve is finished, read once;
// a block then steps over a finished problem's items in one jump.
struct ItemWalk {
  int voff[kMaxBatch + 1];
  int done[kMaxBatch];
  __device__ __forceinline__ void load(const BProb* __restrict__ probs, int nprob, int nitems) {
    for (int q = threadIdx.x; q < nprob; q += blockDim.x) {
      voff[q] = probs[q].v_off;
      done[q] = probs[q].st->done;
    }
    if (threadIdx.x == 0) voff[nprob] = nitems;
    __syncthreads();
  }
  // first item at or after it, in steps of stride, whose problem is running
  __device__ __forceinline__ int next(const int* __restrict__ item_prob, int it, int stride,
                                      int nitems) const {
    while (it < nitems) {
      const int pi = item_prob[it];
      if (!done[pi]) break;
      it += (voff[pi + 1] - it + stride - 1) / stride * stride;
    }
    return it;
  }
};

}  // namespace sem

#include "batch_apply.cuh"

namespace sem {

// ---------------------------------------------------------------- batched Ax
// Persistent bulk-copy Ax over every element of the problems of one order P;
// CTAs of K P^2 threads take work items of K consecutive elements of one
// problem and keep STAGES items in flight.
template <int P, int STAGES>
__global__ void __launch_bounds__(BaxCfg<P>::THREADS)
bax_kernel(const BProb* __restrict__ probs, const int* __restrict__ cls_prob,
           const long long* __restrict__ cls_ioff, int ncls, long long Itot,
           int* __restrict__ err, uint64_t timeout_ns) {
  constexpr int K = BaxCfg<P>::K, P3 = P * P * P;
  constexpr int SV = 8 * K * P3;                 // values per stage
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ long long s_off[kMaxBatch];
  __shared__ int s_skip[kMaxBatch];
  __shared__ int s_prob[kMaxBatch];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);
  float* stage0 = reinterpret_cast<float*>(smem_raw + 128);
  float* work = stage0 + STAGES * SV;
  ClsProb* cp = reinterpret_cast<ClsProb*>(work + 3 * K * P3);
  const int tid = threadIdx.x;
  for (int q = tid; q < ncls; q += blockDim.x) {
    s_off[q] = cls_ioff[q];
    s_prob[q] = cls_prob[q];
    const BProb& b = probs[cls_prob[q]];
    s_skip[q] = b.st->done;
    ClsProb c;
    c.p = b.p;
    c.G = b.G;
    c.B = b.B;
    c.w = b.w;
    c.E = b.E;
    c.h1 = b.h1;
    c.h2 = b.h2;
    c.pad = 0;
    cp[q] = c;
  }
  if (tid == 0) {
#pragma unroll
    for (int s = 0; s < STAGES; ++s) mbar_init(&bar[s], 1);
    mbar_fence_init();
  }
  __syncthreads();
  const long long G = gridDim.x;
  // next item of this CTA at or after g whose problem is still running:
  // a finished problem is stepped over in one jump
  auto next = [&](long long g) {
    while (g < Itot) {
      const int c = find_prob(s_off, ncls, g);
      if (!s_skip[c]) break;
      const long long end = c + 1 < ncls ? s_off[c + 1] : Itot;
      g += (end - g + G - 1) / G * G;
    }
    return g;
  };
  auto issue = [&](long long g, int s) {
    const int c = find_prob(s_off, ncls, g);
    const ClsProb& pr = cp[c];
    const long long e0 = (g - s_off[c]) * K;
    const int cnt = (int)min((long long)K, (long long)pr.E - e0);
    const uint32_t FB = (uint32_t)(P3 * cnt) * 4u;
    const bool helm = pr.h2 != 0.0f;
    float* dst = stage0 + s * SV;
    const uint64_t pol = l2_policy_evict_first();   // G and B are read once
    mbar_arrive_expect_tx(&bar[s], (helm ? 8u : 7u) * FB);
    bulk_g2s(dst, pr.p + e0 * P3, FB, &bar[s]);
    bulk_g2s_hint(dst + K * P3, pr.G + e0 * 6 * P3, 6 * FB, &bar[s], pol);
    if (helm) bulk_g2s_hint(dst + 7 * K * P3, pr.B + e0 * P3, FB, &bar[s], pol);
  };
  long long ahead = next(blockIdx.x);    // thread 0: next item to prefetch
  if (tid == 0) {
    for (int s = 0; s < STAGES && ahead < Itot; ++s) {
      issue(ahead, s);
      ahead = next(ahead + G);
    }
  }
  constexpr int P2 = P * P;
  const int slot = tid / P2;
  auto Dm = [](int r, int c) { return c_b32_D[P][r * P + c]; };
  TileThread<P, float> t;
  t.init(tid - slot * P2, Dm);
  float* sT = work + slot * P3;
  float* swr = work + K * P3 + slot * P3;
  float* swsT = work + 2 * K * P3 + slot * P3;
  int n = 0;
  for (long long g = next(blockIdx.x); g < Itot; g = next(g + G), ++n) {
    const int s = n % STAGES;
    const bool ok = mbar_wait_bounded(&bar[s], (uint32_t)(n / STAGES) & 1u, err, timeout_ns);
    const int c = find_prob(s_off, ncls, g);
    const ClsProb& pr = cp[c];
    const long long e0 = (g - s_off[c]) * K;
    const int cnt = (int)min((long long)K, (long long)pr.E - e0);
    const bool act = slot < cnt;
    const bool helm = pr.h2 != 0.0f;
    const float* stage = stage0 + s * SV;
    const float* su = stage + slot * P3;
    const float* sg = stage + K * P3 + slot * 6 * P3;
    const float* sb = helm ? stage + 7 * K * P3 + slot * P3 : nullptr;
    float uc[P], bk[P], ck[P], wt[P];
    if (act) tile_load<P, float>(t, su, sb, nullptr, pr.h1, sT, uc, bk, ck);
    if (__syncthreads_or(!ok)) {
      if (tid == 0)
        for (int m = 1; m < STAGES; ++m)
          mbar_wait_bounded(&bar[(n + m) % STAGES], (uint32_t)((n + m) / STAGES) & 1u, err,
                            timeout_ns);
      return;
    }
    if (act) tile_forward<P, float>(t, su, sT, sg, uc, ck, swr, swsT, wt, Dm);
    __syncthreads();
    if (tid == 0 && ahead < Itot) {            // stage s consumed
      fence_proxy_async_smem();
      issue(ahead, s);
      ahead = next(ahead + G);
    }
    if (act)
    {
      float* we = pr.w + (e0 + slot) * P3;
      tile_backward<P, float>(t, swr, swsT, wt, uc, bk, pr.h2, helm, Dm,
                              [&](int k, float v) { we[k * P2 + t.lt] = v; });
    }
  }
}

// ---------------------------------------------------------------- batched dssum
__device__ __forceinline__ void blat2el(int c, const FastDiv& dN, int N, int nel, int& ec,
                                        int& lc) {
  ec = (int)dN.div((uint32_t)c);
  if (ec >= nel) ec = nel - 1;
  lc = c - ec * N;
  if (lc == 0 && ec > 0) {
    --ec;
    lc = N;
  }
}

__device__ __forceinline__ int bfree(int m, int nfree, int g, const BProb& b) {
  if (m == 0) return 0;
  if (m == nfree - 1) return g - 1;
  const uint32_t q = (uint32_t)(m - 1);
  const uint32_t a = b.dN1.div(q);
  return (int)(a * b.N + 1 + (q - a * (uint32_t)(b.N - 1)));
}

__global__ void __launch_bounds__(256)
bdssum_kernel(const BProb* __restrict__ probs, const long long* __restrict__ d_off, int nprob,
              long long Dtot) {
  __shared__ long long s_off[kMaxBatch];
  for (int q = threadIdx.x; q < nprob; q += blockDim.x) s_off[q] = d_off[q];
  __syncthreads();
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < Dtot; t += stride) {
    const int pi = find_prob(s_off, nprob, t);
    const BProb& b = probs[pi];
    if (b.st->done) {
      // step over the rest of this problem's items in one jump
      const long long end = pi + 1 < nprob ? s_off[pi + 1] : Dtot;
      t += (end - t - 1) / stride * stride;
      continue;
    }
    uint32_t r = (uint32_t)(t - b.d_off);
    int ix, iy, iz;
    if (r < b.nSX) {
      const uint32_t r1 = b.dgy.div(r);
      iy = (int)(r - r1 * b.gy);
      const uint32_t r2 = b.dnx1.div(r1);
      ix = (int)(r1 - r2 * (uint32_t)(b.nelx - 1) + 1) * b.N;
      iz = (int)r2;
    } else if ((r -= b.nSX) < b.nSY) {
      const uint32_t r1 = b.dnix.div(r);
      ix = bfree((int)(r - r1 * b.nix), b.nix, b.gx, b);
      const uint32_t r2 = b.dny1.div(r1);
      iy = (int)(r1 - r2 * (uint32_t)(b.nely - 1) + 1) * b.N;
      iz = (int)r2;
    } else if ((r -= b.nSY) < b.nSZ) {
      const uint32_t r1 = b.dnix.div(r);
      ix = bfree((int)(r - r1 * b.nix), b.nix, b.gx, b);
      const uint32_t r2 = b.dniy.div(r1);
      iy = bfree((int)(r1 - r2 * b.niy), b.niy, b.gy, b);
      iz = ((int)r2 + 1) * b.N;
    } else {
      b.w[b.mfree[r - b.nSZ]] = 0.0f;
      continue;
    }
    const int N = b.N, P = b.P;
    int ex, i, ey, j, ez, k;
    blat2el(ix, b.dN, N, b.nelx, ex, i);
    blat2el(iy, b.dN, N, b.nely, ey, j);
    blat2el(iz, b.dN, N, b.nelz, ez, k);
    const bool fx = (i == N) && (ex < b.nelx - 1);
    const bool fy = (j == N) && (ey < b.nely - 1);
    const bool fz = (k == N) && (ez < b.nelz - 1);
    const long long P3 = (long long)P * P * P;
    const long long e0 = (long long)ex + (long long)b.nelx * (ey + (long long)b.nely * ez);
    const long long sx = P3, sy = (long long)b.nelx * P3, sz = (long long)b.nelx * b.nely * P3;
    long long idx[8];
    int nc = 0;
    for (int cz = 0; cz <= (fz ? 1 : 0); ++cz)
      for (int cy = 0; cy <= (fy ? 1 : 0); ++cy)
        for (int cx = 0; cx <= (fx ? 1 : 0); ++cx)
          idx[nc++] = e0 * P3 + cx * sx + cy * sy + cz * sz +
                      ((long long)(cz ? 0 : k) * P + (cy ? 0 : j)) * P + (cx ? 0 : i);
    const bool masked = ((b.faces & SEM_FACE_XMIN) && ix == 0) ||
                        ((b.faces & SEM_FACE_XMAX) && ix == b.gx - 1) ||
                        ((b.faces & SEM_FACE_YMIN) && iy == 0) ||
                        ((b.faces & SEM_FACE_YMAX) && iy == b.gy - 1) ||
                        ((b.faces & SEM_FACE_ZMIN) && iz == 0) ||
                        ((b.faces & SEM_FACE_ZMAX) && iz == b.gz - 1);
    if (masked) {
      for (int c = 0; c < nc; ++c) b.w[idx[c]] = 0.0f;
      continue;
    }
    float sum = b.w[idx[0]];
    for (int c = 1; c < nc; ++c) sum += b.w[idx[c]];
    for (int c = 0; c < nc; ++c) b.w[idx[c]] = sum;
  }
}

// ---------------------------------------------------------------- batched vector kernels
struct KahanF {
  float s = 0.0f, c = 0.0f;
  __device__ __forceinline__ void add(float v) {
    const float y = __fsub_rn(v, c);
    const float t = __fadd_rn(s, y);
    c = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

// Stores this item's partial sums; the last item block of the problem returns
// true with the problem's totals (thread 0), summed over items in order.
template <int NV>
__device__ __forceinline__ bool item_sum(double (&v)[NV], double* partials, int item,
                                         int v_off, int v_cnt, unsigned int* ticket,
                                         double (&tot)[NV], int total_items) {
  __shared__ bool am_last;
  block_sum<NV>(v);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) partials[q * total_items + item] = v[q];
    __threadfence();
    const unsigned t = atomicInc(ticket, (unsigned)v_cnt - 1u);
    am_last = (t == (unsigned)v_cnt - 1u);
  }
  __syncthreads();
  if (!am_last) return false;
  __threadfence();
  double a[NV];
#pragma unroll
  for (int q = 0; q < NV; ++q) a[q] = 0.0;
  for (int it = threadIdx.x; it < v_cnt; it += blockDim.x)
#pragma unroll
    for (int q = 0; q < NV; ++q) a[q] += __ldcg(partials + q * total_items + v_off + it);
  block_sum<NV>(a);
#pragma unroll
  for (int q = 0; q < NV; ++q) tot[q] = a[q];
  return true;
}

// Starts the inner solve of the problems owning items [item0, item0 + count).
__global__ void __launch_bounds__(256)
binit_kernel(const BProb* __restrict__ probs, const int* __restrict__ item_prob, int item0,
             int count, int nitems, double* partials, unsigned* tickets, double tol, int maxit) {
  for (int it = item0 + blockIdx.x; it < item0 + count; it += gridDim.x) {
    const int pi = item_prob[it];
    const BProb& b = probs[pi];
    const long long lo = (long long)(it - b.v_off) * kChunk;
    const long long hi = min(lo + kChunk, b.nL);
    KahanF rz, rr;
    for (long long q = lo + threadIdx.x; q < hi; q += blockDim.x) {
      const float r = b.r[q];
      const float z = b.dinv[q] * r;
      b.p[q] = z;
      b.x[q] = 0.0f;
      const float im = b.imult[q];
      rz.add(__fmul_rn(__fmul_rn(r, z), im));
      rr.add(__fmul_rn(__fmul_rn(r, r), im));
    }
    double v[2] = {rz.value(), rr.value()}, tot[2];
    if (item_sum<2>(v, partials, it, b.v_off, b.v_cnt, &tickets[pi], tot, nitems) &&
        threadIdx.x == 0) {
      CGState* st = b.st;
      st->rz = tot[0];
      st->rr = tot[1];
      st->bb = tot[1];
      st->tol2 = tol * tol * tot[1];
      st->iter = 0;
      st->status = SEM_OK;
      st->maxit = maxit;
      st->alpha = st->beta = 0.0;
      st->done = (tot[1] <= st->tol2 || tot[1] == 0.0 || maxit <= 0) ? 1 : 0;
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(256)
bpw_kernel(const BProb* __restrict__ probs, const int* __restrict__ item_prob, int nprob,
           int nitems, double* partials, unsigned* tickets) {
  __shared__ ItemWalk wk;
  wk.load(probs, nprob, nitems);
  for (int it = wk.next(item_prob, blockIdx.x, gridDim.x, nitems); it < nitems;
       it = wk.next(item_prob, it + gridDim.x, gridDim.x, nitems)) {
    const int pi = item_prob[it];
    const BProb& b = probs[pi];
    const long long lo = (long long)(it - b.v_off) * kChunk;
    const long long hi = min(lo + kChunk, b.nL);
    const float4* p4 = reinterpret_cast<const float4*>(b.p + lo);
    const float4* w4 = reinterpret_cast<const float4*>(b.w + lo);
    const float4* m4 = reinterpret_cast<const float4*>(b.imult + lo);
    const int n4 = (int)((hi - lo) >> 2);
    KahanF pw;
#pragma unroll 4
    for (int q = threadIdx.x; q < n4; q += blockDim.x) {
      const float4 p = p4[q], w = w4[q], m = m4[q];
      pw.add(__fmul_rn(__fmul_rn(p.x, w.x), m.x));
      pw.add(__fmul_rn(__fmul_rn(p.y, w.y), m.y));
      pw.add(__fmul_rn(__fmul_rn(p.z, w.z), m.z));
      pw.add(__fmul_rn(__fmul_rn(p.w, w.w), m.w));
    }
    double v[1] = {pw.value()}, tot[1];
    if (item_sum<1>(v, partials, it, b.v_off, b.v_cnt, &tickets[pi], tot, nitems) &&
        threadIdx.x == 0) {
      CGState* st = b.st;
      st_after_pw(st, tot[0]);
    }
    __syncthreads();
  }
}

__device__ __forceinline__ void upd1(float& x, float& r, float p, float w, float d, float m,
                                     float alpha, KahanF& rz, KahanF& rr) {
  x += alpha * p;
  r -= alpha * w;
  const float z = d * r;
  rz.add(__fmul_rn(__fmul_rn(r, z), m));
  rr.add(__fmul_rn(__fmul_rn(r, r), m));
}

__global__ void __launch_bounds__(256)
bupdate_kernel(const BProb* __restrict__ probs, const int* __restrict__ item_prob, int nprob,
               int nitems, double* partials, unsigned* tickets) {
  __shared__ ItemWalk wk;
  wk.load(probs, nprob, nitems);
  for (int it = wk.next(item_prob, blockIdx.x, gridDim.x, nitems); it < nitems;
       it = wk.next(item_prob, it + gridDim.x, gridDim.x, nitems)) {
    const int pi = item_prob[it];
    const BProb& b = probs[pi];
    const float alpha = (float)b.st->alpha;
    const long long lo = (long long)(it - b.v_off) * kChunk;
    const long long hi = min(lo + kChunk, b.nL);
    float4* x4 = reinterpret_cast<float4*>(b.x + lo);
    float4* r4 = reinterpret_cast<float4*>(b.r + lo);
    const float4* p4 = reinterpret_cast<const float4*>(b.p + lo);
    const float4* w4 = reinterpret_cast<const float4*>(b.w + lo);
    const float4* d4 = reinterpret_cast<const float4*>(b.dinv + lo);
    const float4* m4 = reinterpret_cast<const float4*>(b.imult + lo);
    const int n4 = (int)((hi - lo) >> 2);
    KahanF rz, rr;
#pragma unroll 2
    for (int q = threadIdx.x; q < n4; q += blockDim.x) {
      float4 x = x4[q], r = r4[q];
      const float4 p = p4[q], w = w4[q], d = d4[q], m = m4[q];
      upd1(x.x, r.x, p.x, w.x, d.x, m.x, alpha, rz, rr);
      upd1(x.y, r.y, p.y, w.y, d.y, m.y, alpha, rz, rr);
      upd1(x.z, r.z, p.z, w.z, d.z, m.z, alpha, rz, rr);
      upd1(x.w, r.w, p.w, w.w, d.w, m.w, alpha, rz, rr);
      x4[q] = x;
      r4[q] = r;
    }
    double v[2] = {rz.value(), rr.value()}, tot[2];
    if (item_sum<2>(v, partials, it, b.v_off, b.v_cnt, &tickets[pi], tot, nitems) &&
        threadIdx.x == 0) {
      CGState* st = b.st;
      st_after_update(st, tot);
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(256)
bpupd_kernel(const BProb* __restrict__ probs, const int* __restrict__ item_prob, int nprob,
             int nitems) {
  __shared__ ItemWalk wk;
  wk.load(probs, nprob, nitems);
  for (int it = wk.next(item_prob, blockIdx.x, gridDim.x, nitems); it < nitems;
       it = wk.next(item_prob, it + gridDim.x, gridDim.x, nitems)) {
    const int pi = item_prob[it];
    const BProb& b = probs[pi];
    const float beta = (float)b.st->beta;
    const long long lo = (long long)(it - b.v_off) * kChunk;
    const long long hi = min(lo + kChunk, b.nL);
    float4* p4 = reinterpret_cast<float4*>(b.p + lo);
    const float4* r4 = reinterpret_cast<const float4*>(b.r + lo);
    const float4* d4 = reinterpret_cast<const float4*>(b.dinv + lo);
    const int n4 = (int)((hi - lo) >> 2);
#pragma unroll 4
    for (int q = threadIdx.x; q < n4; q += blockDim.x) {
      float4 p = p4[q];
      const float4 r = r4[q], d = d4[q];
      p.x = d.x * r.x + beta * p.x;
      p.y = d.y * r.y + beta * p.y;
      p.z = d.z * r.z + beta * p.z;
      p.w = d.w * r.w + beta * p.w;
      p4[q] = p;
    }
  }
}

}  // namespace sem

#include "batch_glob.cuh"

using namespace sem;

struct sem_batch {
  std::vector<sem_handle*> hs;
  std::vector<BProb> hp;                 // host copy of the descriptors
  DevBuf<BProb> probs;
  DevBuf<long long> d_off;
  DevBuf<int> item_prob;
  DevBuf<double> partials;
  DevBuf<unsigned> tickets;
  DevBuf<CGState> states;                // inner solve state per problem
  long long Etot = 0, Dtot = 0;
  // per order class (P = 2, 4, 6, 8, 10): problems and work-item offsets
  int ncls[kMaxP + 1] = {};
  long long Icls[kMaxP + 1] = {};
  DevBuf<int> cls_prob[kMaxP + 1];
  DevBuf<long long> cls_ioff[kMaxP + 1];
  int bax_grid_cls[kMaxP + 1] = {};
  // fused operator (every class with one element per CTA): per class the
  // segment offsets, and the work-item offsets of the three finishing passes
  bool fused = false;
  long long Scls[kMaxP + 1] = {}, Tcut[kMaxP + 1] = {}, Tsy[kMaxP + 1] = {},
            Tsz[kMaxP + 1] = {};
  DevBuf<long long> cls_soff[kMaxP + 1], cut_off[kMaxP + 1], sy_off[kMaxP + 1],
      sz_off[kMaxP + 1];
  int bapply_grid[kMaxP + 1] = {};
  // inner solves on global vectors (every handle allows it): per class the
  // element offsets of its problems, the global vector items
  bool glob = false;
  DevBuf<long long> cls_eoff[kMaxP + 1];
  long long Ecls[kMaxP + 1] = {};
  int bglob_grid[kMaxP + 1] = {};
  DevBuf<int> gitem_prob;
  DevBuf<double> pwacc;                  // per problem
  int ngitems = 0;
  int nitems = 0, maxP = 0;
  cudaStream_t stream = nullptr;
  // per-order element launches as concurrent branches (fork on fork_ev, one
  // side stream per order class, joined back by join_ev) when concurrent
  bool concurrent = false;
  cudaStream_t side[kMaxP / 2] = {};
  cudaEvent_t fork_ev = nullptr, join_ev[kMaxP / 2] = {};
  ~sem_batch() {
    for (int q = 0; q < kMaxP / 2; ++q) {
      if (join_ev[q]) cudaEventDestroy(join_ev[q]);
      if (side[q]) cudaStreamDestroy(side[q]);
    }
    if (fork_ev) cudaEventDestroy(fork_ev);
  }
};

namespace sem {

static void batch_upload_d(const sem_handle* h) {
  static bool done[kMaxP + 1] = {};
  if (done[h->P]) return;
  float d[kMaxP * kMaxP] = {};
  for (int q = 0; q < h->P * h->P; ++q) d[q] = (float)h->Dh[q];
  SEM_CUDA(cudaMemcpyToSymbol(c_b32_D, d, sizeof(d), (size_t)h->P * sizeof(d)));
  SEM_CUDA(cudaDeviceSynchronize());   // the pageable copy is complete for every stream
  done[h->P] = true;
}

template <int P>
static int bax_occupancy(int ncls) {
  using C = BaxCfg<P>;
  auto kern = bax_kernel<P, C::STAGES>;
  SEM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)C::smem(kMaxBatch)));
  int occ = 0;
  SEM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, C::THREADS,
                                                         C::smem(ncls)));
  return occ;
}

template <int P>
static void launch_bax(sem_batch* bt, cudaStream_t s) {
  using C = BaxCfg<P>;
  bax_kernel<P, C::STAGES><<<bt->bax_grid_cls[P], C::THREADS, C::smem(bt->ncls[P]), s>>>(
      bt->probs.ptr, bt->cls_prob[P].ptr, bt->cls_ioff[P].ptr, bt->ncls[P], bt->Icls[P],
      bt->hs[0]->dev_err.ptr, kWaitTimeoutNs);
  SEM_CHECK_LAUNCH();
}

template <int P>
static int bapply_occupancy(int ncls) {
  using C = BApplyCfg<P>;
  auto kern = bapply_kernel<P, C::STAGES>;
  SEM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)C::smem(kMaxBatch)));
  int occ = 0;
  SEM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, C::THREADS,
                                                         C::smem(ncls)));
  return occ;
}

template <int P>
static int bglob_occupancy(int ncls) {
  using C = BGlobCfg<P>;
  auto kern = bglob_kernel<P>;
  SEM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)C::smem(kMaxBatch)));
  int occ = 0;
  SEM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, C::THREADS,
                                                         C::smem(ncls)));
  return occ;
}

template <int P>
static void launch_bglob(sem_batch* bt, cudaStream_t s) {
  using C = BGlobCfg<P>;
  bglob_kernel<P><<<bt->bglob_grid[P], C::THREADS, C::smem(bt->ncls[P]), s>>>(
      bt->probs.ptr, bt->cls_prob[P].ptr, bt->cls_eoff[P].ptr, bt->ncls[P], bt->Ecls[P],
      bt->hs[0]->dev_err.ptr, kWaitTimeoutNs);
  SEM_CHECK_LAUNCH();
}

static int pass_blocks(long long total) {
  return (int)std::max<long long>(1, std::min<long long>((total + 255) / 256, 16LL * sem_num_sms()));
}

template <int P>
static void launch_bapply(sem_batch* bt, cudaStream_t s) {
  using C = BApplyCfg<P>;
  bapply_kernel<P, C::STAGES><<<bt->bapply_grid[P], C::THREADS, C::smem(bt->ncls[P]), s>>>(
      bt->probs.ptr, bt->cls_prob[P].ptr, bt->cls_soff[P].ptr, bt->ncls[P], bt->Scls[P],
      bt->hs[0]->dev_err.ptr, kWaitTimeoutNs);
  SEM_CHECK_LAUNCH();
}

template <int P>
static void launch_bfinish(sem_batch* bt, cudaStream_t s) {
  const int nc = bt->ncls[P];
  if (bt->Tcut[P] > 0) {
    bcut_kernel<P><<<pass_blocks(bt->Tcut[P]), 256, 0, s>>>(bt->probs.ptr, bt->cls_prob[P].ptr,
                                                            bt->cut_off[P].ptr, nc, bt->Tcut[P]);
    SEM_CHECK_LAUNCH();
  }
  if (bt->Tsy[P] > 0) {
    bsy_kernel<P><<<pass_blocks(bt->Tsy[P]), 256, 0, s>>>(bt->probs.ptr, bt->cls_prob[P].ptr,
                                                          bt->sy_off[P].ptr, nc, bt->Tsy[P]);
    SEM_CHECK_LAUNCH();
  }
  if (bt->Tsz[P] > 0) {
    bsz_kernel<P><<<pass_blocks(bt->Tsz[P]), 256, 0, s>>>(bt->probs.ptr, bt->cls_prob[P].ptr,
                                                          bt->sz_off[P].ptr, nc, bt->Tsz[P]);
    SEM_CHECK_LAUNCH();
  }
}

// launch(P, stream) for every order class present: on s one after another,
// or (bt->concurrent, two or more classes) as branches forked from s on the
// side streams and joined back into s, so that the classes' persistent grids
// fill one another's tails; in a stream capture the branches become parallel
// paths of the graph
template <class F>
static void for_classes(sem_batch* bt, cudaStream_t s, F launch) {
  int ncl = 0;
  for (int P = 2; P <= kMaxP; P += 2) ncl += bt->ncls[P] ? 1 : 0;
  if (!bt->concurrent || ncl < 2) {
    for (int P = 2; P <= kMaxP; P += 2)
      if (bt->ncls[P]) launch(P, s);
    return;
  }
  SEM_CUDA(cudaEventRecord(bt->fork_ev, s));
  int q = 0;
  for (int P = 2; P <= kMaxP; P += 2) {
    if (!bt->ncls[P]) continue;
    SEM_CUDA(cudaStreamWaitEvent(bt->side[q], bt->fork_ev, 0));
    launch(P, bt->side[q]);
    SEM_CUDA(cudaEventRecord(bt->join_ev[q], bt->side[q]));
    ++q;
  }
  for (int k = 0; k < q; ++k) SEM_CUDA(cudaStreamWaitEvent(s, bt->join_ev[k], 0));
}

// one inner iteration over the batch (captured into a graph)
static void batch_iteration(sem_batch* bt, cudaStream_t s) {
  const int n = (int)bt->hs.size();
  if (bt->glob) {
    for_classes(bt, s, [&](int P, cudaStream_t t) {
      switch (P) {
        case 2: launch_bglob<2>(bt, t); break;
        case 4: launch_bglob<4>(bt, t); break;
        case 6: launch_bglob<6>(bt, t); break;
        case 8: launch_bglob<8>(bt, t); break;
        default: launch_bglob<10>(bt, t); break;
      }
    });
    const int gblocks = std::min(bt->ngitems, 8 * sem_num_sms());
    bgpw_kernel<<<gblocks, 256, 0, s>>>(bt->probs.ptr, bt->gitem_prob.ptr, n, bt->ngitems,
                                        bt->partials.ptr, bt->tickets.ptr);
    SEM_CHECK_LAUNCH();
    bgupdate_kernel<<<gblocks, 256, 0, s>>>(bt->probs.ptr, bt->gitem_prob.ptr, n, bt->ngitems,
                                            bt->partials.ptr, bt->tickets.ptr);
    SEM_CHECK_LAUNCH();
    bgpupd_kernel<<<gblocks, 256, 0, s>>>(bt->probs.ptr, bt->gitem_prob.ptr, n, bt->ngitems);
    SEM_CHECK_LAUNCH();
    return;
  }
  if (bt->fused) {
    // each class: its element launch, then its finishing passes
    for_classes(bt, s, [&](int P, cudaStream_t t) {
      if (P == 6) { launch_bapply<6>(bt, t); launch_bfinish<6>(bt, t); }
      else if (P == 8) { launch_bapply<8>(bt, t); launch_bfinish<8>(bt, t); }
      else { launch_bapply<10>(bt, t); launch_bfinish<10>(bt, t); }
    });
  } else {
    for_classes(bt, s, [&](int P, cudaStream_t t) {
      switch (P) {
        case 2: launch_bax<2>(bt, t); break;
        case 4: launch_bax<4>(bt, t); break;
        case 6: launch_bax<6>(bt, t); break;
        case 8: launch_bax<8>(bt, t); break;
        default: launch_bax<10>(bt, t); break;
      }
    });
  }
  if (!bt->fused) {
    const int dblocks = (int)std::min<long long>((bt->Dtot + 255) / 256, 32LL * sem_num_sms());
    bdssum_kernel<<<dblocks, 256, 0, s>>>(bt->probs.ptr, bt->d_off.ptr, n, bt->Dtot);
    SEM_CHECK_LAUNCH();
  }
  const int vblocks = std::min(bt->nitems, 8 * sem_num_sms());
  bpw_kernel<<<vblocks, 256, 0, s>>>(bt->probs.ptr, bt->item_prob.ptr, n, bt->nitems,
                                     bt->partials.ptr, bt->tickets.ptr);
  SEM_CHECK_LAUNCH();
  bupdate_kernel<<<vblocks, 256, 0, s>>>(bt->probs.ptr, bt->item_prob.ptr, n, bt->nitems,
                                         bt->partials.ptr, bt->tickets.ptr);
  SEM_CHECK_LAUNCH();
  bpupd_kernel<<<vblocks, 256, 0, s>>>(bt->probs.ptr, bt->item_prob.ptr, n, bt->nitems);
  SEM_CHECK_LAUNCH();
}

}  // namespace sem

extern "C" sem_status sem_batch_create(sem_handle* const* handles, int n, sem_batch** out) {
  return guarded("sem_batch_create", [&] {
    SEM_REQUIRE(handles && out && n >= 1 && n <= kMaxBatch, "sem_batch_create: bad arguments");
    *out = nullptr;
    std::unique_ptr<sem_batch> bt(new sem_batch());
    bt->hs.assign(handles, handles + n);
    long long eoff = 0, doff = 0;
    int voff = 0;
    std::vector<long long> d_off(n);
    std::vector<int> item_prob;
    for (int p = 0; p < n; ++p) {
      sem_handle* h = handles[p];
      SEM_REQUIRE(h, "sem_batch_create: null handle");
      SEM_REQUIRE(h->f32.G.ptr, "sem_batch_create: every handle needs FP32 geometry");
      SEM_REQUIRE(h->P % 2 == 0, "sem_batch_create: orders must be odd (even points per direction)");
      SEM_REQUIRE(h->nL % 4 == 0, "sem_batch_create: local point count must be a multiple of 4");
      batch_upload_d(h);
      BProb b{};
      b.G = h->f32.G.ptr;
      b.B = h->f32.B.ptr;
      b.imult = h->imult.ptr;
      b.N = h->N;
      b.P = h->P;
      b.E = (int)h->E;
      b.nelx = h->nelx; b.nely = h->nely; b.nelz = h->nelz;
      b.faces = h->faces;
      b.nL = h->nL;
      b.e_off = eoff;
      eoff += h->E;
      b.gx = h->N * h->nelx + 1;
      b.gy = h->N * h->nely + 1;
      b.gz = h->N * h->nelz + 1;
      b.nix = b.gx - (h->nelx - 1);
      b.niy = b.gy - (h->nely - 1);
      b.nSX = (unsigned)((long long)(h->nelx - 1) * b.gy * b.gz);
      b.nSY = (unsigned)((long long)(h->nely - 1) * b.nix * b.gz);
      b.nSZ = (unsigned)((long long)(h->nelz - 1) * b.nix * b.niy);
      b.nmf = (unsigned)h->nmasked_free;
      b.mfree = h->masked_free_idx.ptr;
      b.d_off = doff;
      d_off[p] = doff;
      doff += (long long)b.nSX + b.nSY + b.nSZ + b.nmf;
      b.dN = FastDiv((uint32_t)h->N);
      b.dN1 = FastDiv((uint32_t)std::max(1, h->N - 1));
      b.dgy = FastDiv((uint32_t)b.gy);
      b.dnx1 = FastDiv((uint32_t)std::max(1, h->nelx - 1));
      b.dny1 = FastDiv((uint32_t)std::max(1, h->nely - 1));
      b.dnix = FastDiv((uint32_t)b.nix);
      b.dniy = FastDiv((uint32_t)b.niy);
      b.v_off = voff;
      b.v_cnt = (int)((h->nL + kChunk - 1) / kChunk);
      for (int q = 0; q < b.v_cnt; ++q) item_prob.push_back(p);
      voff += b.v_cnt;
      bt->maxP = std::max(bt->maxP, h->P);
      bt->hp.push_back(b);
    }
    bt->Etot = eoff;
    bt->Dtot = doff;
    bt->nitems = voff;
    int nsm = 0, dev = 0;
    SEM_CUDA(cudaGetDevice(&dev));
    SEM_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    for (int P = 2; P <= kMaxP; P += 2) {
      std::vector<int> ids;
      std::vector<long long> ioff;
      long long items = 0;
      const int K = P == 2 ? BaxCfg<2>::K : P == 4 ? BaxCfg<4>::K : P == 6 ? BaxCfg<6>::K
                  : P == 8 ? BaxCfg<8>::K : BaxCfg<10>::K;
      for (int p = 0; p < n; ++p)
        if (bt->hp[p].P == P) {
          ids.push_back(p);
          ioff.push_back(items);
          items += (bt->hp[p].E + K - 1) / K;
        }
      bt->ncls[P] = (int)ids.size();
      bt->Icls[P] = items;
      if (ids.empty()) continue;
      bt->cls_prob[P].alloc(ids.size());
      bt->cls_prob[P].upload(ids.data(), ids.size(), nullptr);
      bt->cls_ioff[P].alloc(ioff.size());
      bt->cls_ioff[P].upload(ioff.data(), ioff.size(), nullptr);
      int occ = 0;
      switch (P) {
        case 2: occ = bax_occupancy<2>((int)ids.size()); break;
        case 4: occ = bax_occupancy<4>((int)ids.size()); break;
        case 6: occ = bax_occupancy<6>((int)ids.size()); break;
        case 8: occ = bax_occupancy<8>((int)ids.size()); break;
        default: occ = bax_occupancy<10>((int)ids.size()); break;
      }
      bt->bax_grid_cls[P] = (int)std::min<long long>(items, (long long)std::max(1, occ) * nsm);
    }
    // fused operator when every order present runs one element per CTA
    bt->fused = bt->ncls[2] == 0 && bt->ncls[4] == 0;
    for (int P = 6; P <= kMaxP && bt->fused; P += 2) {
      if (!bt->ncls[P]) continue;
      std::vector<long long> soff, coff, yoff, zoff;
      long long S = 0, C = 0, Y = 0, Z = 0;
      for (int p = 0; p < n; ++p) {
        const BProb& b = bt->hp[p];
        if (b.P != P) continue;
        const long long nseg = (b.E + kFuseSeg - 1) / kFuseSeg;
        soff.push_back(S);
        coff.push_back(C);
        yoff.push_back(Y);
        zoff.push_back(Z);
        S += nseg;
        C += (nseg - 1) * P * P;
        Y += (long long)b.nelx * (b.nely - 1) * b.nelz * P * (P / 2);
        Z += (long long)b.nelx * b.nely * (b.nelz - 1) * (P * P / 4);
      }
      bt->Scls[P] = S;
      bt->Tcut[P] = C;
      bt->Tsy[P] = Y;
      bt->Tsz[P] = Z;
      DevBuf<long long>* bufs[4] = {&bt->cls_soff[P], &bt->cut_off[P], &bt->sy_off[P],
                                    &bt->sz_off[P]};
      std::vector<long long>* vals[4] = {&soff, &coff, &yoff, &zoff};
      for (int a = 0; a < 4; ++a) {
        bufs[a]->alloc(vals[a]->size());
        bufs[a]->upload(vals[a]->data(), vals[a]->size(), nullptr);
      }
      const int ncl = bt->ncls[P];
      const int occ = P == 6 ? bapply_occupancy<6>(ncl)
                    : P == 8 ? bapply_occupancy<8>(ncl) : bapply_occupancy<10>(ncl);
      bt->bapply_grid[P] = (int)std::min<long long>(S, (long long)std::max(1, occ) * nsm);
    }
    // global-vector inner solves when every handle allows them
    bt->glob = true;
    for (int p = 0; p < n; ++p)
      bt->glob = bt->glob && handles[p]->inner_vectors != SEM_INNER_LOCAL &&
                 glob_supported(handles[p]);
    if (bt->glob) {
      std::vector<int> gitem_prob;
      int goff = 0;
      for (int p = 0; p < n; ++p) {
        BProb& b = bt->hp[p];
        b.nGp = glob_padded(handles[p]);
        b.g_off = goff;
        b.g_cnt = (int)((b.nGp + kGChunk - 1) / kGChunk);
        for (int q = 0; q < b.g_cnt; ++q) gitem_prob.push_back(p);
        goff += b.g_cnt;
        b.dnx = FastDiv((uint32_t)b.nelx);
        b.dny = FastDiv((uint32_t)b.nely);
        b.fused_pw = (b.P * b.P) % 32 == 0 ? 1 : 0;
      }
      bt->pwacc.alloc(n);
      SEM_CUDA(cudaMemset(bt->pwacc.ptr, 0, n * sizeof(double)));
      for (int p = 0; p < n; ++p) bt->hp[p].pwacc = bt->pwacc.ptr + p;
      bt->ngitems = goff;
      bt->gitem_prob.alloc(gitem_prob.size());
      bt->gitem_prob.upload(gitem_prob.data(), gitem_prob.size(), nullptr);
      for (int P = 2; P <= kMaxP; P += 2) {
        if (!bt->ncls[P]) continue;
        std::vector<long long> eoff;
        long long Ec = 0;
        for (int p = 0; p < n; ++p)
          if (bt->hp[p].P == P) {
            eoff.push_back(Ec);
            Ec += bt->hp[p].E;
          }
        bt->Ecls[P] = Ec;
        bt->cls_eoff[P].alloc(eoff.size());
        bt->cls_eoff[P].upload(eoff.data(), eoff.size(), nullptr);
        const int ncl = bt->ncls[P];
        const int occ = P == 2 ? bglob_occupancy<2>(ncl) : P == 4 ? bglob_occupancy<4>(ncl)
                      : P == 6 ? bglob_occupancy<6>(ncl) : P == 8 ? bglob_occupancy<8>(ncl)
                      : bglob_occupancy<10>(ncl);
        bt->bglob_grid[P] = (int)std::min<long long>(Ec, (long long)std::max(1, occ) * nsm);
      }
    }
    bt->d_off.alloc(n);
    bt->d_off.upload(d_off.data(), n, nullptr);
    bt->item_prob.alloc(item_prob.size());
    bt->item_prob.upload(item_prob.data(), item_prob.size(), nullptr);
    bt->partials.alloc(2 * (size_t)std::max(bt->nitems, bt->ngitems));
    bt->tickets.alloc(n);
    SEM_CUDA(cudaMemset(bt->tickets.ptr, 0, n * sizeof(unsigned)));
    bt->states.alloc(n);
    SEM_CUDA(cudaMemset(bt->states.ptr, 0, n * sizeof(CGState)));
    bt->probs.alloc(n);
    for (int q = 0; q < kMaxP / 2; ++q) {
      SEM_CUDA(cudaStreamCreateWithFlags(&bt->side[q], cudaStreamNonBlocking));
      SEM_CUDA(cudaEventCreateWithFlags(&bt->join_ev[q], cudaEventDisableTiming));
    }
    SEM_CUDA(cudaEventCreateWithFlags(&bt->fork_ev, cudaEventDisableTiming));
    SEM_CUDA(cudaDeviceSynchronize());
    *out = bt.release();
  });
}

extern "C" sem_status sem_batch_set_concurrency(sem_batch* bt, int concurrent) {
  return guarded("sem_batch_set_concurrency", [&] {
    SEM_REQUIRE(bt, "sem_batch_set_concurrency: null batch");
    SEM_REQUIRE(concurrent == 0 || concurrent == 1, "sem_batch_set_concurrency: flag not 0 or 1");
    bt->concurrent = concurrent != 0;
  });
}

extern "C" sem_status sem_batch_destroy(sem_batch* bt) {
  return guarded("sem_batch_destroy", [&] {
    if (!bt) return;
    cudaDeviceSynchronize();
    delete bt;
  });
}

extern "C" sem_status sem_batch_solve(sem_batch* bt, const double* const* b_L,
                                      double* const* x_L, const double* h1, const double* h2,
                                      const sem_solve_opts* opts, sem_solve_info* infos) {
  return guarded("sem_batch_solve", [&] {
    SEM_REQUIRE(bt && b_L && x_L && h1 && h2, "sem_batch_solve: null argument");
    sem_solve_opts o;
    if (opts) o = *opts; else sem_solve_opts_default(&o);
    SEM_REQUIRE(o.inner_tol > 0.0 && o.inner_tol < 1.0, "sem_batch_solve: bad inner_tol");
    const int n = (int)bt->hs.size();
    cudaStream_t s = (cudaStream_t)o.stream;
    SEM_CUDA(cudaStreamSynchronize(s));
    cudaStream_t own;
    SEM_CUDA(cudaStreamCreateWithFlags(&own, cudaStreamNonBlocking));
    struct Cleanup {
      cudaStream_t st;
      cudaGraphExec_t ex = nullptr;
      ~Cleanup() {
        if (ex) cudaGraphExecDestroy(ex);
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
      }
    } cleanup{own};
    // per-problem preparation and descriptors
    std::vector<sem_solve_opts> po(n, o);
    for (int p = 0; p < n; ++p) {
      sem_handle* h = bt->hs[p];
      SEM_REQUIRE(b_L[p] && x_L[p], "sem_batch_solve: null vector");
      po[p].h1 = h1[p];
      po[p].h2 = h2[p];
      po[p].h1_field = nullptr;
      mixed_prepare(h, po[p], own);
      if (bt->glob) glob_prepare(h, own);
      BProb& b = bt->hp[p];
      b.dinv = h->f32.dinv.ptr;
      b.x = h->x32.ptr;
      b.r = h->r32.ptr;
      b.p = h->p32.ptr;
      b.w = h->w32.ptr;
      b.h1 = (float)h1[p];
      b.h2 = (float)h2[p];
      b.st = bt->states.ptr + p;
      b.xg = h->xg.ptr;
      b.rg = h->rg.ptr;
      b.pg = h->pg.ptr;
      b.wg = h->wg.ptr;
      b.dinvg = h->dinvg.ptr;
      if (o.x0_is_zero) SEM_CUDA(cudaMemsetAsync(x_L[p], 0, h->nL * sizeof(double), own));
      outer_norm_b(h, b_L[p], own);
      inner_scale_from_b(h, own);
    }
    bt->probs.upload(bt->hp.data(), n, own);
    // Each problem moves on its own: FP64 residual -> (converged | FP32 inner
    // solve in the batch) -> correction -> FP64 residual ...  The graph of
    // batched iterations skips problems whose inner solve is not running.
    enum { RUNNING = 0, FINISHED = 1 };
    std::vector<int> phase(n, RUNNING), iters(n, 0), outer(n, 0), status(n, SEM_ERR_NOCONV);
    std::vector<double> rel(n, 0.0);
    const int batch_it = std::max(1, o.check_every);
    cudaGraphExec_t exec = nullptr;
    if (o.use_graph) {
      cudaGraph_t graph = nullptr;
      SEM_CUDA(cudaStreamBeginCapture(own, cudaStreamCaptureModeThreadLocal));
      try {
        for (int c = 0; c < batch_it; ++c) batch_iteration(bt, own);
      } catch (...) {
        cudaStreamEndCapture(own, &graph);
        if (graph) cudaGraphDestroy(graph);
        throw;
      }
      SEM_CUDA(cudaStreamEndCapture(own, &graph));
      cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
      cudaGraphDestroy(graph);
      SEM_CUDA(e);
      cleanup.ex = exec;
    }
    SEM_CUDA(cudaMemsetAsync(bt->tickets.ptr, 0, n * sizeof(unsigned), own));
    // FP64 residual of problem p; starts its next inner solve unless it is finished
    auto refine = [&](int p) {
      sem_handle* h = bt->hs[p];
      if (bt->glob) outer_residual_global(h, b_L[p], x_L[p], po[p], own);
      else outer_residual(h, b_L[p], x_L[p], po[p], own);
      const CGState hs0 = state_to_host(h->state.ptr, own, h->dev_err.ptr);
      rel[p] = hs0.bb > 0 ? std::sqrt(hs0.rr / hs0.bb) : 0.0;
      if (!(rel[p] == rel[p])) { status[p] = SEM_ERR_BREAKDOWN; phase[p] = FINISHED; }
      else if (rel[p] <= o.tol) { status[p] = SEM_OK; phase[p] = FINISHED; }
      else if (outer[p] >= o.max_outer || iters[p] >= o.maxit) { phase[p] = FINISHED; }
      if (phase[p] == FINISHED) {
        CGState fin{};
        fin.done = 1;
        SEM_CUDA(cudaMemcpyAsync(bt->states.ptr + p, &fin, sizeof(CGState),
                                 cudaMemcpyHostToDevice, own));
        SEM_CUDA(cudaStreamSynchronize(own));
        return;
      }
      const BProb& b = bt->hp[p];
      if (bt->glob) {
        bginit_kernel<<<std::min(b.g_cnt, 4 * sem_num_sms()), 256, 0, own>>>(
            bt->probs.ptr, bt->gitem_prob.ptr, b.g_off, b.g_cnt, bt->ngitems, bt->partials.ptr,
            bt->tickets.ptr, inner_target(o.inner_tol, o.tol, rel[p]),
            std::max(1, o.maxit - iters[p]));
      } else {
        binit_kernel<<<std::min(b.v_cnt, 4 * sem_num_sms()), 256, 0, own>>>(
            bt->probs.ptr, bt->item_prob.ptr, b.v_off, b.v_cnt, bt->nitems, bt->partials.ptr,
            bt->tickets.ptr, inner_target(o.inner_tol, o.tol, rel[p]),
            std::max(1, o.maxit - iters[p]));
      }
      SEM_CHECK_LAUNCH();
    };
    for (int p = 0; p < n; ++p) refine(p);
    std::vector<CGState> st(n);
    for (long guard = 0;; ++guard) {
      bool any = false;
      for (int p = 0; p < n; ++p) any = any || phase[p] == RUNNING;
      if (!any) break;
      if (guard > 10000000L) throw Error(SEM_ERR_NOCONV, "sem_batch_solve: iteration guard");
      if (exec) SEM_CUDA(cudaGraphLaunch(exec, own));
      else
        for (int c = 0; c < batch_it; ++c) batch_iteration(bt, own);
      SEM_CUDA(cudaMemcpyAsync(st.data(), bt->states.ptr, n * sizeof(CGState),
                               cudaMemcpyDeviceToHost, own));
      int herr = 0;
      SEM_CUDA(cudaMemcpyAsync(&herr, bt->hs[0]->dev_err.ptr, sizeof(int),
                               cudaMemcpyDeviceToHost, own));
      SEM_CUDA(cudaStreamSynchronize(own));
      if (herr) {
        SEM_CUDA(cudaMemsetAsync(bt->hs[0]->dev_err.ptr, 0, sizeof(int), own));
        throw Error(SEM_ERR_TIMEOUT, "sem_batch_solve: a bounded device wait timed out");
      }
      for (int p = 0; p < n; ++p) {
        if (phase[p] != RUNNING || !st[p].done) continue;
        // inner solve of p finished: correction, then the next refinement step
        iters[p] += st[p].iter;
        ++outer[p];
        if (st[p].status == SEM_ERR_BREAKDOWN && st[p].iter == 0) {
          status[p] = SEM_ERR_BREAKDOWN;
          phase[p] = FINISHED;
          continue;
        }
        if (bt->glob) add_from_global(bt->hs[p], x_L[p], bt->hs[p]->xg.ptr, own,
                                      1.0 / bt->hs[p]->rscale);
        else outer_update(bt->hs[p], x_L[p], own);
        refine(p);
      }
    }
    SEM_CUDA(cudaStreamSynchronize(own));
    for (int p = 0; p < n; ++p) {
      if (infos) {
        infos[p].iters = iters[p];
        infos[p].outer_iters = outer[p];
        infos[p].rel_res = rel[p];
        infos[p].status = status[p];
      }
    }
  });
}
