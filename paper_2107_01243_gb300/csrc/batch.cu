// Batched solves: many independent Helmholtz problems of uneven element count
// and order N advance together, FP32-inner PCG inside FP64 refinement per
// problem (the solver of cg.cu, arXiv 2107.01243 §2 end and §4, applied to a
// batch).  Every stage of an inner CG iteration is one launch over all
// problems:
//   bax     persistent bulk-copy (TMA) Ax over the flat list of all elements,
//           each element dispatched to the kernel body of its order
//   bdssum  index-free gather-scatter over all problems' shared points
//   bpw, bupdate, bpupd  vector updates over fixed-size chunks; the chunk
//           partial sums of one problem are reduced, in a fixed order, by the
//           last chunk block to finish (a ticket per problem)
// Converged problems are skipped by every stage.  A batch of iterations is
// captured in a CUDA graph; the host reads one counter of finished problems
// per graph launch.
#include <cmath>
#include <memory>
#include <vector>

#include "sem_internal.cuh"
#include "tma.cuh"
#include "reduce.cuh"

namespace sem {

constexpr int kMaxBatch = 256;
constexpr int kBaxThreads = 128;       // >= P^2 for every supported order
constexpr int kChunk = 16384;          // points per vector work item

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
  long long d_off;       // first flat gather-scatter item
  int v_off, v_cnt;      // vector chunk items
  int gx, gy, gz, nix, niy;
  unsigned nSX, nSY, nSZ, nmf;
  const int* mfree;
  FastDiv dN, dN1, dgy, dnx1, dny1, dnix, dniy;
};

__device__ __forceinline__ int find_prob(const long long* off, int n, long long g) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= g) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// ---------------------------------------------------------------- batched Ax
template <int P>
__device__ __forceinline__ void load_row_f(const float* __restrict__ p, float (&v)[P]) {
  if constexpr ((P * 4) % 16 == 0) {
    const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
    for (int a = 0; a < P / 4; ++a) {
      const float4 f = q[a];
      v[4 * a] = f.x; v[4 * a + 1] = f.y; v[4 * a + 2] = f.z; v[4 * a + 3] = f.w;
    }
  } else if constexpr ((P * 4) % 8 == 0) {
    const float2* q = reinterpret_cast<const float2*>(p);
#pragma unroll
    for (int a = 0; a < P / 2; ++a) {
      const float2 f = q[a];
      v[2 * a] = f.x; v[2 * a + 1] = f.y;
    }
  } else {
#pragma unroll
    for (int a = 0; a < P; ++a) v[a] = p[a];
  }
}

// One element of order P from a filled stage (u, 6 G, [B]); release() is
// called by all threads once the stage is no longer read.
template <int P, class Rel>
__device__ __forceinline__ void belem(const float* __restrict__ su, float* sT, float* swr,
                                      float* swsT, float* __restrict__ we, float h1, float h2,
                                      bool helm, int tid, Rel release) {
  constexpr int P2 = P * P, P3 = P2 * P;
  const bool act = tid < P2;
  const int i = tid % P, j = tid / P;
  const float* sg = su + P3;
  const float* sb = su + 7 * P3;
  float uc[P], bk[P], wt[P];
  if (act) {
#pragma unroll
    for (int k = 0; k < P; ++k) {
      uc[k] = su[k * P2 + tid];
      sT[k * P2 + i * P + j] = uc[k];
      bk[k] = helm ? sb[k * P2 + tid] : 0.0f;
    }
  }
  __syncthreads();
  if (act) {
#pragma unroll
    for (int k = 0; k < P; ++k) {
      float row[P], col[P];
      load_row_f<P>(su + k * P2 + j * P, row);
      load_row_f<P>(sT + k * P2 + i * P, col);
      float ur = 0.0f, us = 0.0f, ut = 0.0f;
#pragma unroll
      for (int l = 0; l < P; ++l) {
        ur = fmaf(c_b32_D[P][i * P + l], row[l], ur);
        us = fmaf(c_b32_D[P][j * P + l], col[l], us);
        ut = fmaf(c_b32_D[P][k * P + l], uc[l], ut);
      }
      const int q = k * P2 + tid;
      const float g11 = sg[q], g22 = sg[P3 + q], g33 = sg[2 * P3 + q];
      const float g12 = sg[3 * P3 + q], g13 = sg[4 * P3 + q], g23 = sg[5 * P3 + q];
      swr[k * P2 + j * P + i] = h1 * (g11 * ur + g12 * us + g13 * ut);
      swsT[k * P2 + i * P + j] = h1 * (g12 * ur + g22 * us + g23 * ut);
      wt[k] = h1 * (g13 * ur + g23 * us + g33 * ut);
    }
  }
  __syncthreads();
  release();
  if (act) {
#pragma unroll
    for (int k = 0; k < P; ++k) {
      float row[P], col[P];
      load_row_f<P>(swr + k * P2 + j * P, row);
      load_row_f<P>(swsT + k * P2 + i * P, col);
      float acc = 0.0f;
#pragma unroll
      for (int l = 0; l < P; ++l) {
        acc = fmaf(c_b32_D[P][l * P + i], row[l], acc);
        acc = fmaf(c_b32_D[P][l * P + j], col[l], acc);
        acc = fmaf(c_b32_D[P][l * P + k], wt[l], acc);
      }
      if (helm) acc = fmaf(h2 * bk[k], uc[k], acc);
      we[k * P2 + tid] = acc;
    }
  }
}

template <int STAGES>
__global__ void __launch_bounds__(kBaxThreads)
bax_kernel(const BProb* __restrict__ probs, int nprob, long long Etot, int stage_vals,
           int work_vals, int* __restrict__ err, uint64_t timeout_ns) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ long long s_off[kMaxBatch];
  __shared__ int s_skip[kMaxBatch];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);
  float* stage0 = reinterpret_cast<float*>(smem_raw + 128);
  float* sT = stage0 + STAGES * stage_vals;
  float* swr = sT + work_vals;
  float* swsT = swr + work_vals;
  const int tid = threadIdx.x;
  for (int q = tid; q < nprob; q += blockDim.x) {
    s_off[q] = probs[q].e_off;
    s_skip[q] = probs[q].st->done;
  }
  if (tid == 0) {
#pragma unroll
    for (int s = 0; s < STAGES; ++s) mbar_init(&bar[s], 1);
    mbar_fence_init();
  }
  __syncthreads();
  const long long G = gridDim.x;
  // next element of this CTA at or after g whose problem is still running
  auto next = [&](long long g) {
    while (g < Etot && s_skip[find_prob(s_off, nprob, g)]) g += G;
    return g;
  };
  auto issue = [&](long long g, int s) {
    const int pi = find_prob(s_off, nprob, g);
    const BProb& pr = probs[pi];
    const long long e = g - pr.e_off;
    const int P3 = pr.P * pr.P * pr.P;
    const uint32_t FB = (uint32_t)P3 * 4u;
    const bool helm = pr.h2 != 0.0f;
    float* dst = stage0 + s * stage_vals;
    mbar_arrive_expect_tx(&bar[s], (helm ? 8u : 7u) * FB);
    bulk_g2s(dst, pr.p + e * P3, FB, &bar[s]);
    bulk_g2s(dst + P3, pr.G + e * 6 * P3, 6 * FB, &bar[s]);
    if (helm) bulk_g2s(dst + 7 * P3, pr.B + e * P3, FB, &bar[s]);
  };
  long long ahead = next(blockIdx.x);    // thread 0: next element to prefetch
  if (tid == 0) {
    for (int s = 0; s < STAGES && ahead < Etot; ++s) {
      issue(ahead, s);
      ahead = next(ahead + G);
    }
  }
  int n = 0;
  for (long long g = next(blockIdx.x); g < Etot; g = next(g + G), ++n) {
    const int s = n % STAGES;
    const bool ok = mbar_wait_bounded(&bar[s], (uint32_t)(n / STAGES) & 1u, err, timeout_ns);
    if (__syncthreads_or(!ok)) {
      if (tid == 0)
        for (int m = 1; m < STAGES; ++m)
          mbar_wait_bounded(&bar[(n + m) % STAGES], (uint32_t)((n + m) / STAGES) & 1u, err,
                            timeout_ns);
      return;
    }
    const int pi = find_prob(s_off, nprob, g);
    const BProb& pr = probs[pi];
    const long long e = g - pr.e_off;
    const float* su = stage0 + s * stage_vals;
    const bool helm = pr.h2 != 0.0f;
    auto release = [&]() {
      if (tid == 0 && ahead < Etot) {
        fence_proxy_async_smem();
        issue(ahead, s);
        ahead = next(ahead + G);
      }
    };
    const int P3 = pr.P * pr.P * pr.P;
    float* we = pr.w + e * P3;
    switch (pr.P) {
      case 2: belem<2>(su, sT, swr, swsT, we, pr.h1, pr.h2, helm, tid, release); break;
      case 4: belem<4>(su, sT, swr, swsT, we, pr.h1, pr.h2, helm, tid, release); break;
      case 6: belem<6>(su, sT, swr, swsT, we, pr.h1, pr.h2, helm, tid, release); break;
      case 8: belem<8>(su, sT, swr, swsT, we, pr.h1, pr.h2, helm, tid, release); break;
      case 10: belem<10>(su, sT, swr, swsT, we, pr.h1, pr.h2, helm, tid, release); break;
      default: break;
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
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < Dtot;
       t += (long long)gridDim.x * blockDim.x) {
    const int pi = find_prob(d_off, nprob, t);
    const BProb& b = probs[pi];
    if (b.st->done) continue;
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

__global__ void __launch_bounds__(256)
binit_kernel(const BProb* __restrict__ probs, const int* __restrict__ item_prob, int nitems,
             double* partials, unsigned* tickets, const int* __restrict__ active, double tol,
             int maxit, int* ndone) {
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
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
      st->done = (!active[pi] || tot[1] <= st->tol2 || tot[1] == 0.0 || maxit <= 0) ? 1 : 0;
      if (st->done) atomicAdd(ndone, 1);
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(256)
bpw_kernel(const BProb* __restrict__ probs, const int* __restrict__ item_prob, int nitems,
           double* partials, unsigned* tickets, int* ndone) {
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const int pi = item_prob[it];
    const BProb& b = probs[pi];
    if (b.st->done) continue;
    const long long lo = (long long)(it - b.v_off) * kChunk;
    const long long hi = min(lo + kChunk, b.nL);
    KahanF pw;
    for (long long q = lo + threadIdx.x; q < hi; q += blockDim.x)
      pw.add(__fmul_rn(__fmul_rn(b.p[q], b.w[q]), b.imult[q]));
    double v[1] = {pw.value()}, tot[1];
    if (item_sum<1>(v, partials, it, b.v_off, b.v_cnt, &tickets[pi], tot, nitems) &&
        threadIdx.x == 0) {
      CGState* st = b.st;
      st->pw = tot[0];
      if (!(tot[0] > 0.0)) {
        st->status = SEM_ERR_BREAKDOWN;
        st->done = 1;
        atomicAdd(ndone, 1);
      } else {
        st->alpha = st->rz / tot[0];
      }
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(256)
bupdate_kernel(const BProb* __restrict__ probs, const int* __restrict__ item_prob, int nitems,
               double* partials, unsigned* tickets, int* ndone) {
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const int pi = item_prob[it];
    const BProb& b = probs[pi];
    if (b.st->done) continue;
    const float alpha = (float)b.st->alpha;
    const long long lo = (long long)(it - b.v_off) * kChunk;
    const long long hi = min(lo + kChunk, b.nL);
    KahanF rz, rr;
    for (long long q = lo + threadIdx.x; q < hi; q += blockDim.x) {
      b.x[q] += alpha * b.p[q];
      const float r = b.r[q] - alpha * b.w[q];
      b.r[q] = r;
      const float z = b.dinv[q] * r;
      const float im = b.imult[q];
      rz.add(__fmul_rn(__fmul_rn(r, z), im));
      rr.add(__fmul_rn(__fmul_rn(r, r), im));
    }
    double v[2] = {rz.value(), rr.value()}, tot[2];
    if (item_sum<2>(v, partials, it, b.v_off, b.v_cnt, &tickets[pi], tot, nitems) &&
        threadIdx.x == 0) {
      CGState* st = b.st;
      st->iter += 1;
      st->rr = tot[1];
      if (!(tot[1] == tot[1]) || !(tot[0] == tot[0])) {
        st->status = SEM_ERR_BREAKDOWN;
        st->done = 1;
      } else if (tot[1] <= st->tol2) {
        st->done = 1;
      } else if (st->iter >= st->maxit) {
        st->status = SEM_ERR_NOCONV;
        st->done = 1;
      } else {
        st->beta = tot[0] / st->rz;
        st->rz = tot[0];
      }
      if (st->done) atomicAdd(ndone, 1);
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(256)
bpupd_kernel(const BProb* __restrict__ probs, const int* __restrict__ item_prob, int nitems) {
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const int pi = item_prob[it];
    const BProb& b = probs[pi];
    if (b.st->done) continue;
    const float beta = (float)b.st->beta;
    const long long lo = (long long)(it - b.v_off) * kChunk;
    const long long hi = min(lo + kChunk, b.nL);
    for (long long q = lo + threadIdx.x; q < hi; q += blockDim.x)
      b.p[q] = b.dinv[q] * b.r[q] + beta * b.p[q];
  }
}

}  // namespace sem

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
  DevBuf<int> active;
  DevBuf<int> ndone;
  long long Etot = 0, Dtot = 0;
  int nitems = 0, maxP = 0, stage_vals = 0, work_vals = 0;
  int bax_grid = 0;
  size_t bax_smem = 0;
  cudaStream_t stream = nullptr;
};

namespace sem {

static void batch_upload_d(const sem_handle* h) {
  static bool done[kMaxP + 1] = {};
  if (done[h->P]) return;
  float d[kMaxP * kMaxP] = {};
  for (int q = 0; q < h->P * h->P; ++q) d[q] = (float)h->Dh[q];
  SEM_CUDA(cudaMemcpyToSymbol(c_b32_D, d, sizeof(d), (size_t)h->P * sizeof(d)));
  done[h->P] = true;
}

// one inner iteration over the batch (captured into a graph)
static void batch_iteration(sem_batch* bt, cudaStream_t s) {
  const int n = (int)bt->hs.size();
  bax_kernel<2><<<bt->bax_grid, kBaxThreads, bt->bax_smem, s>>>(
      bt->probs.ptr, n, bt->Etot, bt->stage_vals, bt->work_vals, bt->hs[0]->dev_err.ptr,
      kWaitTimeoutNs);
  SEM_CHECK_LAUNCH();
  const int dblocks = (int)std::min<long long>((bt->Dtot + 255) / 256, 32LL * kNumSMs);
  bdssum_kernel<<<dblocks, 256, 0, s>>>(bt->probs.ptr, bt->d_off.ptr, n, bt->Dtot);
  SEM_CHECK_LAUNCH();
  const int vblocks = std::min(bt->nitems, 8 * kNumSMs);
  bpw_kernel<<<vblocks, 256, 0, s>>>(bt->probs.ptr, bt->item_prob.ptr, bt->nitems,
                                     bt->partials.ptr, bt->tickets.ptr, bt->ndone.ptr);
  SEM_CHECK_LAUNCH();
  bupdate_kernel<<<vblocks, 256, 0, s>>>(bt->probs.ptr, bt->item_prob.ptr, bt->nitems,
                                         bt->partials.ptr, bt->tickets.ptr, bt->ndone.ptr);
  SEM_CHECK_LAUNCH();
  bpupd_kernel<<<vblocks, 256, 0, s>>>(bt->probs.ptr, bt->item_prob.ptr, bt->nitems);
  SEM_CHECK_LAUNCH();
}

}  // namespace sem

extern "C" sem_status sem_batch_create(sem_handle* const* handles, int n, sem_batch** out) {
  return guarded([&] {
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
    const int P3 = bt->maxP * bt->maxP * bt->maxP;
    bt->stage_vals = 8 * P3;
    bt->work_vals = P3;
    bt->bax_smem = 128 + (size_t)(2 * bt->stage_vals + 3 * bt->work_vals) * sizeof(float);
    auto kern = bax_kernel<2>;
    SEM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)bt->bax_smem));
    int occ = 0;
    SEM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kBaxThreads, bt->bax_smem));
    int nsm = 0, dev = 0;
    SEM_CUDA(cudaGetDevice(&dev));
    SEM_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    bt->bax_grid = (int)std::min<long long>(bt->Etot, (long long)std::max(1, occ) * nsm);
    bt->d_off.alloc(n);
    bt->d_off.upload(d_off.data(), n, nullptr);
    bt->item_prob.alloc(item_prob.size());
    bt->item_prob.upload(item_prob.data(), item_prob.size(), nullptr);
    bt->partials.alloc(2 * (size_t)bt->nitems);
    bt->tickets.alloc(n);
    SEM_CUDA(cudaMemset(bt->tickets.ptr, 0, n * sizeof(unsigned)));
    bt->states.alloc(n);
    SEM_CUDA(cudaMemset(bt->states.ptr, 0, n * sizeof(CGState)));
    bt->active.alloc(n);
    bt->ndone.alloc(1);
    bt->probs.alloc(n);
    SEM_CUDA(cudaDeviceSynchronize());
    *out = bt.release();
  });
}

extern "C" sem_status sem_batch_destroy(sem_batch* bt) {
  return guarded([&] {
    if (!bt) return;
    cudaDeviceSynchronize();
    delete bt;
  });
}

extern "C" sem_status sem_batch_solve(sem_batch* bt, const double* const* b_L,
                                      double* const* x_L, const double* h1, const double* h2,
                                      const sem_solve_opts* opts, sem_solve_info* infos) {
  return guarded([&] {
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
      BProb& b = bt->hp[p];
      b.dinv = h->f32.dinv.ptr;
      b.x = h->x32.ptr;
      b.r = h->r32.ptr;
      b.p = h->p32.ptr;
      b.w = h->w32.ptr;
      b.h1 = (float)h1[p];
      b.h2 = (float)h2[p];
      b.st = bt->states.ptr + p;
      if (o.x0_is_zero) SEM_CUDA(cudaMemsetAsync(x_L[p], 0, h->nL * sizeof(double), own));
      outer_norm_b(h, b_L[p], own);
    }
    bt->probs.upload(bt->hp.data(), n, own);
    std::vector<int> active(n, 1), iters(n, 0), outer(n, 0), status(n, SEM_ERR_NOCONV);
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
    int total_inner = 0;
    for (int step = 0;; ++step) {
      // FP64 residual of every running problem
      int nactive = 0;
      for (int p = 0; p < n; ++p) {
        if (!active[p]) continue;
        sem_handle* h = bt->hs[p];
        outer_residual(h, b_L[p], x_L[p], po[p], own);
        const CGState hs0 = state_to_host(h->state.ptr, own, h->dev_err.ptr);
        rel[p] = hs0.bb > 0 ? std::sqrt(hs0.rr / hs0.bb) : 0.0;
        if (!(rel[p] == rel[p])) { status[p] = SEM_ERR_BREAKDOWN; active[p] = 0; continue; }
        if (rel[p] <= o.tol) { status[p] = SEM_OK; active[p] = 0; continue; }
        if (outer[p] >= o.max_outer || iters[p] >= o.maxit) { active[p] = 0; continue; }
        ++nactive;
      }
      if (nactive == 0) break;
      // batched FP32 inner PCG of the running problems
      bt->active.upload(active.data(), n, own);
      SEM_CUDA(cudaMemsetAsync(bt->ndone.ptr, 0, sizeof(int), own));
      SEM_CUDA(cudaMemsetAsync(bt->tickets.ptr, 0, n * sizeof(unsigned), own));
      binit_kernel<<<std::min(bt->nitems, 8 * kNumSMs), 256, 0, own>>>(
          bt->probs.ptr, bt->item_prob.ptr, bt->nitems, bt->partials.ptr, bt->tickets.ptr,
          bt->active.ptr, o.inner_tol, o.maxit, bt->ndone.ptr);
      SEM_CHECK_LAUNCH();
      int ndone = 0;
      for (int guard = 0;; ++guard) {
        SEM_CUDA(cudaMemcpyAsync(&ndone, bt->ndone.ptr, sizeof(int), cudaMemcpyDeviceToHost, own));
        SEM_CUDA(cudaStreamSynchronize(own));
        if (ndone >= n) break;
        if (exec) SEM_CUDA(cudaGraphLaunch(exec, own));
        else
          for (int c = 0; c < batch_it; ++c) batch_iteration(bt, own);
        if (guard > 1000000) throw Error(SEM_ERR_NOCONV, "sem_batch_solve: inner loop guard");
      }
      std::vector<CGState> st(n);
      SEM_CUDA(cudaMemcpyAsync(st.data(), bt->states.ptr, n * sizeof(CGState),
                               cudaMemcpyDeviceToHost, own));
      int herr = 0;
      SEM_CUDA(cudaMemcpyAsync(&herr, bt->hs[0]->dev_err.ptr, sizeof(int), cudaMemcpyDeviceToHost,
                               own));
      SEM_CUDA(cudaStreamSynchronize(own));
      if (herr) {
        SEM_CUDA(cudaMemsetAsync(bt->hs[0]->dev_err.ptr, 0, sizeof(int), own));
        throw Error(SEM_ERR_TIMEOUT, "sem_batch_solve: a bounded device wait timed out");
      }
      for (int p = 0; p < n; ++p) {
        if (!active[p]) continue;
        iters[p] += st[p].iter;
        total_inner += st[p].iter;
        ++outer[p];
        if (st[p].status == SEM_ERR_BREAKDOWN && st[p].iter == 0) {
          status[p] = SEM_ERR_BREAKDOWN;
          active[p] = 0;
          continue;
        }
        outer_update(bt->hs[p], x_L[p], own);
      }
      (void)step;
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
    (void)total_inner;
  });
}
