// The assembled operator of the batched solver with the gather-scatter split
// by direction (the single-problem form is apply.cu): per order class, one
// persistent element launch over all problems of the class whose CTAs take
// segments of kFuseSeg consecutive elements of one problem (segments strided
// over the CTAs, x-neighbour pairs inside a segment summed in the CTA, masked
// points zeroed), then three passes over the class's problems: x-pairs between
// segments, y-pairs, z-pairs.  Finished problems are stepped over in one jump
// by every kernel.  Included by batch.cu (it needs BProb, ClsProb, c_b32_D).
#pragma once

namespace sem {

// what the batched fused kernels read of one problem, copied to shared memory
struct BApplyProb {
  const float* p;
  const float* G;
  const float* B;
  float* w;
  int E;
  float h1, h2;
  int nelx, nely, nelz, faces;
  int pad;
};
static_assert(sizeof(BApplyProb) == 64, "BApplyProb layout");

template <int P>
struct BApplyCfg {
  static constexpr int THREADS = P * P;
  static constexpr int STAGES = P >= 10 ? 1 : 2;
  static constexpr size_t smem(int ncls) {
    return 128 + (size_t)(STAGES * 8 + 3) * P * P * P * sizeof(float) + (size_t)ncls * 64;
  }
};

// A CTA's position in its sequence of elements: segment ordinal seg (over the
// class), element k of the segment, class problem c, element e of problem c.
struct SegCur {
  long long seg;
  int k, c, e;
};

// Element launch of one order class.  soff[c]: first segment ordinal of class
// problem c; Stot: segments of the class.
template <int P, int STAGES>
__global__ void __launch_bounds__(P * P)
bapply_kernel(const BProb* __restrict__ probs, const int* __restrict__ cls_prob,
              const long long* __restrict__ cls_soff, int ncls, long long Stot,
              int* __restrict__ err, uint64_t timeout_ns) {
  constexpr int P2 = P * P, P3 = P2 * P;
  constexpr int SV = 8 * P3;                      // values per stage: u, 6 G, B
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ long long s_soff[kMaxBatch + 1];
  __shared__ int s_skip[kMaxBatch];
  __shared__ unsigned s_fl;
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);
  float* stage0 = reinterpret_cast<float*>(smem_raw + 128);
  float* work = stage0 + STAGES * SV;
  BApplyProb* cp = reinterpret_cast<BApplyProb*>(work + 3 * P3);
  const int tid = threadIdx.x;
  for (int q = tid; q < ncls; q += blockDim.x) {
    s_soff[q] = cls_soff[q];
    const BProb& b = probs[cls_prob[q]];
    s_skip[q] = b.st->done;
    BApplyProb a;
    a.p = b.p;
    a.G = b.G;
    a.B = b.B;
    a.w = b.w;
    a.E = b.E;
    a.h1 = b.h1;
    a.h2 = b.h2;
    a.nelx = b.nelx;
    a.nely = b.nely;
    a.nelz = b.nelz;
    a.faces = b.faces;
    a.pad = 0;
    cp[q] = a;
  }
  if (tid == 0) {
    s_soff[ncls] = Stot;
#pragma unroll
    for (int s = 0; s < STAGES; ++s) mbar_init(&bar[s], 1);
    mbar_fence_init();
  }
  __syncthreads();
  const long long G = gridDim.x;
  // first segment at or after seg (in steps of G) whose problem is running
  auto resolve = [&](long long seg) {
    SegCur cur{seg, 0, 0, 0};
    while (cur.seg < Stot) {
      const int c = find_prob(s_soff, ncls, cur.seg);
      if (!s_skip[c]) {
        cur.c = c;
        cur.e = (int)(cur.seg - s_soff[c]) * kFuseSeg;
        return cur;
      }
      cur.seg += (s_soff[c + 1] - cur.seg + G - 1) / G * G;
    }
    return cur;
  };
  auto advance = [&](SegCur cur) {
    if (cur.k + 1 < kFuseSeg && cur.e + 1 < cp[cur.c].E) {
      ++cur.k;
      ++cur.e;
      return cur;
    }
    return resolve(cur.seg + G);
  };
  auto issue = [&](const SegCur& cur, int s) {
    const BApplyProb& pr = cp[cur.c];
    constexpr uint32_t FB = P3 * 4u;
    const bool helm = pr.h2 != 0.0f;
    float* dst = stage0 + s * SV;
    const uint64_t pol = l2_policy_evict_first();   // G and B are read once
    mbar_arrive_expect_tx(&bar[s], (helm ? 8u : 7u) * FB);
    bulk_g2s(dst, pr.p + (long long)cur.e * P3, FB, &bar[s]);
    bulk_g2s_hint(dst + P3, pr.G + (long long)cur.e * 6 * P3, 6 * FB, &bar[s], pol);
    if (helm) bulk_g2s_hint(dst + 7 * P3, pr.B + (long long)cur.e * P3, FB, &bar[s], pol);
  };
  SegCur ahead = resolve(blockIdx.x);                // thread 0: next element to prefetch
  int issued = 0;
  if (tid == 0) {
    for (int s = 0; s < STAGES && ahead.seg < Stot; ++s) {
      issue(ahead, s);
      ahead = advance(ahead);
      ++issued;
    }
  }
  auto Dm = [](int r, int c) { return c_b32_D[P][r * P + c]; };
  TileThread<P, float> t;
  t.init(tid, Dm);
  float* sT = work;
  float* swr = work + P3;
  float* swsT = work + 2 * P3;
  BoxWalk bw;                                       // thread 0
  int n = 0;
  for (SegCur cur = resolve(blockIdx.x); cur.seg < Stot; cur = advance(cur), ++n) {
    const int s = n % STAGES;
    const bool ok = mbar_wait_bounded(&bar[s], (uint32_t)(n / STAGES) & 1u, err, timeout_ns);
    const BApplyProb& pr = cp[cur.c];
    const bool helm = pr.h2 != 0.0f;
    const float* stage = stage0 + s * SV;
    float uc[P], bk[P], ck[P], wt[P];
    tile_load<P, float>(t, stage, helm ? stage + 7 * P3 : nullptr, nullptr, pr.h1, sT, uc, bk,
                        ck);
    if (__syncthreads_or(!ok)) {
      if (tid == 0)
        for (int nn = n; nn < issued; ++nn)
          mbar_wait_bounded(&bar[nn % STAGES], (uint32_t)(nn / STAGES) & 1u, err, timeout_ns);
      return;
    }
    if (tid == 0) {
      const FuseBox fb{pr.nelx, pr.nely, pr.nelz, pr.faces};
      if (cur.k == 0) bw.start(cur.e, fb); else bw.step(fb);
      s_fl = fused_flags(cur.e, bw, fb);
    }
    tile_forward<P, float>(t, stage, sT, stage + P3, uc, ck, swr, swsT, wt, Dm);
    __syncthreads();
    if (tid == 0 && ahead.seg < Stot) {            // stage s consumed
      fence_proxy_async_smem();
      issue(ahead, s);
      ahead = advance(ahead);
      ++issued;
    }
    FusedStore<P, float> fs;
    fs.we = pr.w + (long long)cur.e * P3;
    fs.fl = s_fl;
    tile_backward<P, float>(t, swr, swsT, wt, uc, bk, pr.h2, helm, Dm,
                            [&](int k, float v) { fs.store(t.i, t.j, k, v); });
  }
}

// The finishing passes of one class.  off[c]: first work item of class
// problem c in the pass; skip finished problems in one jump.
struct BFinProb {
  float* w;
  int nelx, nely, nelz, done;
};

__device__ __forceinline__ void bfin_load(const BProb* __restrict__ probs,
                                          const int* __restrict__ cls_prob,
                                          const long long* __restrict__ off, int ncls,
                                          long long total, long long* s_off, BFinProb* s_p) {
  for (int q = threadIdx.x; q < ncls; q += blockDim.x) {
    s_off[q] = off[q];
    const BProb& b = probs[cls_prob[q]];
    s_p[q] = BFinProb{b.w, b.nelx, b.nely, b.nelz, b.st->done};
  }
  if (threadIdx.x == 0) s_off[ncls] = total;
  __syncthreads();
}

// item t at or after t0 (steps of stride) whose problem is running; c out
__device__ __forceinline__ long long bfin_next(long long t, long long stride, long long total,
                                               const long long* s_off, const BFinProb* s_p,
                                               int ncls, int& c) {
  while (t < total) {
    c = find_prob(s_off, ncls, t);
    if (!s_p[c].done) return t;
    t += (s_off[c + 1] - t + stride - 1) / stride * stride;
  }
  return t;
}

// x-pairs at segment starts: item (boundary b, j, k), boundary b >= 0 is the
// start of segment b + 1 of the problem
template <int P>
__global__ void __launch_bounds__(256)
bcut_kernel(const BProb* __restrict__ probs, const int* __restrict__ cls_prob,
            const long long* __restrict__ off, int ncls, long long total) {
  constexpr int P2 = P * P, P3 = P2 * P;
  __shared__ long long s_off[kMaxBatch + 1];
  __shared__ BFinProb s_p[kMaxBatch];
  bfin_load(probs, cls_prob, off, ncls, total, s_off, s_p);
  const long long stride = (long long)gridDim.x * blockDim.x;
  int c = 0;
  for (long long t = bfin_next(blockIdx.x * (long long)blockDim.x + threadIdx.x, stride, total,
                               s_off, s_p, ncls, c);
       t < total; t = bfin_next(t + stride, stride, total, s_off, s_p, ncls, c)) {
    const long long r = t - s_off[c];
    const long long eb = (r / P2 + 1) * kFuseSeg;
    const BFinProb& b = s_p[c];
    if (eb % b.nelx == 0) continue;
    const int q = (int)(r % P2);
    const long long hi = eb * P3 + (long long)(q / P) * P2 + (q % P) * P;   // (eb, 0, j, k)
    const long long lo = hi - P3 + (P - 1);                             // (eb - 1, N, j, k)
    const float sum = b.w[lo] + b.w[hi];
    b.w[lo] = sum;
    b.w[hi] = sum;
  }
}

// y-pairs: item (i pair, k, element with ey < nely - 1), float2 per thread
template <int P>
__global__ void __launch_bounds__(256)
bsy_kernel(const BProb* __restrict__ probs, const int* __restrict__ cls_prob,
           const long long* __restrict__ off, int ncls, long long total) {
  constexpr int H = P / 2, P2 = P * P, P3 = P2 * P;
  __shared__ long long s_off[kMaxBatch + 1];
  __shared__ BFinProb s_p[kMaxBatch];
  bfin_load(probs, cls_prob, off, ncls, total, s_off, s_p);
  const long long stride = (long long)gridDim.x * blockDim.x;
  int c = 0;
  for (long long t = bfin_next(blockIdx.x * (long long)blockDim.x + threadIdx.x, stride, total,
                               s_off, s_p, ncls, c);
       t < total; t = bfin_next(t + stride, stride, total, s_off, s_p, ncls, c)) {
    const BFinProb& b = s_p[c];
    const long long r = t - s_off[c];
    const int ip = (int)(r % H);
    const long long r1 = r / H;
    const int k = (int)(r1 % P);
    const long long m = r1 / P;
    const long long ex = m % b.nelx, r2 = m / b.nelx;
    const long long ey = r2 % (b.nely - 1), ez = r2 / (b.nely - 1);
    const long long e = ex + (long long)b.nelx * (ey + (long long)b.nely * ez);
    float2* wv = reinterpret_cast<float2*>(b.w);
    const long long lo = (e * P3 + (long long)k * P2 + (P - 1) * P) / 2 + ip;
    const long long hi = ((e + b.nelx) * P3 + (long long)k * P2) / 2 + ip;
    const float2 a = wv[lo], bb = wv[hi];
    const float2 sum = make_float2(a.x + bb.x, a.y + bb.y);
    wv[lo] = sum;
    wv[hi] = sum;
  }
}

// z-pairs: item (float4 of the plane, element with ez < nelz - 1)
template <int P>
__global__ void __launch_bounds__(256)
bsz_kernel(const BProb* __restrict__ probs, const int* __restrict__ cls_prob,
           const long long* __restrict__ off, int ncls, long long total) {
  constexpr int P2 = P * P, P3 = P2 * P, Q = P2 / 4;
  __shared__ long long s_off[kMaxBatch + 1];
  __shared__ BFinProb s_p[kMaxBatch];
  bfin_load(probs, cls_prob, off, ncls, total, s_off, s_p);
  const long long stride = (long long)gridDim.x * blockDim.x;
  int c = 0;
  for (long long t = bfin_next(blockIdx.x * (long long)blockDim.x + threadIdx.x, stride, total,
                               s_off, s_p, ncls, c);
       t < total; t = bfin_next(t + stride, stride, total, s_off, s_p, ncls, c)) {
    const BFinProb& b = s_p[c];
    const long long r = t - s_off[c];
    const int q = (int)(r % Q);
    const long long e = r / Q;
    const long long layer = (long long)b.nelx * b.nely;
    float4* wv = reinterpret_cast<float4*>(b.w);
    const long long lo = (e * P3 + (long long)(P - 1) * P2) / 4 + q;
    const long long hi = ((e + layer) * P3) / 4 + q;
    float4 a = wv[lo];
    const float4 bb = wv[hi];
    a.x += bb.x;
    a.y += bb.y;
    a.z += bb.z;
    a.w += bb.w;
    wv[lo] = a;
    wv[hi] = a;
  }
}

}  // namespace sem
