// The batched solver's FP32 inner PCG on global (unique-dof) vectors (the
// single-problem form is global.cu and cg.cu): per order class, one
// persistent element launch over the elements of all problems of the class
// (each CTA gathers an element's u from its problem's lattice by cp.async,
// takes its geometric factors by a bulk copy, adds face values to the
// problem's w by L2 reductions), then per-problem-chunk vector kernels with
// plain dots that also clear w for the next operator.  Finished problems are
// stepped over.  At P = 8 the element kernel also forms <p, H p> from the
// local products (p is continuous and zero on Dirichlet points): each CTA
// adds its sum for a problem to the problem's accumulator when it moves to
// another problem, and the update kernel takes alpha = <r, z> / <p, H p>
// from it (no pw pass; the accumulation order, and so the last bits of
// alpha, vary from run to run, as the face sums of w already do).  Included by batch.cu (it needs BProb, c_b32_D, find_prob,
// item_sum, KahanF).
#pragma once

namespace sem {

// what the batched global kernel reads of one problem, in shared memory
struct BGlobProb {
  const float* u;
  float* w;
  double* pwacc;           // <p, H p> accumulated over the launch (P = 8)
  const float* G;
  const float* B;
  long long sk;            // lattice stride in z
  float h1, h2;
  int nelx, nely, nelz, faces, gx;
  FastDiv dnx, dny;
};

template <int P>
struct BGlobCfg {
  static constexpr int THREADS = P * P;
  // one stage of (6 G + B), two u buffers, transposed plane, two work planes
  static constexpr size_t smem(int ncls) {
    return 128 + (size_t)(7 + 5) * P * P * P * sizeof(float) + (size_t)ncls * sizeof(BGlobProb);
  }
};

// Element launch of one order class: item g = element g - eoff[c] of class
// problem c; Etot elements in the class.
template <int P>
__global__ void __launch_bounds__(P * P)
bglob_kernel(const BProb* __restrict__ probs, const int* __restrict__ cls_prob,
             const long long* __restrict__ cls_eoff, int ncls, long long Etot,
             int* __restrict__ err, uint64_t timeout_ns) {
  constexpr int P2 = P * P, P3 = P2 * P, N = P - 1;
  constexpr int SV = 7 * P3;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ long long s_off[kMaxBatch];
  __shared__ int s_skip[kMaxBatch];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);
  float* stage = reinterpret_cast<float*>(smem_raw + 128);
  float* su = stage + SV;                  // [2][P3]
  float* sT = su + 2 * P3;
  float* swr = su + 3 * P3;
  float* swsT = su + 4 * P3;
  BGlobProb* cp = reinterpret_cast<BGlobProb*>(su + 5 * P3);
  const int tid = threadIdx.x;
  for (int q = tid; q < ncls; q += blockDim.x) {
    s_off[q] = cls_eoff[q];
    const BProb& b = probs[cls_prob[q]];
    s_skip[q] = b.st->done;
    BGlobProb c;
    c.u = b.pg;
    c.w = b.wg;
    c.pwacc = b.pwacc;
    c.G = b.G;
    c.B = b.B;
    c.sk = (long long)b.gx * b.gy;
    c.h1 = b.h1;
    c.h2 = b.h2;
    c.nelx = b.nelx;
    c.nely = b.nely;
    c.nelz = b.nelz;
    c.faces = b.faces;
    c.gx = b.gx;
    c.dnx = b.dnx;
    c.dny = b.dny;
    cp[q] = c;
  }
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_fence_init();
  }
  __syncthreads();
  const long long Gs = gridDim.x;
  // first item at or after g whose problem is running; its class problem in c
  auto next = [&](long long g, int& c) {
    c = 0;
    while (g < Etot) {
      c = find_prob(s_off, ncls, g);
      if (!s_skip[c]) break;
      const long long end = c + 1 < ncls ? s_off[c + 1] : Etot;
      g += (end - g + Gs - 1) / Gs * Gs;
    }
    return g;
  };
  auto Dm = [](int r, int c) { return c_b32_D[P][r * P + c]; };
  TileThread<P, float> t;
  t.init(tid, Dm);
  // lattice index of element e's point (0, 0, 0) in problem pr; box position out
  auto origin = [&](const BGlobProb& pr, int e, int& ex, int& ey, int& ez) {
    const uint32_t r1 = pr.dnx.div((uint32_t)e);
    ex = e - (int)r1 * pr.nelx;
    const uint32_t q1 = pr.dny.div(r1);
    ey = (int)(r1 - q1 * (uint32_t)pr.nely);
    ez = (int)q1;
    return (long long)(ex * N) + (long long)pr.gx * (ey * N) + pr.sk * (long long)(ez * N);
  };
  // this thread's k-column of element g (problem c) into dst; returns the
  // lattice index of the element's point (0, 0, 0), box position in ex, ey, ez
  auto gather = [&](long long g, int c, float* dst, int& ex, int& ey, int& ez) {
    const BGlobProb& pr = cp[c];
    const long long org = origin(pr, (int)(g - s_off[c]), ex, ey, ez);
    const float* src = pr.u + org + t.i + (long long)pr.gx * t.j;
#pragma unroll
    for (int k = 0; k < P; ++k) cp_async4(dst + k * P2 + t.lt, src + pr.sk * k);
    return org;
  };
  auto issue = [&](long long g, int c) {
    const BGlobProb& pr = cp[c];
    const long long e = g - s_off[c];
    const bool helm = pr.h2 != 0.0f;
    constexpr uint32_t FB = P3 * sizeof(float);
    const uint64_t pol = l2_policy_evict_first();   // G and B are read once
    mbar_arrive_expect_tx(&bar[0], (helm ? 7u : 6u) * FB);
    bulk_g2s_hint(stage, pr.G + e * 6 * P3, 6 * FB, &bar[0], pol);
    if (helm) bulk_g2s_hint(stage + 6 * P3, pr.B + e * P3, FB, &bar[0], pol);
  };
  int c0;
  const long long g0 = next(blockIdx.x, c0);
  long long org_n = 0;                       // origin and box position of the element
  int exn = 0, eyn = 0, ezn = 0;             // whose u was gathered last
  if (tid == 0 && g0 < Etot) issue(g0, c0);
  if (g0 < Etot) org_n = gather(g0, c0, su, exn, eyn, ezn);
  cp_async_commit();
  const bool fi = t.i == 0 || t.i == N, fj = t.j == 0 || t.j == N;
  const unsigned pij = (t.i == 0 ? 4u : 0u) | (t.i == N ? 8u : 0u) | (t.j == 0 ? 16u : 0u) |
                       (t.j == N ? 32u : 0u);
  constexpr bool PW = (P * P) % 32 == 0;     // warp-aligned CTA: fused <p, H p>
  __shared__ double s_pw[P * P / 32 + 1];
  float pw_s = 0.0f, pw_c = 0.0f;             // Kahan sum of this CTA's current problem
  int pw_prob = -1;
  // adds the CTA's sum to problem pw_prob's accumulator (all threads call it)
  auto pw_flush = [&]() {
    if constexpr (PW) {
      double v = (double)pw_s - (double)pw_c;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
      if ((tid & 31) == 0) s_pw[tid >> 5] = v;
      __syncthreads();
      if (tid == 0 && pw_prob >= 0) {
        double tsum = 0.0;
        for (int q = 0; q < P * P / 32; ++q) tsum += s_pw[q];
        atomicAdd(cp[pw_prob].pwacc, tsum);
      }
      __syncthreads();
      pw_s = 0.0f;
      pw_c = 0.0f;
    }
  };
  int n = 0;
  int c = c0;
  for (long long g = g0; g < Etot; ++n) {
    const long long org = org_n;
    const int ex = exn, ey = eyn, ez = ezn;
    int cn;
    const long long gn = next(g + Gs, cn);
    const bool ok = mbar_wait_bounded(&bar[0], (uint32_t)n & 1u, err, timeout_ns);
    const float* cu = su + (n & 1) * P3;
    if (gn < Etot) org_n = gather(gn, cn, su + ((n + 1) & 1) * P3, exn, eyn, ezn);
    cp_async_commit();
    cp_async_wait<1>();
    if (PW && c != pw_prob) {
      if (pw_prob >= 0) pw_flush();
      pw_prob = c;
    }
    const BGlobProb& pr = cp[c];
    const bool helm = pr.h2 != 0.0f;
    float uc[P], bk[P], ck[P], wt[P];
#pragma unroll
    for (int k = 0; k < P; ++k) {
      uc[k] = cu[k * P2 + t.lt];
      sT[k * P2 + t.tpos] = uc[k];
      ck[k] = pr.h1;
      bk[k] = helm ? stage[6 * P3 + k * P2 + t.lt] : 0.0f;
    }
    if (__syncthreads_or(!ok)) {
      // the stage's copy did not complete: wait for it once more (bounded), leave
      cp_async_wait<0>();
      if (tid == 0) mbar_wait_bounded(&bar[0], (uint32_t)n & 1u, err, timeout_ns);
      return;
    }
    tile_forward<P, float>(t, cu, sT, stage, uc, ck, swr, swsT, wt, Dm);
    __syncthreads();
    if (tid == 0 && gn < Etot) {             // the stage is free
      fence_proxy_async_smem();
      issue(gn, cn);
    }
    float* we = pr.w + org + t.i + (long long)pr.gx * t.j;
    unsigned fl = 0;
    if (pr.faces) {
      fl = ((pr.faces & SEM_FACE_XMIN) && ex == 0 ? 4u : 0u) |
           ((pr.faces & SEM_FACE_XMAX) && ex == pr.nelx - 1 ? 8u : 0u) |
           ((pr.faces & SEM_FACE_YMIN) && ey == 0 ? 16u : 0u) |
           ((pr.faces & SEM_FACE_YMAX) && ey == pr.nely - 1 ? 32u : 0u) |
           ((pr.faces & SEM_FACE_ZMIN) && ez == 0 ? 64u : 0u) |
           ((pr.faces & SEM_FACE_ZMAX) && ez == pr.nelz - 1 ? 128u : 0u);
    }
    const long long skz = pr.sk;
    tile_backward<P, float>(t, swr, swsT, wt, uc, bk, pr.h2, helm, Dm, [&](int k, float v) {
      if constexpr (PW) {
        const float y = __fsub_rn(__fmul_rn(uc[k], v), pw_c);
        const float tt = __fadd_rn(pw_s, y);
        pw_c = __fsub_rn(__fsub_rn(tt, pw_s), y);
        pw_s = tt;
      }
      const unsigned pf = pij | (k == 0 ? 64u : 0u) | (k == N ? 128u : 0u);
      if (pf & fl) return;
      float* dst = we + skz * k;
      if (fi || fj || k == 0 || k == N)
        red_add(dst, v);
      else
        *dst = v;
    });
    g = gn;
    c = cn;
  }
  if (PW && pw_prob >= 0) pw_flush();
  cp_async_wait<0>();
}

// ---- vector kernels on global vectors: items of kGChunk values of one
// problem (a quarter of the L-vector item: small problems still give every
// SM several blocks)

// Starts the inner solve of the problems owning global items [item0, item0 + count).
__global__ void __launch_bounds__(256)
bginit_kernel(const BProb* __restrict__ probs, const int* __restrict__ item_prob, int item0,
              int count, int nitems, double* partials, unsigned* tickets, double tol, int maxit) {
  for (int it = item0 + blockIdx.x; it < item0 + count; it += gridDim.x) {
    const int pi = item_prob[it];
    const BProb& b = probs[pi];
    const long long lo = (long long)(it - b.g_off) * kGChunk;
    const long long hi = min(lo + kGChunk, b.nGp);
    KahanF rz, rr;
    for (long long q = lo + threadIdx.x; q < hi; q += blockDim.x) {
      const float r = b.rg[q];
      const float z = b.dinvg[q] * r;
      b.pg[q] = z;
      b.xg[q] = 0.0f;
      b.wg[q] = 0.0f;
      rz.add(__fmul_rn(r, z));
      rr.add(__fmul_rn(r, r));
    }
    double v[2] = {rz.value(), rr.value()}, tot[2];
    if (item_sum<2>(v, partials, it, b.g_off, b.g_cnt, &tickets[pi], tot, nitems) &&
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
      *b.pwacc = 0.0;
    }
    __syncthreads();
  }
}

// the global items of a launch, finished problems stepped over
struct GItemWalk {
  int goff[kMaxBatch + 1];
  int done[kMaxBatch];
  __device__ __forceinline__ void load(const BProb* __restrict__ probs, int nprob, int nitems) {
    for (int q = threadIdx.x; q < nprob; q += blockDim.x) {
      goff[q] = probs[q].g_off;
      done[q] = probs[q].st->done;
    }
    if (threadIdx.x == 0) goff[nprob] = nitems;
    __syncthreads();
  }
  __device__ __forceinline__ int next(const int* __restrict__ item_prob, int it, int stride,
                                      int nitems) const {
    while (it < nitems) {
      const int pi = item_prob[it];
      if (!done[pi]) break;
      it += (goff[pi + 1] - it + stride - 1) / stride * stride;
    }
    return it;
  }
};

__global__ void __launch_bounds__(256)
bgpw_kernel(const BProb* __restrict__ probs, const int* __restrict__ item_prob, int nprob,
            int nitems, double* partials, unsigned* tickets) {
  __shared__ GItemWalk wk;
  wk.load(probs, nprob, nitems);
  for (int it = wk.next(item_prob, blockIdx.x, gridDim.x, nitems); it < nitems;
       it = wk.next(item_prob, it + gridDim.x, gridDim.x, nitems)) {
    const int pi = item_prob[it];
    const BProb& b = probs[pi];
    if (b.fused_pw) continue;                // the element kernel formed <p, H p>
    const long long lo = (long long)(it - b.g_off) * kGChunk;
    const long long hi = min(lo + kGChunk, b.nGp);
    const float4* p4 = reinterpret_cast<const float4*>(b.pg + lo);
    const float4* w4 = reinterpret_cast<const float4*>(b.wg + lo);
    const int n4 = (int)((hi - lo) >> 2);
    KahanF pw;
#pragma unroll 4
    for (int q = threadIdx.x; q < n4; q += blockDim.x) {
      const float4 p = p4[q], w = w4[q];
      pw.add(__fmul_rn(p.x, w.x));
      pw.add(__fmul_rn(p.y, w.y));
      pw.add(__fmul_rn(p.z, w.z));
      pw.add(__fmul_rn(p.w, w.w));
    }
    double v[1] = {pw.value()}, tot[1];
    if (item_sum<1>(v, partials, it, b.g_off, b.g_cnt, &tickets[pi], tot, nitems) &&
        threadIdx.x == 0)
      st_after_pw(b.st, tot[0]);
    __syncthreads();
  }
}

__device__ __forceinline__ void gupd1(float& x, float& r, float p, float w, float d, float alpha,
                                      KahanF& rz, KahanF& rr) {
  x += alpha * p;
  r -= alpha * w;
  const float z = d * r;
  rz.add(__fmul_rn(r, z));
  rr.add(__fmul_rn(r, r));
}

// fused_pw: alpha = <r, z> / *pwacc (the element kernel accumulated <p, H p>);
// the problem's last item block checks it, records it and clears the accumulator
__global__ void __launch_bounds__(256)
bgupdate_kernel(const BProb* __restrict__ probs, const int* __restrict__ item_prob, int nprob,
                int nitems, double* partials, unsigned* tickets) {
  __shared__ GItemWalk wk;
  wk.load(probs, nprob, nitems);
  for (int it = wk.next(item_prob, blockIdx.x, gridDim.x, nitems); it < nitems;
       it = wk.next(item_prob, it + gridDim.x, gridDim.x, nitems)) {
    const int pi = item_prob[it];
    const BProb& b = probs[pi];
    const double pwv = b.fused_pw ? *(volatile double*)b.pwacc : 0.0;
    const float alpha = (float)(b.fused_pw ? b.st->rz / pwv : b.st->alpha);
    const long long lo = (long long)(it - b.g_off) * kGChunk;
    const long long hi = min(lo + kGChunk, b.nGp);
    float4* x4 = reinterpret_cast<float4*>(b.xg + lo);
    float4* r4 = reinterpret_cast<float4*>(b.rg + lo);
    const float4* p4 = reinterpret_cast<const float4*>(b.pg + lo);
    float4* w4 = reinterpret_cast<float4*>(b.wg + lo);
    const float4* d4 = reinterpret_cast<const float4*>(b.dinvg + lo);
    const int n4 = (int)((hi - lo) >> 2);
    const float4 zero = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    KahanF rz, rr;
#pragma unroll 2
    for (int q = threadIdx.x; q < n4; q += blockDim.x) {
      float4 x = x4[q], r = r4[q];
      const float4 p = p4[q], w = w4[q], d = d4[q];
      gupd1(x.x, r.x, p.x, w.x, d.x, alpha, rz, rr);
      gupd1(x.y, r.y, p.y, w.y, d.y, alpha, rz, rr);
      gupd1(x.z, r.z, p.z, w.z, d.z, alpha, rz, rr);
      gupd1(x.w, r.w, p.w, w.w, d.w, alpha, rz, rr);
      x4[q] = x;
      r4[q] = r;
      w4[q] = zero;
    }
    double v[2] = {rz.value(), rr.value()}, tot[2];
    if (item_sum<2>(v, partials, it, b.g_off, b.g_cnt, &tickets[pi], tot, nitems) &&
        threadIdx.x == 0) {
      CGState* st = b.st;
      if (b.fused_pw) {
        *b.pwacc = 0.0;
        st_after_pw(st, pwv);                // breakdown when <p, H p> <= 0
      }
      if (!st->done) st_after_update(st, tot);
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(256)
bgpupd_kernel(const BProb* __restrict__ probs, const int* __restrict__ item_prob, int nprob,
              int nitems) {
  __shared__ GItemWalk wk;
  wk.load(probs, nprob, nitems);
  for (int it = wk.next(item_prob, blockIdx.x, gridDim.x, nitems); it < nitems;
       it = wk.next(item_prob, it + gridDim.x, gridDim.x, nitems)) {
    const int pi = item_prob[it];
    const BProb& b = probs[pi];
    const float beta = (float)b.st->beta;
    const long long lo = (long long)(it - b.g_off) * kGChunk;
    const long long hi = min(lo + kGChunk, b.nGp);
    float4* p4 = reinterpret_cast<float4*>(b.pg + lo);
    const float4* r4 = reinterpret_cast<const float4*>(b.rg + lo);
    const float4* d4 = reinterpret_cast<const float4*>(b.dinvg + lo);
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
