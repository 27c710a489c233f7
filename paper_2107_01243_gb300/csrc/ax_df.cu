// FP64-accurate element operator w_e = (h1 D^T G_e D + h2 B_e) u_e (arXiv
// 2107.01243 §2, Eq. 9) evaluated in double-float arithmetic on the FP32
// pipes (df.cuh).  FP64 in, FP64 out; the geometric factors are stored as
// float pairs (8 bytes per value, the same traffic as FP64).
//
// A persistent CTA of 3 x P x P threads walks its elements; thread 0 keeps
// STAGES elements in flight with bulk copies (u_e as doubles, the 6 G pairs,
// B pairs for Helmholtz).  Contractions are "line tasks": a thread reads one
// line of P pairs and makes the P outputs of that line, so every D index is a
// compile-time constant (D's tables are immediates).  The three thread
// groups take the r-, s- and t-lines side by side and run the same code with
// different element positions, which keeps the kernel small enough for the instruction
// cache:
//   phase 0  u -> pairs U
//   forward  group g: lines of U along direction g -> UR | US | UT   (D)
//   G        every point: (WR, WS, WT) = h1 G (UR, US, UT), in place
//   backward group g: lines of W along direction g, in place          (D^T)
//   final    w = CR + CS + CT (+ h2 B u) -> double
// Sums use exact float transformations.  The forward derivatives use TwoSum
// and FMA product errors, whose error stays relative to the products where
// smooth u makes the derivatives cancel; the G products and the backward
// contractions use the cheaper extraction form (df.cuh: 7 instead of 12
// instructions a term), which lost 2-3 bits against TwoSum on the forward
// derivatives of smooth fields in a float32 emulation against the FP64
// oracle and about one bit where it is used.  D's tables are compile-time
// constants (df_tables.cuh).
// The shared-memory layout (DFLayout) keeps the line and point accesses free
// of bank conflicts; each thread computes its positions once per launch.
#include "sem_internal.cuh"
#include "tma.cuh"
#include "df.cuh"
#include "df_tables.cuh"
#include "ax_tile.cuh"
#include "reduce.cuh"
#include "cg_state.cuh"

namespace sem {

// D's even-odd tables as compile-time constants (df_tables.cuh, written by
// gen_df_tables.py): [t: D or D^T][A or S][high or low][i * (P/2) + l] with
// A = (M_il - M_i,N-l)/2, S = (M_il + M_i,N-l)/2, and the bounds of the
// transposed extraction dots

// h1 = m1 2^t1, h2 = m2 2^t2 with the mantissas as pairs (t = 0 while
// |h| lies in [2^-16, 2^16), see df.cuh)
struct DFScal {
  float h1h, h1l, h2h, h2l;
  int t1, t2;
};

// Shared-memory layout of one element's pairs.  P = 8: unpadded planes of 64
// pairs with rows and columns XOR-swizzled by the plane parity, position of
// (i, j, k) = 64 k + 8 (j ^ (k & 1)) + (i ^ ((j >> 1) + 4 (k & 1))): the i-, j-
// and k-lines read by the three thread groups and the per-point phases are
// all free of bank conflicts (16 threads of a half warp hit 16 distinct bank
// pairs), and an element takes 4 KB per array.  Other orders: rows padded to
// P + 2 and planes to 8 mod 16 pairs.
template <int P>
struct DFLayout {
  static constexpr int RS = P + 2;
  static constexpr int PL0 = P * RS;
  static constexpr int PL = PL0 + ((8 - (PL0 % 16)) + 16) % 16;
  static constexpr int VOL = P * PL;
  __device__ static int at(int i, int j, int k) { return k * PL + j * RS + i; }
};
template <>
struct DFLayout<8> {
  static constexpr int PL = 64;
  static constexpr int VOL = 8 * PL;
  __device__ static int at(int i, int j, int k) {
    return k * PL + 8 * (j ^ (k & 1)) + (i ^ (((j >> 1) + 4 * (k & 1)) & 7));
  }
};

// One line task: the P outputs y_i = sum_l M[i][l] x_l of the line whose
// elements sit at positions off[0..P) (M = D, or D^T when TRANS); in may equal out.
// M is centro-antisymmetric (M[N-i][N-l] = -M[i][l] on GLL nodes), so with
// e_l = x_l + x_{N-l}, o_l = x_l - x_{N-l} (l < P/2) the outputs come in pairs
// y_i = A o + S e, y_{N-i} = A o - S e with two (P/2)-term dots per pair.
template <int P, bool TRANS>
__device__ __forceinline__ void line_task(const float2* in, float2* out, const int (&off)[P]) {
  static_assert(P % 2 == 0, "even-odd split needs an even number of points");
  constexpr int H = P / 2, N = P - 1, T = TRANS ? 1 : 0;
  float xh[P], xl[P];
#pragma unroll
  for (int l = 0; l < P; ++l) {
    const float2 v = in[off[l]];
    xh[l] = v.x;
    xl[l] = v.y;
  }
  float eh[H], el[H], oh[H], ol[H];
#pragma unroll
  for (int l = 0; l < H; ++l) {
    dfadd(xh[l], xl[l], xh[N - l], xl[N - l], eh[l], el[l]);
    dfadd(xh[l], xl[l], -xh[N - l], -xl[N - l], oh[l], ol[l]);
  }
  // D annihilates constants (its rows sum to zero), hence so do the rows of S:
  // S e = sum_{l >= 1} S_il (e_l - e_0), one term fewer per dot for the
  // price of H - 1 pair subtractions.  D^T has no such property.
  constexpr int L0 = TRANS ? 0 : 1;
  if constexpr (!TRANS) {
#pragma unroll
    for (int l = 1; l < H; ++l) dfadd(eh[l], el[l], -eh[0], -el[0], eh[l], el[l]);
  }
  float yh[P], yl[P];
#pragma unroll
  for (int i = 0; i < H; ++i) {
    float Ph, Pl, Mh, Ml;
    tmac0(DFTab<P>::eo(T, 0, 0, i * H), DFTab<P>::eo(T, 0, 1, i * H), oh[0], ol[0], Ph, Pl);
    tmac0(DFTab<P>::eo(T, 1, 0, i * H + L0), DFTab<P>::eo(T, 1, 1, i * H + L0), eh[L0], el[L0], Mh,
          Ml);
#pragma unroll
    for (int l = 1; l < H; ++l)
      tmac(DFTab<P>::eo(T, 0, 0, i * H + l), DFTab<P>::eo(T, 0, 1, i * H + l), oh[l], ol[l], Ph, Pl);
#pragma unroll
    for (int l = L0 + 1; l < H; ++l)
      tmac(DFTab<P>::eo(T, 1, 0, i * H + l), DFTab<P>::eo(T, 1, 1, i * H + l), eh[l], el[l], Mh, Ml);
    dfadd(Ph, Pl, Mh, Ml, yh[i], yl[i]);
    dfadd(Ph, Pl, -Mh, -Ml, yh[N - i], yl[N - i]);
  }
#pragma unroll
  for (int i = 0; i < P; ++i) out[off[i]] = make_float2(yh[i], yl[i]);
}

// The transposed line task y_i = sum_l D_li x_l with extraction dots (df.cuh):
// the same even-odd split, with one power-of-two bound per output pair,
// sigma_i >= sum_l |A_il| |o_l| + |S_il| |e_l|.  P <= 8: the bound is taken
// from the row sums of the tables (DFTab::rb) and the largest |o| and |e| of
// the line; P = 10, whose rows are longer and whose bound that way is looser,
// forms the sum itself from the absolute entries (DFTab::ab).  Both tables
// are enlarged by 2^-18 to cover the roundings of the bound.  Both dots of a
// pair share sigma_i, so y_i = SP + SM and y_{N-i} = SP - SM are exact too.
template <int P>
__device__ __forceinline__ void line_task_xt(const float2* in, float2* out, const int (&off)[P]) {
  static_assert(P % 2 == 0, "even-odd split needs an even number of points");
  constexpr int H = P / 2, N = P - 1;
  float xh[P], xl[P];
#pragma unroll
  for (int l = 0; l < P; ++l) {
    const float2 v = in[off[l]];
    xh[l] = v.x;
    xl[l] = v.y;
  }
  float eh[H], el[H], oh[H], ol[H];
  float me = 0.0f, mo = 0.0f;
#pragma unroll
  for (int l = 0; l < H; ++l) {
    dfadd(xh[l], xl[l], xh[N - l], xl[N - l], eh[l], el[l]);
    dfadd(xh[l], xl[l], -xh[N - l], -xl[N - l], oh[l], ol[l]);
    me = fmaxf(me, fabsf(eh[l]));
    mo = fmaxf(mo, fabsf(oh[l]));
  }
#pragma unroll
  for (int i = 0; i < H; ++i) {
    float sig;
    if constexpr (P >= 10) {
      float b = 0.0f;
#pragma unroll
      for (int l = 0; l < H; ++l) {
        b = __fmaf_rn(DFTab<P>::ab(0, i * H + l), fabsf(oh[l]), b);
        b = __fmaf_rn(DFTab<P>::ab(1, i * H + l), fabsf(eh[l]), b);
      }
      sig = df_pow2_ceil(b);
    } else {
      sig = df_pow2_ceil(__fmaf_rn(DFTab<P>::rb(0, i), mo, __fmul_rn(DFTab<P>::rb(1, i), me)));
    }
    float SP, EP, SM, EM;
    xmac0(DFTab<P>::eo(1, 0, 0, i * H), DFTab<P>::eo(1, 0, 1, i * H), oh[0], ol[0], sig, SP, EP);
    xmac0(DFTab<P>::eo(1, 1, 0, i * H), DFTab<P>::eo(1, 1, 1, i * H), eh[0], el[0], sig, SM, EM);
#pragma unroll
    for (int l = 1; l < H; ++l) {
      xmac(DFTab<P>::eo(1, 0, 0, i * H + l), DFTab<P>::eo(1, 0, 1, i * H + l), oh[l], ol[l], sig, SP,
           EP);
      xmac(DFTab<P>::eo(1, 1, 0, i * H + l), DFTab<P>::eo(1, 1, 1, i * H + l), eh[l], el[l], sig, SM,
           EM);
    }
    // the line's inputs are all in registers, so the outputs may go out now
    out[off[i]] = make_float2(__fadd_rn(SP, SM), __fadd_rn(EP, EM));
    out[off[N - i]] = make_float2(__fsub_rn(SP, SM), __fsub_rn(EP, EM));
  }
}

// sum of three products g_a * v_a with extraction against sigma (df.cuh)
__device__ __forceinline__ void dot3_x(float2 g0, float2 g1, float2 g2, float2 v0, float2 v1,
                                       float2 v2, float sig, float& oh, float& ol) {
  float S, E;
  xmac0(g0.x, g0.y, v0.x, v0.y, sig, S, E);
  xmac(g1.x, g1.y, v1.x, v1.y, sig, S, E);
  xmac(g2.x, g2.y, v2.x, v2.y, sig, S, E);
  oh = S;
  ol = E;
}

// Three groups of P x P threads, one per direction, run the line tasks of the
// r-, s- and t-direction side by side.
//
// FUSE: the CTA walks segments of kFuseSeg consecutive elements and writes
// the fused output (FusedStore: mask, x-neighbour pairs of the segment summed
// in the CTA) for the assembled operator of apply.cu.
//
// Range (df.cuh): esc[e] holds the element's power-of-two exponents of G and
// B (bits 0-15 and 16-31, signed; the float pairs hold G 2^-sG and B 2^-sB).
// Each warp takes the largest magnitude key of its u values; the CTA barrier
// after the conversion also tells whether some warp saw a key outside
// [2^-60, 2^76).  Then (rarely) the whole CTA reads the element maximum and
// either rescales u by 2^-kU, kU = floor(log2 max |u_e|), or, for an Inf or
// NaN in u_e, marks the element, whose outputs are then all NaN.  Thread 0
// combines the exponents into the element's coefficients c1, c2 (both
// <= 2 in magnitude after scaling, or h1, h2 themselves in the common case)
// and the output exponent, by which the FP64 result is multiplied.
template <int P, int STAGES, int MODE>
__global__ void __launch_bounds__(3 * P * P, P == 8 ? 5 : 1)     // P = 8: five CTAs per SM
ax_df_kernel(const double* __restrict__ u, double* __restrict__ w, const float2* __restrict__ G,
             const float2* __restrict__ B, const int* __restrict__ esc, DFScal C, int E,
             const CGState* __restrict__ st, int* __restrict__ err, uint64_t timeout_ns,
             FuseBox fb, CGState* __restrict__ pwst, double* __restrict__ partials) {
  // MODE 0: plain output; 1: fused output (FUSE); 2: fused output and
  // <p, H p> (PW, pwst set; whole-warp CTAs only)
  constexpr bool FUSE = MODE >= 1, PW = MODE == 2;
  static_assert(!PW || (3 * P * P) % 32 == 0, "<p, H p> needs whole-warp CTAs");
  using L = DFLayout<P>;
  constexpr int P2 = P * P, P3 = P2 * P, NT = 3 * P2;
  constexpr int NW = (NT + 31) / 32;
  constexpr unsigned LASTMASK = (NT % 32) ? ((1u << (NT % 32)) - 1u) : 0xffffffffu;
  constexpr uint32_t UB = P3 * sizeof(double), GB = 6 * P3 * sizeof(float2),
                     BB = P3 * sizeof(float2);
  if (st && st->done) return;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);
  const bool helm = (C.h2h != 0.0f);
  const uint32_t SB = UB + GB + (helm ? BB : 0);          // stage bytes
  unsigned char* stage0 = smem_raw + 128;
  float2* U = reinterpret_cast<float2*>(stage0 + STAGES * SB);
  float2* R[3] = {U + L::VOL, U + 2 * L::VOL, U + 3 * L::VOL};   // r, s, t work arrays
  const int tid = threadIdx.x;
  const int g = tid / P2, lam = tid % P2;
  const int c1 = lam % P, c2 = lam / P;
  const int warp = tid >> 5;
  const unsigned wmask = (warp == NW - 1) ? LASTMASK : 0xffffffffu;
  // line of direction g: r: (j=c1, k=c2); s: (i=c1, k=c2); t: (i=c1, j=c2);
  // its element positions and this thread's point positions, fixed for the kernel
  int loff[P];
#pragma unroll
  for (int l = 0; l < P; ++l)
    loff[l] = g == 0 ? L::at(l, c1, c2) : (g == 1 ? L::at(c1, l, c2) : L::at(c1, c2, l));
  constexpr int NQ = (P3 + NT - 1) / NT;
  int qoff[NQ];
#pragma unroll
  for (int m = 0; m < NQ; ++m) {
    const int q = tid + m * NT;
    qoff[m] = q < P3 ? L::at(q % P, (q / P) % P, q / P2) : 0;
  }
  float2* myR = g == 0 ? R[0] : (g == 1 ? R[1] : R[2]);
  const ItemSeq<FUSE> seq{E};          // this CTA's elements in order
  // FUSE: NT = 3 P^2, so every point of this thread has i = tid % P and
  // j = (tid / P) % P, and k = tid / P^2 + 3 m: the i- and j-face bits of its
  // points (fused_flags' layout) are fixed for the kernel
  static_assert(NT == 3 * P2, "points of a thread must share their i and j");
  const unsigned pij = ((tid % P) == 0 ? 4u : 0u) | ((tid % P) == P - 1 ? 8u : 0u) |
                       (((tid / P) % P) == 0 ? 16u : 0u) | (((tid / P) % P) == P - 1 ? 32u : 0u);
  const int k0 = tid / P2;
  const bool xlow = (tid % P) == 0;    // this thread's points pair with e - 1 along x

  // the element's exponent word comes with its stage (a 4-byte cp.async that
  // thread 0 completes before it reads the word), so that the per-element
  // setup of thread 0 does not wait on a global load
  __shared__ int s_esc[STAGES];
  // u_e, G_e and B_e are read once: they leave L2 first, so that the output
  // w, which the gather-scatter passes read back, stays there
  auto issue = [&](int e, int s) {
    unsigned char* dst = stage0 + s * SB;
    const uint64_t pol = l2_policy_evict_first();
    mbar_arrive_expect_tx(&bar[s], SB);
    bulk_g2s_hint(dst, u + (size_t)e * P3, UB, &bar[s], pol);
    bulk_g2s_hint(dst + UB, G + (size_t)e * 6 * P3, GB, &bar[s], pol);
    if (helm) bulk_g2s_hint(dst + UB + GB, B + (size_t)e * P3, BB, &bar[s], pol);
    cp_async4(&s_esc[s], esc + e);
    cp_async_commit();
  };
  if (tid == 0) {
#pragma unroll
    for (int s = 0; s < STAGES; ++s) mbar_init(&bar[s], 1);
    mbar_fence_init();
  }
  __syncthreads();
  // thread 0's state, kept in shared memory so that it takes no registers in
  // the other threads: next element to prefetch, copies issued, box position
  __shared__ struct {
    int ahead, issued;
    BoxWalk bw;
  } s_pr;
  if (tid == 0) {
    int ahead = seq.first(), issued = 0;
#pragma unroll
    for (int s = 0; s < STAGES; ++s) {
      if (ahead < E) {
        issue(ahead, s);
        ahead = seq.next(ahead);
        ++issued;
      }
    }
    s_pr.ahead = ahead;
    s_pr.issued = issued;
  }

  __shared__ unsigned s_fl;            // FusedStore flags of the current element
  __shared__ unsigned s_key[NW];       // per-warp magnitude keys of u_e
  __shared__ float4 s_cf;              // the element's c1 (x, y) and c2 (z, w) pairs
  __shared__ int2 s_ci;                // output exponent; <p, H p> rescaling exponent
  // FUSE with pwst: <p, H p> = sum over local points of p (H_L p) (p continuous
  // and zero on Dirichlet points), accumulated per thread in pair arithmetic;
  // elements with a nonzero scaling exponent are added in FP64 (pw_d)
  float pw_s = 0.0f, pw_e = 0.0f;
  double pw_d = 0.0;
  int n = 0;
  for (int e = seq.first(); e < E; e = seq.next(e), ++n) {
    const int s = n % STAGES;
    const bool ok = mbar_wait_bounded(&bar[s], (uint32_t)(n / STAGES) & 1u, err, timeout_ns);
    const double* su = reinterpret_cast<const double*>(stage0 + s * SB);
    const float2* sg = reinterpret_cast<const float2*>(stage0 + s * SB + UB);
    const float2* sb = reinterpret_cast<const float2*>(stage0 + s * SB + UB + GB);
    // phase 0: u -> pairs, and the warp's largest magnitude key
    unsigned key = 0u, lor = 0u;
#pragma unroll
    for (int m = 0; m < NQ; ++m) {
      const int q = tid + m * NT;
      if ((m + 1) * NT <= P3 || q < P3) {
        const double x = su[q];
        const unsigned long long xb = (unsigned long long)__double_as_longlong(x);
        key = max(key, (unsigned)(xb >> 32) & 0x7FFFFFFFu);
        lor |= (unsigned)xb;
        float hi, lo;
        d2df(x, hi, lo);
        U[qoff[m]] = make_float2(hi, lo);
      }
    }
    key |= (lor != 0u) ? 1u : 0u;
    const unsigned wkey = __reduce_max_sync(wmask, key);
    if ((tid & 31) == 0) s_key[warp] = wkey;
    const bool wbad = wkey != 0u && (wkey - kDfKeyLo) >= (kDfKeyHi - kDfKeyLo);
    int kU = 0;                        // u_e was scaled by 2^-kU
    bool nanel = false;                // u_e holds an Inf or NaN
    if (__syncthreads_or(!ok || wbad)) {
      if (__syncthreads_or(!ok)) {
        if (tid == 0) {
          for (int nn = n; nn < s_pr.issued; ++nn)
            mbar_wait_bounded(&bar[nn % STAGES], (uint32_t)(nn / STAGES) & 1u, err, timeout_ns);
          cp_async_wait<0>();
        }
        break;                         // the reduction below still counts this CTA
      }
      unsigned km = 0u;
#pragma unroll
      for (int w2 = 0; w2 < NW; ++w2) km = max(km, s_key[w2]);
      if (km >= kDfKeyNonFinite) {
        nanel = true;
      } else if (km < kDfKeyLo || km >= kDfKeyHi) {
        kU = df_key_exp(km);           // the same value in every thread
        const int ka = -kU / 2;
        const double sa = df_pow2d(ka), sbb = df_pow2d(-kU - ka);
#pragma unroll
        for (int m = 0; m < NQ; ++m) {
          const int q = tid + m * NT;
          if (q < P3) {
            float hi, lo;
            d2df(su[q] * sa * sbb, hi, lo);
            U[qoff[m]] = make_float2(hi, lo);
          }
        }
        __syncthreads();
      }
    }
    if (tid == 0) {
      if (FUSE) {                      // box position of e, read back in the output phase
        if (e % kFuseSeg == 0) s_pr.bw.start(e, fb); else s_pr.bw.step(fb);
        s_fl = fused_flags(e, s_pr.bw, fb);
      }
      // the element's coefficients and exponents
      cp_async_wait<0>();
      const int sw = s_esc[s];
      const int a1 = (int)(short)(sw & 0xFFFF) + C.t1;
      const int a2 = helm ? (sw >> 16) + C.t2 : a1;
      const int unit = max(a1, a2);
      s_cf = make_float4(df_scale_down(C.h1h, a1 - unit), df_scale_down(C.h1l, a1 - unit),
                         df_scale_down(C.h2h, a2 - unit), df_scale_down(C.h2l, a2 - unit));
      int kE = 0;
      if (PW && kU == 0 && !nanel) {
        unsigned km = 0u;
#pragma unroll
        for (int w2 = 0; w2 < NW; ++w2) km = max(km, s_key[w2]);
        if (km != 0u && (km < kDfPwLo || km >= kDfPwHi)) kE = df_key_exp(km);
      }
      s_ci = make_int2(unit + kU, kE);
    }
    // forward derivatives: group g differentiates along direction g
    line_task<P, false>(U, myR, loff);
    __syncthreads();
    // geometric factors at every point: (WR, WS, WT) = c1 G (UR, US, UT), in place
    const float4 cf = s_cf;
    const bool scale1 = !(cf.x == 1.0f && cf.y == 0.0f);
#pragma unroll
    for (int m = 0; m < NQ; ++m) {
      const int q = tid + m * NT;
      if ((m + 1) * NT > P3 && q >= P3) break;
      const int at = qoff[m];
      const float2 g11 = sg[q], g22 = sg[P3 + q], g33 = sg[2 * P3 + q];
      const float2 g12 = sg[3 * P3 + q], g13 = sg[4 * P3 + q], g23 = sg[5 * P3 + q];
      const float2 ur = R[0][at], us = R[1][at], ut = R[2][at];
      float rh, rl, sh, sl, th, tl;
      // one bound for the point's three rows: 3 max|G| max|u'| (1 + 2^-18)
      const float mg = fmaxf(fmaxf(fmaxf(fabsf(g11.x), fabsf(g22.x)), fmaxf(fabsf(g33.x),
                                                                         fabsf(g12.x))),
                             fmaxf(fabsf(g13.x), fabsf(g23.x)));
      const float mu = fmaxf(fmaxf(fabsf(ur.x), fabsf(us.x)), fabsf(ut.x));
      const float sig = df_pow2_ceil(__fmul_rn(__fmul_rn(mg, 3.0f * (1.0f + 0x1p-18f)), mu));
      dot3_x(g11, g12, g13, ur, us, ut, sig, rh, rl);
      dot3_x(g12, g22, g23, ur, us, ut, sig, sh, sl);
      dot3_x(g13, g23, g33, ur, us, ut, sig, th, tl);
      if (scale1) {
        dfmul(cf.x, cf.y, rh, rl, rh, rl);
        dfmul(cf.x, cf.y, sh, sl, sh, sl);
        dfmul(cf.x, cf.y, th, tl, th, tl);
      }
      R[0][at] = make_float2(rh, rl);
      R[1][at] = make_float2(sh, sl);
      R[2][at] = make_float2(th, tl);
    }
    __syncthreads();
    if (!helm && tid == 0) {                   // stage s consumed
      if (s_pr.ahead < E) {
        fence_proxy_async_smem();
        issue(s_pr.ahead, s);
        s_pr.ahead = seq.next(s_pr.ahead);
        ++s_pr.issued;
      }
    }
    // transposed derivatives, in place: group g along direction g
    line_task_xt<P>(myR, myR, loff);
    __syncthreads();
    // w = CR + CS + CT (+ c2 B u), times 2^oexp -> double
    const int2 ci = s_ci;
    // <p, H p> of an element with a nonzero exponent: the running pair is
    // moved to FP64 first, the element's own sum is scaled and added after
    const int pwexp = 2 * (ci.y + kU) + ci.x - kU;
    if (PW && (pwexp != 0 || nanel)) {
      pw_d += (double)pw_s + (double)pw_e;
      pw_s = 0.0f;
      pw_e = 0.0f;
    }
    double* we = w + (size_t)e * P3;
    // FUSE: masked points are written as zero, and the i = 0 points of an
    // element that pairs with e - 1 add the copy e - 1 stored before
    const unsigned fl = FUSE ? s_fl : 0u;
    const bool xpair = (fl & 1u) && xlow;
    // MODE 1: the lower neighbour's copies of this thread's i = 0 points read
    // before the output sums, so that the loads overlap them
    double xprev[NQ];
    if constexpr (FUSE && !PW) {
#pragma unroll
      for (int m = 0; m < NQ; ++m) {
        const int q = tid + m * NT;
        xprev[m] = (xpair && ((m + 1) * NT <= P3 || q < P3)) ? we[q - P3 + (P - 1)] : 0.0;
      }
    }
#pragma unroll
    for (int m = 0; m < NQ; ++m) {
      const int q = tid + m * NT;
      if ((m + 1) * NT > P3 && q >= P3) break;
      const int at = qoff[m];
      const float2 cr = R[0][at], cs = R[1][at], ct = R[2][at];
      float S = cr.x, er = cr.y;
      tadd(cs.x, cs.y, S, er);
      tadd(ct.x, ct.y, S, er);
      if (helm) {
        const float2 bv = sb[q], uv = U[at];
        float bh, bl;
        dfmul(cf.z, cf.w, bv.x, bv.y, bh, bl);
        tmac(bh, bl, uv.x, uv.y, S, er);
      }
      if constexpr (PW) {
        float2 pv = U[at];
        float ws = S, wl = er;
        if (ci.y != 0) {               // p and H p times 2^-kE, into [1, 2^49)
          const float f = __int_as_float((127 - ci.y) << 23);
          pv.x = __fmul_rn(pv.x, f);
          pv.y = __fmul_rn(pv.y, f);
          ws = __fmul_rn(ws, f);
          wl = __fmul_rn(wl, f);
        }
        tmac(pv.x, pv.y, ws, wl, pw_s, pw_e);
      }
      double val = (double)S + (double)er;   // exact widenings, one rounding
      if (ci.x != 0) val = df_ldexp(val, ci.x);
      if (nanel) val = __longlong_as_double(0x7FF8000000000000ll);
      if constexpr (FUSE) {
        const int k = k0 + 3 * m;
        const unsigned pf = pij | (k == 0 ? 64u : 0u) | (k == P - 1 ? 128u : 0u);
        if (pf & fl & 0xFCu) val = 0.0;
        if (xpair) {
          double* lo = we + q - P3 + (P - 1);
          const double sum = (FUSE && !PW ? xprev[m] : *lo) + val;
          *lo = sum;
          val = sum;
        }
      }
      we[q] = val;
    }
    if (PW && (pwexp != 0 || nanel)) {
      pw_d += nanel ? __longlong_as_double(0x7FF8000000000000ll)
                    : df_ldexp((double)pw_s + (double)pw_e, pwexp);
      pw_s = 0.0f;
      pw_e = 0.0f;
    }
    if (helm) {
      __syncthreads();                         // U and the stage are free
      if (tid == 0) {
        if (s_pr.ahead < E) {
          fence_proxy_async_smem();
          issue(s_pr.ahead, s);
          s_pr.ahead = seq.next(s_pr.ahead);
          ++s_pr.issued;
        }
      }
    }
  }
  if constexpr (PW) {
    double v[1] = {((double)pw_s + (double)pw_e) + pw_d};
    double tot[1];
    if (grid_sum<1>(v, partials, &pwst->counter, tot) && threadIdx.x == 0) {
      st_after_pw(pwst, tot[0]);
    }
  }
}

// ---------------------------------------------------------------- launch
// h = m 2^t with t = df_pick_exp(|h|) and m as a pair (exact: m is h times a
// power of two, split into its leading 24 bits and the next 24)
static void df_split_scalar(double h, float& hi, float& lo, int& t) {
  t = df_pick_exp(std::fabs(h));
  const double m = std::ldexp(h, -t);
  hi = (float)m;
  lo = (float)(m - (double)hi);
}

template <int P, int STAGES>
static size_t df_smem_bytes(bool helm) {
  using L = DFLayout<P>;
  const size_t P3 = (size_t)P * P * P;
  const size_t SB = P3 * 8 + 6 * P3 * 8 + (helm ? P3 * 8 : 0);
  return 128 + STAGES * SB + 4 * (size_t)L::VOL * sizeof(float2);
}

// A slab of whole element planes: elements [e0, e0 + E) of the handle, the
// box fb (its nelz the slab's planes, its faces those the slab touches).
struct DFSlab {
  int64_t e0;
  int E;
  FuseBox fb;
};

// CTAs per SM of one kernel variant (Poisson or Helmholtz stage size); the
// first call also sets the variant's shared-memory attributes
template <int P, int STAGES, int MODE>
static int df_occupancy(bool helm) {
  auto kern = ax_df_kernel<P, STAGES, MODE>;
  static bool configured = false;
  static int occ[2] = {0, 0};
  if (!configured) {
    SEM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)df_smem_bytes<P, STAGES>(true)));
    SEM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                  (int)cudaSharedmemCarveoutMaxShared));
    configured = true;
  }
  int& o = occ[helm ? 1 : 0];
  if (!o) {
    SEM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, 3 * P * P,
                                                           df_smem_bytes<P, STAGES>(helm)));
    if (o < 1) o = 1;
  }
  return o;
}

template <int P>
static void df_prepare_p(const sem_handle* h) {
  for (int helm = 0; helm < 2; ++helm) {
    df_occupancy<P, 1, 0>(helm != 0);
    df_occupancy<P, 2, 0>(helm != 0);
    df_occupancy<P, 1, 1>(helm != 0);
    df_occupancy<P, 2, 1>(helm != 0);
    if constexpr ((3 * P * P) % 32 == 0) {
      df_occupancy<P, 1, 2>(helm != 0);
      df_occupancy<P, 2, 2>(helm != 0);
    }
  }
}

// The once-per-process setup of the double-float kernels (constant tables,
// kernel attributes, occupancies), run by sem_setup: outside any stream
// capture, so that a solve captured into a CUDA graph as the first call of a
// process makes no synchronous copy inside the capture.
void df_prepare(const sem_handle* h) {
  switch (h->P) {
    case 6: df_prepare_p<6>(h); break;
    case 8: df_prepare_p<8>(h); break;
    case 10: df_prepare_p<10>(h); break;
    default: break;
  }
}

// returns the grid it launched (the fused operator's later passes need it)
template <int P, int STAGES, int MODE = 0>
static int launch_df_p(const sem_handle* h, const double* u, double* w, double h1, double h2,
                       const CGState* st, cudaStream_t s, CGState* pwst = nullptr,
                       const DFSlab* slab = nullptr) {
  const bool helm = h2 != 0.0;
  const size_t smem = df_smem_bytes<P, STAGES>(helm);
  auto kern = ax_df_kernel<P, STAGES, MODE>;
  const int o = df_occupancy<P, STAGES, MODE>(helm);
  DFScal c;
  df_split_scalar(h1, c.h1h, c.h1l, c.t1);
  df_split_scalar(h2, c.h2h, c.h2l, c.t2);
  const int E = slab ? slab->E : (int)h->E;
  const int64_t e0 = slab ? slab->e0 : 0;
  constexpr int64_t P3 = (int64_t)P * P * P;
  int grid = (int)std::min<int64_t>(E, (int64_t)o * sem_num_sms());
  if (grid < 1) grid = 1;
  if (pwst) grid = std::min(grid, kFusedPartials);
  const FuseBox fb = slab ? slab->fb : FuseBox{h->nelx, h->nely, h->nelz, h->faces};
  kern<<<grid, 3 * P * P, smem, s>>>(u + e0 * P3, w + e0 * P3, h->gdf.ptr + e0 * 6 * P3,
                                     h->bdf.ptr ? h->bdf.ptr + e0 * P3 : nullptr,
                                     h->escale.ptr + e0, c, E, st, h->dev_err.ptr,
                                     kWaitTimeoutNs, fb, pwst, h->partials.ptr + 4 * kRedBlocks);
  SEM_CHECK_LAUNCH();
  return grid;
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
    case 6:
      if (h->tune.df_variant) launch_df_p<6, 2>(h, u, w, h1, h2, st, s);
      else launch_df_p<6, 1>(h, u, w, h1, h2, st, s);
      break;
    case 8:
      if (h->tune.df_variant) launch_df_p<8, 2>(h, u, w, h1, h2, st, s);
      else launch_df_p<8, 1>(h, u, w, h1, h2, st, s);
      break;
    case 10:
      if (h->tune.df_variant) launch_df_p<10, 2>(h, u, w, h1, h2, st, s);
      else launch_df_p<10, 1>(h, u, w, h1, h2, st, s);
      break;
    default: throw Error(SEM_ERR_ARG, "launch_ax_df: unsupported order");
  }
}

// pwst (may be NULL): state that receives <p, H p> and alpha, for the order
// whose CTAs are whole warps (P = 8); returns whether it was computed
bool launch_ax_df_fused(const sem_handle* h, const double* u, double* w, double h1, double h2,
                        const CGState* st, CGState* pwst, cudaStream_t s) {
  const bool two = h->tune.df_variant != 0;
  switch (h->P) {
    case 6:
      if (two) launch_df_p<6, 2, 1>(h, u, w, h1, h2, st, s);
      else launch_df_p<6, 1, 1>(h, u, w, h1, h2, st, s);
      return false;
    case 8:
      if (pwst) {
        if (two) launch_df_p<8, 2, 2>(h, u, w, h1, h2, st, s, pwst);
        else launch_df_p<8, 1, 2>(h, u, w, h1, h2, st, s, pwst);
      } else {
        if (two) launch_df_p<8, 2, 1>(h, u, w, h1, h2, st, s);
        else launch_df_p<8, 1, 1>(h, u, w, h1, h2, st, s);
      }
      return pwst != nullptr;
    case 10:
      if (two) launch_df_p<10, 2, 1>(h, u, w, h1, h2, st, s);
      else launch_df_p<10, 1, 1>(h, u, w, h1, h2, st, s);
      return false;
    default: throw Error(SEM_ERR_ARG, "launch_ax_df_fused: unsupported order");
  }
}

// The fused element kernel on the slab of element planes [z0, z1): faces of
// the box that the slab does not touch are not Dirichlet faces of the slab.
void launch_ax_df_fused_slab(const sem_handle* h, const double* u, double* w, double h1,
                             double h2, int z0, int z1, cudaStream_t s) {
  const int64_t layer = (int64_t)h->nelx * h->nely;
  int faces = h->faces;
  if (z0 > 0) faces &= ~SEM_FACE_ZMIN;
  if (z1 < h->nelz) faces &= ~SEM_FACE_ZMAX;
  const DFSlab sl{z0 * layer, (int)((z1 - z0) * layer), FuseBox{h->nelx, h->nely, z1 - z0, faces}};
  const bool two = h->tune.df_variant != 0;
  switch (h->P) {
    case 6:
      if (two) launch_df_p<6, 2, 1>(h, u, w, h1, h2, nullptr, s, nullptr, &sl);
      else launch_df_p<6, 1, 1>(h, u, w, h1, h2, nullptr, s, nullptr, &sl);
      break;
    case 8:
      if (two) launch_df_p<8, 2, 1>(h, u, w, h1, h2, nullptr, s, nullptr, &sl);
      else launch_df_p<8, 1, 1>(h, u, w, h1, h2, nullptr, s, nullptr, &sl);
      break;
    case 10:
      if (two) launch_df_p<10, 2, 1>(h, u, w, h1, h2, nullptr, s, nullptr, &sl);
      else launch_df_p<10, 1, 1>(h, u, w, h1, h2, nullptr, s, nullptr, &sl);
      break;
    default: throw Error(SEM_ERR_ARG, "launch_ax_df_fused_slab: unsupported order");
  }
}

}  // namespace sem
