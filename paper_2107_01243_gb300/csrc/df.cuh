// Double-float ("df") arithmetic on the FP32 pipes for FP64-accurate results.
//
// A value is an unevaluated pair hi + lo of floats (about 48 significant bits).
// GB300 runs FP32 FMA 60x faster than FP64 FMA, so FP64-accurate kernels that
// would be bound by the FP64 pipe run on pairs instead.  The conversion from
// double uses integer bit manipulation only (no FP64 instructions); results
// go back to double as the exact widening of both parts and one FP64 add.
//
// Dot products keep the running sum S of the rounded high-part products and
// an FP32 error term: each product's rounding error comes from an FMA, each
// addition's from TwoSum (Knuth), both exact; the low-part cross terms are
// added to the error term in FP32.  The error of a result is then about
// 2^-48 of the largest partial sum.  Every rounding below is requested
// explicitly (the _rn intrinsics are never contracted into FMAs).
#pragma once
#include <stdint.h>

namespace sem {

// double -> (hi, lo): hi keeps the top 24 significand bits (truncated), lo the
// next 23.  |x| below 2^-80 keeps hi only; zero and denormals give (0, 0).
__device__ __forceinline__ void d2df(double x, float& hi, float& lo) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  const unsigned int h32 = (unsigned int)(bits >> 32), l32 = (unsigned int)bits;
  const unsigned int sign = h32 & 0x80000000u;
  const int ex = (int)((h32 >> 20) & 0x7FF);
  const int fe = ex - 1023 + 127;
  // the funnel shift leaves ex's low 9 bits in 31..23 and the top 23
  // significand bits below them; adding 2^30 subtracts 896 from the exponent
  // modulo 2^9, which gives fe with bit 31 clear for fe in [1, 254]
  const float h = __uint_as_float(((__funnelshift_l(l32, h32, 3) + 0x40000000u) & 0x7FFFFFFFu) |
                                  sign);
  // remaining 29 bits: keep the top 23 as an exact float integer, then scale
  const unsigned int r = (l32 & 0x1FFFFFFFu) >> 6;
  const float ri = __fsub_rn(__uint_as_float(0x4B000000u | r), 8388608.0f);
  const int se = ex - 942;                       // 2^(ex - 1075 + 6) as a float exponent
  const float scale = se > 0 ? __int_as_float(se << 23) : 0.0f;
  const float l = __uint_as_float(__float_as_uint(__fmul_rn(ri, scale)) | sign);
  // selects rather than a branch: fe <= 0 (below FP32's normal range) gives 0
  hi = fe > 0 ? h : 0.0f;
  lo = fe > 0 ? l : 0.0f;
}

// First term of a dot product: (S, err) = c z exactly up to the dropped cl zl.
__device__ __forceinline__ void tmac0(float ch, float cl, float zh, float zl, float& S,
                                      float& err) {
  const float p = __fmul_rn(ch, zh);
  float e = __fmaf_rn(ch, zh, -p);
  e = __fmaf_rn(ch, zl, e);
  S = p;
  err = __fmaf_rn(cl, zh, e);
}

// Next term: S + RN(c zh) by TwoSum (exact), the product error by FMA (exact);
// both errors and the low-part cross terms go to err.
__device__ __forceinline__ void tmac(float ch, float cl, float zh, float zl, float& S,
                                     float& err) {
  const float p = __fmul_rn(ch, zh);
  const float e = __fmaf_rn(ch, zh, -p);
  const float s = __fadd_rn(S, p);
  const float bb = __fsub_rn(s, S);
  const float te = __fadd_rn(__fsub_rn(S, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  err = __fadd_rn(err, __fadd_rn(e, te));
  err = __fmaf_rn(ch, zl, err);
  err = __fmaf_rn(cl, zh, err);
  S = s;
}

// S += z for a pair z (coefficient one), TwoSum on the high parts
__device__ __forceinline__ void tadd(float zh, float zl, float& S, float& err) {
  const float s = __fadd_rn(S, zh);
  const float bb = __fsub_rn(s, S);
  const float te = __fadd_rn(__fsub_rn(S, __fsub_rn(s, bb)), __fsub_rn(zh, bb));
  err = __fadd_rn(err, __fadd_rn(te, zl));
  S = s;
}

// (sh, sl) = a + b for pairs: TwoSum on the high parts, low parts added in FP32
__device__ __forceinline__ void dfadd(float ah, float al, float bh, float bl, float& sh,
                                      float& sl) {
  const float s = __fadd_rn(ah, bh);
  const float bb = __fsub_rn(s, ah);
  const float te = __fadd_rn(__fsub_rn(ah, __fsub_rn(s, bb)), __fsub_rn(bh, bb));
  sh = s;
  sl = __fadd_rn(te, __fadd_rn(al, bl));
}

// exact product of two floats as a pair, plus low-part cross terms: a * b
__device__ __forceinline__ void dfmul(float ah, float al, float bh, float bl, float& ph,
                                      float& pl) {
  const float p = __fmul_rn(ah, bh);
  float e = __fmaf_rn(ah, bh, -p);
  e = __fmaf_rn(ah, bl, e);
  e = __fmaf_rn(al, bh, e);
  ph = p;
  pl = e;
}

// --------------------------------------------------- extraction dot products
// Error-free extraction against a power-of-two bound (Rump, Ogita and Oishi,
// "Accurate floating-point summation", SIAM J. Sci. Comput. 31, 2008): with
// sigma = 2^k >= sum_l |c_l z_l|, the float q = RN(c z + sigma) - sigma is a
// multiple of 2^-24 sigma, so the running sum S of the q of a dot product is
// exact (every partial sum is such a multiple below sigma in magnitude), and
// r = RN(c z - q) is the product's remainder.  A term costs 7 instructions
// instead of the 12 of the TwoSum form above; the price is that the error term
// E collects remainders of size up to 2^-24 sigma rather than 2^-24 |c z|, so
// its rounding costs one to three bits against the TwoSum form (measured in a
// float32 emulation of both against the FP64 oracle).  The kernel therefore
// uses it only where the bound is tight: the geometric-factor products and the
// transposed contractions, not the first derivatives of u.

// smallest power of two >= b for a finite b >= 0 (0 for b = 0)
__device__ __forceinline__ float df_pow2_ceil(float b) {
  return __uint_as_float((__float_as_uint(b) + 0x007FFFFFu) & 0xFF800000u);
}

// first term: S = q, E = r + cross terms
__device__ __forceinline__ void xmac0(float ch, float cl, float zh, float zl, float sig,
                                      float& S, float& E) {
  const float q = __fsub_rn(__fmaf_rn(ch, zh, sig), sig);
  const float r = __fmaf_rn(ch, zh, -q);
  S = q;
  E = __fmaf_rn(cl, zh, __fmaf_rn(ch, zl, r));
}

// next term: S += q exactly, E += r + cross terms
__device__ __forceinline__ void xmac(float ch, float cl, float zh, float zl, float sig,
                                     float& S, float& E) {
  const float q = __fsub_rn(__fmaf_rn(ch, zh, sig), sig);
  const float r = __fmaf_rn(ch, zh, -q);
  S = __fadd_rn(S, q);
  E = __fmaf_rn(cl, zh, __fmaf_rn(ch, zl, __fadd_rn(E, r)));
}

// ------------------------------------------------------------------ range
// Pair arithmetic keeps its 48 bits only while every intermediate stays in
// FP32's exponent range (normal floats from 2^-126 to 2^128).  The element
// operator is linear, so a kernel may scale u, the geometric factors and the
// coefficients by powers of two (exact in binary arithmetic) and undo the
// scaling on the FP64 result.  Quantities whose magnitude lies in
// [2^-16, 2^16) are used unscaled (exponent 0); the others are normalised to
// [1, 2).  With coefficients so bounded (|c G| < 2^32) an element whose
// largest |u| lies in [2^-60, 2^76) keeps every intermediate between about
// 2^-140 and 2^123: products and sums stay finite, and the FP32 error terms
// (2^-48 of the partial sums, subnormal at worst) stay far below the 1e-12
// relative accuracy.  Other elements are rescaled by their own maximum.

// exponent of a nonnegative magnitude a: 0 inside [2^-16, 2^16) (and for 0
// or a non-finite a), else floor(log2 a)
__host__ __device__ inline int df_pick_exp(double a) {
  if (!(a > 0.0) || !(a <= 1.7976931348623157e308)) return 0;
  if (a >= 0x1p-16 && a < 0x1p16) return 0;
  int e = 0;
  (void)frexp(a, &e);
  return e - 1;
}

// Magnitude key of a double: its high word without the sign, with bit 0 set
// when the low word is nonzero (so that only +-0 has key 0).  Keys order
// like magnitudes up to that bit; a key >= kDfKeyNonFinite is an Inf or NaN.
constexpr unsigned kDfKeyLo = (1023u - 60u) << 20;     // |u| >= 2^-60
constexpr unsigned kDfKeyHi = (1023u + 76u) << 20;     // |u| <  2^76
constexpr unsigned kDfKeyNonFinite = 0x7FF00000u;
// <p, H p> of the fused kernel: p is rescaled only outside [2^-20, 2^20)
constexpr unsigned kDfPwLo = (1023u - 20u) << 20;
constexpr unsigned kDfPwHi = (1023u + 20u) << 20;

// floor(log2) of the magnitude a finite key stands for; elements whose
// largest value is subnormal (key below 2^20) are scaled by 2^1060, which
// maps every subnormal into [2^-14, 2^38)
__device__ __forceinline__ int df_key_exp(unsigned key) {
  const int f = (int)(key >> 20);
  return f ? f - 1023 : -1060;
}

// 2^e as a double, e in [-1022, 1023]
__device__ __forceinline__ double df_pow2d(int e) {
  return __longlong_as_double((long long)(e + 1023) << 52);
}

// v 2^e for |e| up to about 3000, in steps that are exact powers of two
__device__ __forceinline__ double df_ldexp(double v, int e) {
  while (e > 1000) {
    v *= df_pow2d(1000);
    e -= 1000;
  }
  while (e < -1000) {
    v *= df_pow2d(-1000);
    e += 1000;
  }
  return v * df_pow2d(e);
}

// x 2^d for d <= 0 (two steps below FP32's normal range, 0 far below it)
__device__ __forceinline__ float df_scale_down(float x, int d) {
  if (d >= -126) return __fmul_rn(x, __int_as_float((127 + d) << 23));
  if (d >= -252) return __fmul_rn(__fmul_rn(x, 0x1p-126f), __int_as_float((253 + d) << 23));
  return __fmul_rn(x, 0.0f);
}

}  // namespace sem
