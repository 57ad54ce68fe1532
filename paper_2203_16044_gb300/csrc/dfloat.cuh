// Double-float arithmetic for the complex128 path.
//
// GB300 executes FP64 FMAs at about 1/64 of the FP32 rate (measured: 1.0 vs
// 74 TFLOP/s), so a complex128 gate computed with native FP64 is bound by
// the FP64 pipe at about a third of HBM bandwidth.  Here a double value is
// carried as an unevaluated sum h + l of two floats (47-48 significant
// bits), products and sums use the error-free transformations
//   TwoSum  (Knuth, TAOCP vol. 2, 4.2.2):  s + e = a + b exactly
//   TwoProd (FMA form):                    p + e = a * b exactly
// and the state stays in the standard FP64 layout in memory: the
// conversions double <-> (h, l) below use integer bit operations only, so
// no FP64 instruction is issued on the hot path.
//
// Accuracy: a split keeps the top 47 significand bits of the double
// (relative error < 2^-46); each 4-term dot product is accurate to about
// 2^-46 of the sum of the term magnitudes.  Values below about 2^-75 in
// magnitude (irrelevant for normalised states at the 1e-12 absolute
// tolerance of the complex128 path) are carried with float precision only,
// and values below 2^-126 flush to zero.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

namespace qs {

struct dfl {
  float h, l;
};

// Knuth's TwoSum (6 flops, no ordering requirement).
__device__ __forceinline__ float two_sum(float a, float b, float& e) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return s;
}

// Dekker's FastTwoSum (exact when |a| >= |b|; otherwise the error term is
// approximate, which costs at most 2^-24 of |b|).
__device__ __forceinline__ float fast_two_sum(float a, float b, float& e) {
  const float s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
  return s;
}

// double -> (h, l), integer operations only.  h takes the sign, exponent and
// the top 23 fraction bits (truncated); l the next 23 fraction bits, scaled.
__device__ __forceinline__ dfl d2df(double d) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
  const unsigned sign = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7ffu);
  const int ef = e - 896;  // float biased exponent of h
  dfl r;
  const unsigned frac23 = ((hi & 0xfffffu) << 3) | (lo >> 29);
  r.h = ef > 0 ? __uint_as_float(sign | ((unsigned)ef << 23) | frac23) : 0.0f;
  // remaining bits 28..6 of the fraction: k * 2^(e - 1069), k < 2^23
  const unsigned k = (lo >> 6) & 0x7fffffu;
  const int es = e - 942;  // biased exponent of 2^(e - 1069)
  const float scale = es > 0 ? __uint_as_float(sign | ((unsigned)es << 23)) : 0.0f;
  const float m = __uint_as_float(0x4B000000u | k);  // 2^23 + k, exactly
  r.l = __fmaf_rn(m, scale, __fmul_rn(-8388608.0f, scale));  // k * scale, exact
  return r;
}

// (h, l) -> double, integer operations only.  Requires |l| <= ulp(h) (true
// for results of the arithmetic below and for d2df splits).
__device__ __forceinline__ double df2d(dfl v) {
  const unsigned hb = __float_as_uint(v.h), lb = __float_as_uint(v.l);
  const unsigned eh = (hb >> 23) & 0xffu, fh = hb & 0x7fffffu;
  if (eh == 0) return 0.0;
  unsigned long long D = ((unsigned long long)(hb & 0x80000000u) << 32) |
                         ((unsigned long long)(eh + 896u) << 52) | ((unsigned long long)fh << 29);
  const unsigned el = (lb >> 23) & 0xffu;
  if (eh < 52u || el == 0) return __longlong_as_double((long long)D);
  // |l| = (2^23 + fl) 2^(el - 150); in units of the double ulp of h,
  // 2^(eh - 179), that is (2^23 + fl) 2^sh with sh = el - eh + 29 <= 6.
  const unsigned ml = 0x800000u | (lb & 0x7fffffu);
  const int sh = (int)el - (int)eh + 29;
  unsigned long long k;
  if (sh >= 0) k = (unsigned long long)ml << sh;
  else if (sh > -24) k = (unsigned long long)(ml >> (-sh));
  else k = 0ull;
  if ((hb ^ lb) & 0x80000000u) {
    // l opposite to h: step down; below a power of two the ulp halves
    D -= (fh == 0u) ? (k << 1) : k;
  } else {
    D += k;
  }
  return __longlong_as_double((long long)D);
}

// acc += v in double-float, low part left unnormalised: it gathers the
// exact rounding errors of the high part (TwoSum) and v's low part.
__device__ __forceinline__ void df_acc(dfl& acc, dfl v) {
  float e;
  acc.h = two_sum(acc.h, v.h, e);
  acc.l = __fadd_rn(acc.l, __fadd_rn(e, v.l));
}

// a + b in double-float, normalised
__device__ __forceinline__ dfl df_add(dfl a, dfl b) {
  float e;
  const float s = two_sum(a.h, b.h, e);
  dfl r;
  r.h = fast_two_sum(s, __fadd_rn(e, __fadd_rn(a.l, b.l)), r.l);
  return r;
}

// a b in double-float (the l*l term, ~2^-48 relative, dropped), unnormalised:
// h = a.h b.h rounded, l = its exact error plus the cross terms
__device__ __forceinline__ dfl df_mul(dfl a, dfl b) {
  dfl r;
  r.h = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -r.h);
  e = __fmaf_rn(a.h, b.l, e);
  r.l = __fmaf_rn(a.l, b.h, e);
  return r;
}

// sum_{k<4} x_k y_k for double-float x_k, y_k; h + l normalised.
__device__ __forceinline__ dfl dot4(float xh0, float xl0, float yh0, float yl0, float xh1, float xl1, float yh1,
                                    float yl1, float xh2, float xl2, float yh2, float yl2, float xh3, float xl3,
                                    float yh3, float yl3) {
  float p = __fmul_rn(xh0, yh0);
  float c = __fmaf_rn(xh0, yh0, -p);
  c = __fmaf_rn(xh0, yl0, c);
  c = __fmaf_rn(xl0, yh0, c);
  float t, q, e;
#define QS_DOT_TERM(XH, XL, YH, YL)       \
  q = __fmul_rn(XH, YH);                  \
  e = __fmaf_rn(XH, YH, -q);              \
  e = __fmaf_rn(XH, YL, e);               \
  e = __fmaf_rn(XL, YH, e);               \
  p = two_sum(p, q, t);                   \
  c = __fadd_rn(c, __fadd_rn(t, e));
  QS_DOT_TERM(xh1, xl1, yh1, yl1)
  QS_DOT_TERM(xh2, xl2, yh2, yl2)
  QS_DOT_TERM(xh3, xl3, yh3, yl3)
#undef QS_DOT_TERM
  dfl r;
  r.h = fast_two_sum(p, c, r.l);
  return r;
}

// sum_{k<2} x_k y_k (complex scalar multiply components).
__device__ __forceinline__ dfl dot2(float xh0, float xl0, float yh0, float yl0, float xh1, float xl1, float yh1,
                                    float yl1) {
  float p = __fmul_rn(xh0, yh0);
  float c = __fmaf_rn(xh0, yh0, -p);
  c = __fmaf_rn(xh0, yl0, c);
  c = __fmaf_rn(xl0, yh0, c);
  const float q = __fmul_rn(xh1, yh1);
  float e = __fmaf_rn(xh1, yh1, -q);
  e = __fmaf_rn(xh1, yl1, e);
  e = __fmaf_rn(xl1, yh1, e);
  float t;
  p = two_sum(p, q, t);
  c = __fadd_rn(c, __fadd_rn(t, e));
  dfl r;
  r.h = fast_two_sum(p, c, r.l);
  return r;
}

// Complex double-float amplitude.
struct cdf {
  float rh, rl, ih, il;
};

// Complex 2x2 matrix in double-float: entries (re, im) row-major, hi and lo.
struct M2df {
  float h[8], l[8];
};

// (a, b) <- U (a, b)
__device__ __forceinline__ void mv2df(const M2df& U, cdf& a, cdf& b) {
  // y0 = u00 a + u01 b ; y1 = u10 a + u11 b
  const dfl y0r = dot4(U.h[0], U.l[0], a.rh, a.rl, -U.h[1], -U.l[1], a.ih, a.il, U.h[2], U.l[2], b.rh, b.rl,
                       -U.h[3], -U.l[3], b.ih, b.il);
  const dfl y0i = dot4(U.h[0], U.l[0], a.ih, a.il, U.h[1], U.l[1], a.rh, a.rl, U.h[2], U.l[2], b.ih, b.il,
                       U.h[3], U.l[3], b.rh, b.rl);
  const dfl y1r = dot4(U.h[4], U.l[4], a.rh, a.rl, -U.h[5], -U.l[5], a.ih, a.il, U.h[6], U.l[6], b.rh, b.rl,
                       -U.h[7], -U.l[7], b.ih, b.il);
  const dfl y1i = dot4(U.h[4], U.l[4], a.ih, a.il, U.h[5], U.l[5], a.rh, a.rl, U.h[6], U.l[6], b.ih, b.il,
                       U.h[7], U.l[7], b.rh, b.rl);
  a.rh = y0r.h; a.rl = y0r.l; a.ih = y0i.h; a.il = y0i.l;
  b.rh = y1r.h; b.rl = y1r.l; b.ih = y1i.h; b.il = y1i.l;
}

// a <- z a for a double-float complex scalar z = (zh[0] + zl[0]) + i (zh[1] + zl[1])
__device__ __forceinline__ void cmul_df(const float* zh, const float* zl, cdf& a) {
  const dfl r = dot2(zh[0], zl[0], a.rh, a.rl, -zh[1], -zl[1], a.ih, a.il);
  const dfl i = dot2(zh[0], zl[0], a.ih, a.il, zh[1], zl[1], a.rh, a.rl);
  a.rh = r.h; a.rl = r.l; a.ih = i.h; a.il = i.l;
}

// A value as double-float: a float exactly, a double by its (h, l) split.
__device__ __forceinline__ dfl to_df(float x) { return dfl{x, 0.f}; }
__device__ __forceinline__ dfl to_df(double x) { return d2df(x); }
// A double-float partial sum into an FP64 accumulator (two FP64 additions),
// then reset.
__device__ __forceinline__ void df_flush(double& acc, dfl& v) {
  acc += (double)v.h;
  acc += (double)v.l;
  v = dfl{0.f, 0.f};
}

}  // namespace qs
