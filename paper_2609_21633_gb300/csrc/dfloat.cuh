// Double-float ("double-word") arithmetic: a value is the unevaluated sum hi + lo of two FP32
// numbers with |lo| <= ulp(hi) / 2, about 48 significand bits.  The FP64 pipe of this GPU issues
// two fused multiply-adds per clock per SM against 128 for FP32, so element arithmetic that the
// FP64 pipe bounds runs faster as FP32 pairs at nearly FP64 accuracy.
//
// Building blocks (error-free transformations, round-to-nearest FP32):
//   TwoSum (Knuth 1969, Moller 1965): s + e = a + b exactly, 6 operations;
//   FastTwoSum (Dekker 1971): the same when |a| >= |b| (or a = 0), 3 operations;
//   TwoProd with FMA: p + e = a b exactly, 2 operations.
// Double-word operations from Joldes, Muller, Popescu, "Tight and rigorous error bounds for basic
// building blocks of double-word arithmetic", ACM TOMS 44 (2017):
//   addition "AccurateDWPlusDW" (their Algorithm 6), relative error <= 3u^2 + 13u^3;
//   multiplication "DWTimesDW3" (Algorithm 12, with FMA), relative error <= 4u^2;
// u = 2^-24.  Every operation is written out with the _rn intrinsics so that the compiler neither
// contracts nor reorders it.
//
// Conversions from and to binary64 use integer operations only (no FP64 instruction):
//   split: hi = the double truncated to 24 significand bits, lo = the next 23 bits (exact
//   integer-to-float trick), then FastTwoSum to restore |lo| <= ulp(hi) / 2; relative error
//   below 2^-46 (both parts are truncated).  Magnitudes below 2^-80 keep only hi, and values outside the FP32 exponent range
//   are not representable (the wedge operator's data are far inside both limits).
//   join: hi and lo widened exactly to binary64 (bit manipulation) and added with one FP64 add,
//   which is exact because hi + lo has at most 48 significant bits.
#pragma once

#include <cstdint>
#include <cstring>

namespace tn {

#if defined(__CUDA_ARCH__)
#define TN_DF_HD __device__ __forceinline__
#define TN_FADD(a, b) __fadd_rn(a, b)
#define TN_FSUB(a, b) __fsub_rn(a, b)
#define TN_FMUL(a, b) __fmul_rn(a, b)
#define TN_FFMA(a, b, c) __fmaf_rn(a, b, c)
#else
#define TN_DF_HD inline
#define TN_FADD(a, b) ((float)((a) + (b)))
#define TN_FSUB(a, b) ((float)((a) - (b)))
#define TN_FMUL(a, b) ((float)((a) * (b)))
#define TN_FFMA(a, b, c) std::fma((float)(a), (float)(b), (float)(c))
#endif

TN_DF_HD void two_sum(float a, float b, float& s, float& e) {
  s = TN_FADD(a, b);
  const float bb = TN_FSUB(s, a);
  e = TN_FADD(TN_FSUB(a, TN_FSUB(s, bb)), TN_FSUB(b, bb));
}
TN_DF_HD void fast_two_sum(float a, float b, float& s, float& e) {
  s = TN_FADD(a, b);
  e = TN_FSUB(b, TN_FSUB(s, a));
}

struct dfl {
  float hi, lo;
  dfl() = default;
  TN_DF_HD constexpr dfl(float h, float l) : hi(h), lo(l) {}
  // from a double known at compile time (constants of the element ops); folded by the compiler
  TN_DF_HD constexpr dfl(double x) : hi((float)x), lo((float)(x - (double)(float)x)) {}
};

TN_DF_HD dfl operator-(dfl a) { return dfl(-a.hi, -a.lo); }

// AccurateDWPlusDW
TN_DF_HD dfl operator+(dfl x, dfl y) {
  float sh, sl, th, tl, vh, vl, zh, zl;
  two_sum(x.hi, y.hi, sh, sl);
  two_sum(x.lo, y.lo, th, tl);
  const float c = TN_FADD(sl, th);
  fast_two_sum(sh, c, vh, vl);
  const float w = TN_FADD(tl, vl);
  fast_two_sum(vh, w, zh, zl);
  return dfl(zh, zl);
}
TN_DF_HD dfl operator-(dfl x, dfl y) { return x + (-y); }

// DWTimesDW3
TN_DF_HD dfl operator*(dfl x, dfl y) {
  const float ch = TN_FMUL(x.hi, y.hi);
  const float cl1 = TN_FFMA(x.hi, y.hi, -ch);
  const float tl0 = TN_FMUL(x.lo, y.lo);
  const float tl1 = TN_FFMA(x.hi, y.lo, tl0);
  const float cl2 = TN_FFMA(x.lo, y.hi, tl1);
  const float cl3 = TN_FADD(cl1, cl2);
  float zh, zl;
  fast_two_sum(ch, cl3, zh, zl);
  return dfl(zh, zl);
}

// Sum without the second TwoSum (the "sloppy" double-word addition): absolute error about
// 2u^2 (|x| + |y|), so it is kept for sums whose terms do not cancel; 11 operations.
TN_DF_HD dfl add_nc(dfl x, dfl y) {
  float sh, sl, zh, zl;
  two_sum(x.hi, y.hi, sh, sl);
  const float w = TN_FADD(sl, TN_FADD(x.lo, y.lo));
  fast_two_sum(sh, w, zh, zl);
  return dfl(zh, zl);
}
// x y + w in one pass: the exact product of the high parts (TwoProd), the cross terms by FMA,
// then the sloppy addition of w; absolute error about 3u^2 (|x y| + |w|), for the same use;
// 15 operations against 20 for a multiplication followed by an addition.
TN_DF_HD dfl fma_nc(dfl x, dfl y, dfl w) {
  const float ph = TN_FMUL(x.hi, y.hi);
  float pl = TN_FFMA(x.hi, y.hi, -ph);
  pl = TN_FFMA(x.hi, y.lo, pl);
  pl = TN_FFMA(x.lo, y.hi, pl);
  float sh, sl, zh, zl;
  two_sum(ph, w.hi, sh, sl);
  const float t = TN_FADD(sl, TN_FADD(pl, w.lo));
  fast_two_sum(sh, t, zh, zl);
  return dfl(zh, zl);
}

TN_DF_HD dfl& operator+=(dfl& a, dfl b) { return a = a + b; }
TN_DF_HD dfl& operator-=(dfl& a, dfl b) { return a = a - b; }

TN_DF_HD uint64_t df_bits_of(double x) {
#if defined(__CUDA_ARCH__)
  return (uint64_t)__double_as_longlong(x);
#else
  uint64_t b;
  std::memcpy(&b, &x, 8);
  return b;
#endif
}
TN_DF_HD double df_double_of(uint64_t b) {
#if defined(__CUDA_ARCH__)
  return __longlong_as_double((long long)b);
#else
  double x;
  std::memcpy(&x, &b, 8);
  return x;
#endif
}
TN_DF_HD float df_float_of(uint32_t b) {
#if defined(__CUDA_ARCH__)
  return __uint_as_float(b);
#else
  float x;
  std::memcpy(&x, &b, 4);
  return x;
#endif
}
TN_DF_HD uint32_t df_ubits_of(float x) {
#if defined(__CUDA_ARCH__)
  return __float_as_uint(x);
#else
  uint32_t b;
  std::memcpy(&b, &x, 4);
  return b;
#endif
}

// binary64 -> double-float with integer operations (see the file comment)
TN_DF_HD dfl split(double x) {
  const uint64_t b = df_bits_of(x);
  const uint32_t bh = (uint32_t)(b >> 32), bl = (uint32_t)b;
  const uint32_t sign = bh & 0x80000000u;
  const int e = (int)((bh >> 20) & 0x7ffu);         // biased binary64 exponent
  if (e < 1023 - 126) return dfl(df_float_of(sign), 0.0f);  // zero or below the FP32 normal range
  const uint32_t m23 = ((bh & 0xfffffu) << 3) | (bl >> 29);  // top 23 stored significand bits
  const float hi = df_float_of(sign | ((uint32_t)(e - 1023 + 127) << 23) | m23);
  // the next 23 bits as an exact integer t (2^23 + t - 2^23), scaled by 2^(e - 1023 - 46)
  const float t = TN_FSUB(df_float_of(0x4b000000u | ((bl >> 6) & 0x7fffffu)), 8388608.0f);
  const int se = e - 1023 - 46 + 127;
  const float lo_mag = se >= 1 ? TN_FMUL(t, df_float_of((uint32_t)se << 23)) : 0.0f;
  const float lo = df_float_of(df_ubits_of(lo_mag) | sign);
  float zh, zl;
  fast_two_sum(hi, lo, zh, zl);
  return dfl(zh, zl);
}

// exact FP32 -> binary64 widening by bit manipulation (FP32 subnormals become 0)
TN_DF_HD double widen(float f) {
  const uint32_t u = df_ubits_of(f);
  const uint32_t e = (u >> 23) & 0xffu;
  if (e == 0) return df_double_of((uint64_t)(u & 0x80000000u) << 32);
  const uint64_t bits = ((uint64_t)(u & 0x80000000u) << 32) | ((uint64_t)(e + 1023 - 127) << 52) |
                        ((uint64_t)(u & 0x7fffffu) << 29);
  return df_double_of(bits);
}

// double-float -> binary64: one exact FP64 addition
TN_DF_HD double join(dfl a) { return widen(a.hi) + widen(a.lo); }

#if defined(__CUDACC__)
// Packed double-float: two independent values in the lanes of f32x2 registers (hi.x + lo.x,
// hi.y + lo.y), every operation the scalar one lane-wise with the packed FP32 instructions (one
// issue slot per pair).  Lanes never mix inside an operation and every packed instruction rounds
// each lane to nearest, so a lane follows the scalar formula step for step.  A kernel written with
// df2 may still group its sums differently from its scalar version: the two then agree to the
// double-float rounding level (about 2^-46 relative), not bitwise.
struct df2 {
  float2 hi, lo;
};
__device__ __forceinline__ float2 p2add(float2 a, float2 b) { return __fadd2_rn(a, b); }
// a - b lane-wise, rounded to nearest: the packed subtraction of PTX (no intrinsic exists)
__device__ __forceinline__ float2 p2sub(float2 a, float2 b) {
  unsigned long long ra, rb, rd;
  asm("mov.b64 %0, {%1, %2};" : "=l"(ra) : "f"(a.x), "f"(a.y));
  asm("mov.b64 %0, {%1, %2};" : "=l"(rb) : "f"(b.x), "f"(b.y));
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(rd) : "l"(ra), "l"(rb));
  float2 d;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(d.x), "=f"(d.y) : "l"(rd));
  return d;
}
__device__ __forceinline__ float2 p2mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 p2fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 p2neg(float2 a) { return make_float2(-a.x, -a.y); }

__device__ __forceinline__ df2 pack(dfl a, dfl b) { return df2{make_float2(a.hi, b.hi), make_float2(a.lo, b.lo)}; }
__device__ __forceinline__ dfl lane_x(const df2& a) { return dfl(a.hi.x, a.lo.x); }
__device__ __forceinline__ dfl lane_y(const df2& a) { return dfl(a.hi.y, a.lo.y); }

__device__ __forceinline__ void two_sum2(float2 a, float2 b, float2& s, float2& e) {
  s = p2add(a, b);
  const float2 bb = p2sub(s, a);
  e = p2add(p2sub(a, p2sub(s, bb)), p2sub(b, bb));
}
__device__ __forceinline__ void fast_two_sum2(float2 a, float2 b, float2& s, float2& e) {
  s = p2add(a, b);
  e = p2sub(b, p2sub(s, a));
}
// AccurateDWPlusDW, lane-wise
__device__ __forceinline__ df2 add2(const df2& x, const df2& y) {
  float2 sh, sl, th, tl, vh, vl, zh, zl;
  two_sum2(x.hi, y.hi, sh, sl);
  two_sum2(x.lo, y.lo, th, tl);
  fast_two_sum2(sh, p2add(sl, th), vh, vl);
  fast_two_sum2(vh, p2add(tl, vl), zh, zl);
  return df2{zh, zl};
}
__device__ __forceinline__ df2 sub2(const df2& x, const df2& y) { return add2(x, df2{p2neg(y.hi), p2neg(y.lo)}); }
// DWTimesDW3, lane-wise
__device__ __forceinline__ df2 mul2(const df2& x, const df2& y) {
  const float2 ch = p2mul(x.hi, y.hi);
  const float2 cl1 = p2fma(x.hi, y.hi, p2neg(ch));
  const float2 tl1 = p2fma(x.hi, y.lo, p2mul(x.lo, y.lo));
  const float2 cl2 = p2fma(x.lo, y.hi, tl1);
  float2 zh, zl;
  fast_two_sum2(ch, p2add(cl1, cl2), zh, zl);
  return df2{zh, zl};
}
// add_nc / fma_nc, lane-wise
__device__ __forceinline__ df2 add_nc2(const df2& x, const df2& y) {
  float2 sh, sl, zh, zl;
  two_sum2(x.hi, y.hi, sh, sl);
  fast_two_sum2(sh, p2add(sl, p2add(x.lo, y.lo)), zh, zl);
  return df2{zh, zl};
}
__device__ __forceinline__ df2 fma_nc2(const df2& x, const df2& y, const df2& w) {
  const float2 ph = p2mul(x.hi, y.hi);
  float2 pl = p2fma(x.hi, y.hi, p2neg(ph));
  pl = p2fma(x.hi, y.lo, pl);
  pl = p2fma(x.lo, y.hi, pl);
  float2 sh, sl, zh, zl;
  two_sum2(ph, w.hi, sh, sl);
  fast_two_sum2(sh, p2add(sl, p2add(pl, w.lo)), zh, zl);
  return df2{zh, zl};
}
#endif

}  // namespace tn
