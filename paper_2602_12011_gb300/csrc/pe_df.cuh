// pe_df.cuh -- double-word ("double-float") arithmetic on the FP32 pipe: a value is the unevaluated
// sum hi + lo of two floats with |lo| <= ulp(hi)/2, about 48 significant bits (relative error of the
// operations below ~1e-14). Error-free transformations: TwoSum (Knuth, TAOCP 4.2.2), Fast2Sum
// (Dekker 1971), TwoProd by FMA; double-word addition and multiplication after Joldes, Muller and
// Popescu, "Tight and rigorous error bounds for basic building blocks of double-word arithmetic"
// (ACM TOMS 2017), Algorithms 6 (accurate DW + DW) and 12 (DW x DW with FMA). Every float operation
// of the transformations is an explicitly rounded intrinsic, so the compiler cannot contract them.
#pragma once
#include <cuda_runtime.h>

#include "pe_internal.h"

namespace pe {

using df = float2;  // (hi, lo)

__device__ __forceinline__ df df_make(float h, float l) { return make_float2(h, l); }

// s + e = a + b exactly
__device__ __forceinline__ df two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float v = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, v)), __fsub_rn(b, v));
  return df_make(s, e);
}
// s + e = a + b exactly when |a| >= |b| (or a == 0)
__device__ __forceinline__ df fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float e = __fsub_rn(b, __fsub_rn(s, a));
  return df_make(s, e);
}

// accurate DW + DW (Alg. 6): relative error <= 3 u^2 + 13 u^3
__device__ __forceinline__ df df_add(df x, df y) {
  const df s = two_sum(x.x, y.x);
  const df t = two_sum(x.y, y.y);
  const float c = __fadd_rn(s.y, t.x);
  const df v = fast_two_sum(s.x, c);
  const float w = __fadd_rn(t.y, v.y);
  return fast_two_sum(v.x, w);
}
// "sloppy" DW + DW (the same paper's Alg. 5): only x.lo + y.lo and the carry are rounded, so the
// absolute error stays below ~2 u^2 (|x| + |y|). Its relative error is unbounded under
// cancellation, but there the operands' own rounding errors (~u^2 of their size) are as large; it
// is the add of the hot loops, where every operand is itself a rounded result.
__device__ __forceinline__ df df_add_s(df x, df y) {
  const df s = two_sum(x.x, y.x);
  const float v = __fadd_rn(x.y, y.y);
  const float w = __fadd_rn(s.y, v);
  return fast_two_sum(s.x, w);
}
__device__ __forceinline__ df df_sub_s(df x, df y) { return df_add_s(x, make_float2(-y.x, -y.y)); }
__device__ __forceinline__ df df_neg(df x) { return df_make(-x.x, -x.y); }
__device__ __forceinline__ df df_sub(df x, df y) { return df_add(x, df_neg(y)); }

// DW x DW with FMA (Alg. 12): relative error <= 4 u^2
__device__ __forceinline__ df df_mul(df x, df y) {
  const float ch = __fmul_rn(x.x, y.x);
  const float cl1 = __fmaf_rn(x.x, y.x, -ch);
  const float tl0 = __fmul_rn(x.y, y.y);
  const float tl1 = __fmaf_rn(x.x, y.y, tl0);
  const float cl2 = __fmaf_rn(x.y, y.x, tl1);
  const float cl3 = __fadd_rn(cl1, cl2);
  return fast_two_sum(ch, cl3);
}
// DW x float
__device__ __forceinline__ df df_mulf(df x, float y) {
  const float ch = __fmul_rn(x.x, y);
  const float cl1 = __fmaf_rn(x.x, y, -ch);
  const float cl3 = __fmaf_rn(x.y, y, cl1);
  return fast_two_sum(ch, cl3);
}
// multiplication by a power of two is exact
__device__ __forceinline__ df df_scale2(df x, float p2) { return df_make(x.x * p2, x.y * p2); }

__device__ __forceinline__ df df_from(double a) {
  const float h = __double2float_rn(a);
  return df_make(h, __double2float_rn(a - (double)h));
}
__device__ __forceinline__ double df_to(df a) { return (double)a.x + (double)a.y; }

// double -> float by truncation to 24 significant bits on the integer pipe (GB300 runs the F2F
// conversions on its narrow FP64 pipe). Magnitudes below 2^-126, and zero, give 0; the values
// converted here stay far below the float overflow.
__device__ __forceinline__ float trunc_to_float(unsigned long long u) {
  const unsigned hi32 = (unsigned)(u >> 32), lo32 = (unsigned)u;
  const int e = (int)((hi32 >> 20) & 0x7FFu);
  if (e < 897) return 0.0f;
  return __uint_as_float((hi32 & 0x80000000u) | ((unsigned)(e - 896) << 23) | ((hi32 & 0xFFFFFu) << 3) | (lo32 >> 29));
}
// double -> double word by truncation: hi = the top 24 significant bits of a (exactly a float), lo =
// the top 24 of the exact remainder a - hi. |a - (hi + lo)| < 2^-46 |a|; one FP64 subtraction.
__device__ __forceinline__ df df_from_bits(double a) {
  const unsigned long long u = __double_as_longlong(a);
  const float h = trunc_to_float(u);
  const double hd = (h == 0.0f) ? 0.0 : __longlong_as_double((long long)(u & 0xFFFFFFFFE0000000ull));
  return df_make(h, trunc_to_float(__double_as_longlong(a - hd)));
}

// a + b + c of three double words (normalised or lazy) as a normalised double word whose error is
// set by the sum itself, not by the operands: the three high words and the three low words are
// each summed exactly by TwoSum cascades, the high words' residuals join the low words' sum
// exactly, and only the last, tiny residuals are rounded (below 2^-72 of the operands). For sums
// that cancel far below their operands, such as the TDI T channel X' + Y' + Z' at long wavelength.
__device__ __forceinline__ df df_sum3_exact(df a, df b, df c) {
  const df s1 = two_sum(a.x, b.x);
  const df s2 = two_sum(s1.x, c.x);          // a.hi + b.hi + c.hi = s2.x + s1.y + s2.y
  const df t1 = two_sum(a.y, b.y);
  const df t2 = two_sum(t1.x, c.y);          // a.lo + b.lo + c.lo = t2.x + t1.y + t2.y
  const df t3 = two_sum(t2.x, s1.y);
  const df t4 = two_sum(t3.x, s2.y);         // sum = s2.x + t4.x + (t1.y + t2.y + t3.y + t4.y)
  const float r = __fadd_rn(__fadd_rn(t1.y, t2.y), __fadd_rn(t3.y, t4.y));
  const df u = two_sum(s2.x, t4.x);
  return two_sum(u.x, __fadd_rn(u.y, r));
}


// Unnormalised ("lazy") variants for the long chains of the mixed-precision units. dfl_add is
// df_add_s without its closing Fast2Sum: the same rounded quantities, so the same absolute error
// (~2 u^2 (|x| + |y|)), but |lo| may exceed ulp(hi)/2 by a few ulps. dfl_mul is Alg. 12 without
// the lo x lo product (below u^2 |x y|) and without the closing Fast2Sum. Pairs from them are
// fine operands for every operation here; df_cis_turns renormalises its argument, the one place
// that needs |lo| <= ulp(hi)/2.
__device__ __forceinline__ df dfl_add(df x, df y) {
  const df s = two_sum(x.x, y.x);
  return df_make(s.x, __fadd_rn(s.y, __fadd_rn(x.y, y.y)));
}
__device__ __forceinline__ df dfl_sub(df x, df y) { return dfl_add(x, make_float2(-y.x, -y.y)); }
// dfl_add for operands ordered by size, |x.hi| >= |y.hi| (or x.hi = 0): under that ordering Fast2Sum
// returns the same rounded sum and the same exact error as TwoSum, in three additions instead of
// six, so the result is dfl_add's bit for bit. For the Taylor and Horner steps and the Newton
// corrections, where the ordering follows from the magnitudes of the terms.
__device__ __forceinline__ df dfl_add_o(df x, df y) {
  const df s = fast_two_sum(x.x, y.x);
  return df_make(s.x, __fadd_rn(s.y, __fadd_rn(x.y, y.y)));
}
__device__ __forceinline__ df dfl_mul(df x, df y) {
  const float ch = __fmul_rn(x.x, y.x);
  const float cl1 = __fmaf_rn(x.x, y.x, -ch);
  const float cl2 = __fmaf_rn(x.y, y.x, __fmul_rn(x.x, y.y));
  return df_make(ch, __fadd_rn(cl1, cl2));
}
__device__ __forceinline__ df dfl_mulf(df x, float y) {
  const float ch = __fmul_rn(x.x, y);
  return df_make(ch, __fmaf_rn(x.y, y, __fmaf_rn(x.x, y, -ch)));
}
// 1/x: correctly rounded float seed, one Newton step in DW: y = y0 + y0 (1 - x y0) (error delta^2).
// The step runs on the unnormalised operations: 1 - x y0 is exact in its high word (Sterbenz) and
// only ~u in size, so the lazy pairs lose nothing that the step keeps.
__device__ __forceinline__ df df_rcp(df x) {
  const float y0 = __frcp_rn(x.x);
  const df e = dfl_sub(df_make(1.f, 0.f), dfl_mulf(x, y0));
  return dfl_add_o(df_make(y0, 0.f), dfl_mulf(e, y0));
}
// 1/sqrt(x), x > 0: correctly rounded float seed, one Newton step in DW: y = y0 + y0 (1 - x y0^2)/2
// (relative error (3/2) delta^2 for a seed error delta <= u, plus the DW rounding); unnormalised
// operations as df_rcp.
__device__ __forceinline__ df df_rsqrt(df x) {
  const float y0 = __frsqrt_rn(x.x);
  const df xy2 = dfl_mulf(dfl_mulf(x, y0), y0);
  const df e = dfl_sub(df_make(1.f, 0.f), xy2);
  return dfl_add_o(df_make(y0, 0.f), dfl_mulf(df_scale2(e, 0.5f), y0));
}

// complex DW numbers as pairs (re, im)
struct cdf {
  df re, im;
};
__device__ __forceinline__ cdf cdf_mul(const cdf& a, const cdf& b) {
  cdf r;
  r.re = df_sub(df_mul(a.re, b.re), df_mul(a.im, b.im));
  r.im = df_add(df_mul(a.re, b.im), df_mul(a.im, b.re));
  return r;
}
__device__ __forceinline__ cdf cdfl_mul(const cdf& a, const cdf& b) {
  return cdf{dfl_sub(dfl_mul(a.re, b.re), dfl_mul(a.im, b.im)), dfl_add(dfl_mul(a.re, b.im), dfl_mul(a.im, b.re))};
}

// e^{2 pi i x} = (cos, sin)(2 pi x) for x in turns (|x| < 2^20). The reduction is exact: x.hi - rint(x.hi) and
// the step to the nearest table angle 2 pi j/kSinTab are Sterbenz subtractions, and the low word
// joins by Fast2Sum (the reduced high word is a multiple of ulp(x.hi) or zero). The remainder
// t = 2 pi d (|t| <= pi/kSinTab) goes through sin t = t + t t^2 (-1/6 + t^2/120) and
// cos t = 1 + t^2 (-1/2 + t^2/24); the t^2/120 and t^2/24 corrections enter the low words of the
// double-word coefficients (their rounding is below 1e-18 of the result, the dropped t^7 and t^6
// terms below 2e-18). The Taylor sums and the rotation by the table entry use the unnormalised
// operations below (dfl_*: the same rounding error bounds, the result's |lo| possibly a few ulps
// above ulp(hi)/2, as every lazy result). tab[j] = (cos hi, cos lo, sin hi, sin lo) of 2 pi j/kSinTab. Not inlined: the
// mixed unit calls it from five places, and one copy keeps the kernel's hot loop in the
// instruction cache.
static __device__ __noinline__ cdf df_cis_turns(df x, const float4* __restrict__ tab) {
  x = fast_two_sum(x.x, x.y);   // |lo| <= ulp(hi)/2 for the exact reduction below
  // round to nearest integer by adding and subtracting 1.5 * 2^23 (exact for |v| < 2^22), on the
  // FP32 pipe; the table index is read from the biased sum's bits
  const float kR = 12582912.0f;
  const float rh = __fsub_rn(x.x, __fsub_rn(__fadd_rn(x.x, kR), kR));
  const float y = __fmul_rn(rh, (float)kSinTab);
  const float yb = __fadd_rn(y, kR);
  const int j = __float_as_int(yb) - __float_as_int(kR);
  const df d = fast_two_sum(__fsub_rn(rh, __fmul_rn(__fsub_rn(yb, kR), 1.0f / kSinTab)), x.y);
  const float4 e = tab[j & (kSinTab - 1)];
  const df cj = df_make(e.x, e.y), sj = df_make(e.z, e.w);
  const df t = dfl_mul(d, df_make(6.28318548202514648f, -1.74845553e-07f));   // 2 pi as a double word
  const df t2 = dfl_mul(t, t);
  // -1/6 = -0.166666672 + 4.96705388e-09 and -1/2, with the next Taylor terms folded into the lows
  const df ps = df_make(-0.166666672f, __fmaf_rn(t2.x, 1.0f / 120.0f, 4.96705388e-09f));
  const df pc = df_make(-0.5f, __fmul_rn(t2.x, 1.0f / 24.0f));
  const df st = dfl_add_o(t, dfl_mul(t, dfl_mul(t2, ps)));   // |t^3/6| < |t|
  const df ct = dfl_add_o(df_make(1.f, 0.f), dfl_mul(t2, pc));  // |t^2/2| < 1
  cdf r;
  r.re = dfl_sub(dfl_mul(cj, ct), dfl_mul(sj, st));
  r.im = dfl_add(dfl_mul(sj, ct), dfl_mul(cj, st));
  return r;
}

}  // namespace pe
