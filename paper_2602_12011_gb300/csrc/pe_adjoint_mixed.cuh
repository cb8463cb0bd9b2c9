// pe_adjoint_mixed.cuh -- double-word building blocks of the mixed-precision reverse sweep (row G1
// of the gradient, arXiv:2602.12011 Sec. 2.3 on automatic differentiation; pe_df.cuh arithmetic,
// ~1e-14 relative): complex products with a conjugate, and the sincs' derivatives on the
// polynomial and small-argument branches. The sweep itself is mode_bwd_tape_mixed
// (pe_adjoint_tape_mixed.cuh).
#pragma once
#include "pe_adjoint.cuh"
#include "pe_device_mixed.cuh"

namespace pe {

__device__ __forceinline__ cdf cdf_add_s(const cdf& a, const cdf& b) {
  return cdf{dfl_add(a.re, b.re), dfl_add(a.im, b.im)};
}
// a * conj(b). Not inlined (six calls per link), like df_sinc_poly_d (two): the sweep's link loop
// is long, and one copy of each keeps more of it in the instruction cache.
static __device__ __noinline__ cdf cdf_mul_conj(const cdf& a, const cdf& b) {
  return cdf{dfl_add(dfl_mul(a.re, b.re), dfl_mul(a.im, b.im)), dfl_sub(dfl_mul(a.im, b.re), dfl_mul(a.re, b.im))};
}
__device__ __forceinline__ cdf cdf_mul_s(const cdf& a, const cdf& b) {
  return cdf{dfl_sub(dfl_mul(a.re, b.re), dfl_mul(a.im, b.im)), dfl_add(dfl_mul(a.re, b.im), dfl_mul(a.im, b.re))};
}

// sinc(u) and d sinc/du for |u| <= 1 in double words. With x = u^2: sinc = 1 + x P(x) (the series of
// df_sinc_poly) and d sinc/du = 2 u Q(x), Q(x) = sum_k k c_k x^(k-1), c_k = (-1)^k / (2k+1)!:
// Q = c1 + x (2 c2 + x (3 c3 + x (4 c4 + x T))), T = 5 c5 + x (6 c6 + x (7 c7 + x 8 c8)) in float
// (|T| < 1.3e-7); the first dropped term, 9 c9 x^8, is below 7.5e-17. As in df_sinc_poly, each
// Horner step adds a term smaller than its constant (ordered adds).
struct df2 {
  df v, d;
};
static __device__ __noinline__ df2 df_sinc_poly_d(df u) {
  df2 r;
  r.v = df_sinc_poly(u);
  const df x = dfl_mul(u, u);
  float T = __fmaf_rn(x.x, 2.2491659e-14f, -5.3530145e-12f);
  T = __fmaf_rn(T, x.x, 9.635426e-10f);
  T = __fmaf_rn(T, x.x, -1.2526054e-07f);
  df q = dfl_add_o(df_make(1.10229275e-05f, 1.5174285e-13f), dfl_mulf(x, T));   // 4 c4
  q = dfl_add_o(df_make(-0.0005952381f, 2.2728706e-11f), dfl_mul(x, q));          // 3 c3
  q = dfl_add_o(df_make(0.016666668f, -8.692344e-10f), dfl_mul(x, q));            // 2 c2
  q = dfl_add_o(df_make(-0.16666667f, 4.967054e-09f), dfl_mul(x, q));             // c1
  r.d = df_scale2(dfl_mul(u, q), 2.0f);
  return r;
}
// d sinc/du for |u| < 1e-3: u (-1/3 + u^2/30) (the dropped u^5/840 is below 1.2e-15 of the result)
__device__ __forceinline__ df df_dsinc_small(df u) {
  const df u2 = dfl_mul(u, u);
  const df p = df_make(-0.33333334f, __fmaf_rn(u2.x, 0.033333335f, 9.934108e-09f));
  return dfl_mul(u, p);
}

}  // namespace pe
