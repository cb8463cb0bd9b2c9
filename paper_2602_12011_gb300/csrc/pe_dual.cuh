// pe_dual.cuh -- forward-mode dual numbers over the 11 source parameters, used only in the
// per-sample preparation to obtain the exact derivatives of the sample coefficients with
// respect to theta (the chain-rule tail of the hand-written adjoint).
#pragma once
#include <cuda_runtime.h>

#include "pespace_gb300.h"

namespace pe {

// the global double overloads stay visible next to the Dn overloads declared below
using ::cbrt;
using ::cos;
using ::exp;
using ::log;
using ::pow;
using ::rint;
using ::sin;
using ::sincos;
using ::sqrt;

struct Dn {
  double v;
  double d[PE_NPARAM];
};

__device__ __forceinline__ Dn dconst(double x) {
  Dn r;
  r.v = x;
#pragma unroll
  for (int i = 0; i < PE_NPARAM; ++i) r.d[i] = 0.0;
  return r;
}
__device__ __forceinline__ Dn dvar(double x, int i) {
  Dn r = dconst(x);
  r.d[i] = 1.0;
  return r;
}
__device__ __forceinline__ double val(double x) { return x; }
__device__ __forceinline__ double val(const Dn& x) { return x.v; }

// chain rule: f(a) with f'(a.v) = df
__device__ __forceinline__ Dn dchain(const Dn& a, double f, double df) {
  Dn r;
  r.v = f;
#pragma unroll
  for (int i = 0; i < PE_NPARAM; ++i) r.d[i] = df * a.d[i];
  return r;
}
__device__ __forceinline__ Dn operator+(const Dn& a, const Dn& b) {
  Dn r; r.v = a.v + b.v;
#pragma unroll
  for (int i = 0; i < PE_NPARAM; ++i) r.d[i] = a.d[i] + b.d[i];
  return r;
}
__device__ __forceinline__ Dn operator-(const Dn& a, const Dn& b) {
  Dn r; r.v = a.v - b.v;
#pragma unroll
  for (int i = 0; i < PE_NPARAM; ++i) r.d[i] = a.d[i] - b.d[i];
  return r;
}
__device__ __forceinline__ Dn operator-(const Dn& a) {
  Dn r; r.v = -a.v;
#pragma unroll
  for (int i = 0; i < PE_NPARAM; ++i) r.d[i] = -a.d[i];
  return r;
}
__device__ __forceinline__ Dn operator*(const Dn& a, const Dn& b) {
  Dn r; r.v = a.v * b.v;
#pragma unroll
  for (int i = 0; i < PE_NPARAM; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i];
  return r;
}
__device__ __forceinline__ Dn operator/(const Dn& a, const Dn& b) {
  Dn r; r.v = a.v / b.v;
  const double ib = 1.0 / b.v;
#pragma unroll
  for (int i = 0; i < PE_NPARAM; ++i) r.d[i] = (a.d[i] - r.v * b.d[i]) * ib;
  return r;
}
__device__ __forceinline__ Dn operator+(const Dn& a, double b) { Dn r = a; r.v += b; return r; }
__device__ __forceinline__ Dn operator+(double b, const Dn& a) { Dn r = a; r.v += b; return r; }
__device__ __forceinline__ Dn operator-(const Dn& a, double b) { Dn r = a; r.v -= b; return r; }
__device__ __forceinline__ Dn operator-(double b, const Dn& a) { return (-a) + b; }
__device__ __forceinline__ Dn operator*(const Dn& a, double b) {
  Dn r; r.v = a.v * b;
#pragma unroll
  for (int i = 0; i < PE_NPARAM; ++i) r.d[i] = a.d[i] * b;
  return r;
}
__device__ __forceinline__ Dn operator*(double b, const Dn& a) { return a * b; }
__device__ __forceinline__ Dn operator/(const Dn& a, double b) {
  Dn r; r.v = a.v / b;
#pragma unroll
  for (int i = 0; i < PE_NPARAM; ++i) r.d[i] = a.d[i] / b;
  return r;
}
__device__ __forceinline__ Dn operator/(double a, const Dn& b) { return dconst(a) / b; }

__device__ __forceinline__ Dn sin(const Dn& a) { double s, c; ::sincos(a.v, &s, &c); return dchain(a, s, c); }
__device__ __forceinline__ Dn cos(const Dn& a) { double s, c; ::sincos(a.v, &s, &c); return dchain(a, c, -s); }
__device__ __forceinline__ void sincos(const Dn& a, Dn* s, Dn* c) {
  double sv, cv;
  ::sincos(a.v, &sv, &cv);
  *s = dchain(a, sv, cv);
  *c = dchain(a, cv, -sv);
}
__device__ __forceinline__ Dn sqrt(const Dn& a) { const double s = ::sqrt(a.v); return dchain(a, s, 0.5 / s); }
__device__ __forceinline__ Dn cbrt(const Dn& a) { const double c = ::cbrt(a.v); return dchain(a, c, c / (3.0 * a.v)); }
__device__ __forceinline__ Dn log(const Dn& a) { return dchain(a, ::log(a.v), 1.0 / a.v); }
__device__ __forceinline__ Dn pow(const Dn& a, double p) {
  const double f = ::pow(a.v, p);
  return dchain(a, f, p * f / a.v);
}
// rint is piecewise constant: derivative zero
__device__ __forceinline__ Dn rint(const Dn& a) { return dconst(::rint(a.v)); }

}  // namespace pe
