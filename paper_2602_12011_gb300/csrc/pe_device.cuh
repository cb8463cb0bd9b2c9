// pe_device.cuh -- device functions of the hot path (rows A1-A6): per-sample coefficients and
// the per-(sample, mode, bin) waveform, time-frequency map, orbit, single-link responses and TDI.
// arXiv:2602.12011 Sec. 2.1 (Eq. eq_td_resp, eq_tf, eq_fd_resp, FD TDI, A/E/T).
#pragma once
#include <cuda_runtime.h>

#include "pe_dual.cuh"
#include "pe_internal.h"

namespace pe {

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }

// sin and cos of 2 pi x for x in turns (|x| < 2^40): the nearest table angle 2 pi j/kSinTab and the
// remainder t = 2 pi (x - j/kSinTab) (|t| <= pi/kSinTab) through the angle-addition formulas with
// sin t = t - t^3/6 + t^5/120, cos t = 1 - t^2/2 + t^4/24 (truncation below 1e-18).
// tab[j] = (cos, sin)(2 pi j/kSinTab). Adding 1.5 * 2^42 rounds x to the nearest multiple of
// 2^-10 = 1/kSinTab (round to nearest even, as rint); subtracting it again gives that multiple
// exactly, x minus it is exact (Sterbenz), and the low ten bits of the sum's significand are j
// modulo kSinTab. So the turn reduction and the index need three FP64 additions and no FRND or
// conversion; the table's period absorbs the integer part of x.
static_assert(kSinTab == 1024, "the rounding constant below assumes kSinTab = 2^10");
__device__ __forceinline__ void sincos_turns(double x, const double2* __restrict__ tab, double* s, double* c) {
  constexpr double kRound = 6597069766656.0;   // 1.5 * 2^42
  const double sx = __dadd_rn(x, kRound);
  const double d = __dsub_rn(x, __dsub_rn(sx, kRound));
  const double2 cs = tab[__double2loint(sx) & (kSinTab - 1)];
  // sin(2 pi d) = d (c1 + u (c3 + u c5)) and cos(2 pi d) = 1 + u (c2 + u c4), u = d^2, with
  // c_n = (-1)^floor(n/2) (2 pi)^n / n! (correctly rounded): the Taylor series in t = 2 pi d with
  // 2 pi folded into the coefficients
  constexpr double kS1 = 6.283185307179586, kS3 = -41.34170224039976, kS5 = 81.60524927607506;
  constexpr double kC2 = -19.739208802178716, kC4 = 64.9393940226683;
  const double u = d * d;
  const double st = d * fma(u, fma(u, kS5, kS3), kS1);
  const double ct = fma(u, fma(u, kC4, kC2), 1.0);
  *s = fma(cs.y, ct, cs.x * st);
  *c = fma(cs.x, ct, -(cs.y * st));
}
// the same for an argument already reduced to a few turns (kept as a name for those call sites)
__device__ __forceinline__ void sincos_turns_r(double r, const double2* __restrict__ tab, double* s, double* c) {
  sincos_turns(r, tab, s, c);
}

// -2Y_lm(iota, 0) closed forms for the ten (l, +-m) the five modes need; ci, si: cos, sin of iota;
// c2, s2: cos, sin of iota/2.
template <class T>
__device__ inline void sylm_pair(int l, int m, const T& ci, const T& si, const T& c2, const T& s2, T* ypos, T* yneg) {
  const double pi = kPi;
  if (l == 2 && m == 2) {
    *ypos = sqrt(5.0 / (64.0 * pi)) * (1.0 + ci) * (1.0 + ci);
    *yneg = sqrt(5.0 / (64.0 * pi)) * (1.0 - ci) * (1.0 - ci);
  } else if (l == 2 && m == 1) {
    *ypos = sqrt(5.0 / (16.0 * pi)) * si * (1.0 + ci);
    *yneg = sqrt(5.0 / (16.0 * pi)) * si * (1.0 - ci);
  } else if (l == 3 && m == 3) {
    const T c4 = c2 * c2 * c2 * c2, s4 = s2 * s2 * s2 * s2;
    *ypos = -sqrt(21.0 / (2.0 * pi)) * c4 * c2 * s2;
    *yneg = sqrt(21.0 / (2.0 * pi)) * c2 * s4 * s2;
  } else if (l == 3 && m == 2) {
    const T c4 = c2 * c2 * c2 * c2, s4 = s2 * s2 * s2 * s2;
    *ypos = 0.5 * sqrt(7.0 / pi) * c4 * (3.0 * ci - 2.0);
    *yneg = sqrt(7.0 / (4.0 * pi)) * (3.0 * ci + 2.0) * s4;
  } else {  // (4, 4)
    const T cc = c2 * c2, ss = s2 * s2;
    *ypos = 3.0 * sqrt(7.0 / pi) * cc * cc * cc * ss;
    *yneg = 3.0 * sqrt(7.0 / pi) * cc * ss * ss * ss;
  }
}

// double -> double word (FP32 pair)
__device__ __forceinline__ float2 to_dw(double a) {
  const float h = __double2float_rn(a);
  return make_float2(h, __double2float_rn(a - (double)h));
}

__device__ __constant__ static const int kModeL[kNModes] = {2, 2, 3, 3, 4};
__device__ __constant__ static const int kModeM[kNModes] = {2, 1, 3, 2, 4};

// Domain of a parameter sample (out-of-domain samples get logL = -inf).
__device__ inline bool theta_valid(const double* th) {
  for (int i = 0; i < PE_NPARAM; ++i)
    if (!isfinite(th[i])) return false;
  if (!(th[0] >= 1e3 && th[0] <= 1e9)) return false;
  if (!(th[1] >= 1.0)) return false;
  if (!(fabs(th[2]) < 1.0 && fabs(th[3]) < 1.0)) return false;
  if (!(th[4] > 0.0)) return false;
  return true;
}

// Row A1: per-sample coefficients from theta[11].
//  TaylorF2 phase (Buonanno et al. 2009 3.5PN; 1.5PN spin-orbit, 2PN aligned spin-spin),
//  SPA amplitudes of the leading-order spherical modes (Blanchet 2014), C-infinity taper
//  on the orbital frequency between 0.9 F_isco and F_isco, -2Y_lm polarisation weights
//  (h_{l,-m} = (-1)^l h*_lm), sky frame. T = double, or Dn for derivatives with respect to theta.
// ln 6, ln 4, 6^(3/2); m^(-1/3) and ln(m)/3 for m = 0..4 (index m)
constexpr double kLn6 = 1.791759469228055, kLn4 = 1.3862943611198906, k6Pow15 = 14.696938456699069;
__device__ constexpr double kCbrtInv[5] = {0.0, 1.0, 0.7937005259840998, 0.6933612743506348, 0.6299605249474366};
__device__ constexpr double kLnM3[5] = {0.0, 0.0, 0.23104906018664842, 0.3662040962227033, 0.46209812037329684};

template <class T>
__device__ inline void sample_prep_t(const T* th, bool valid, unsigned mask, SampleCoefT<T>& S) {
  S.valid = valid ? 1 : 0;
  const T Mtot = th[0], q = th[1], chi1 = th[2], chi2 = th[3], dL = th[4], iota = th[5];
  const T phic = th[6], lam = th[7], bet = th[8], psi = th[9], tc = th[10];
  const T M = Mtot * kMsunS;
  const T D = dL * kGpcS;
  const T eta = q / ((1.0 + q) * (1.0 + q));
  const T m1 = q / (1.0 + q), m2 = 1.0 / (1.0 + q);
  const T delta = (q - 1.0) / (q + 1.0);
  const double pi = kPi;
  const T bso = chi1 * (113.0 / 12.0 * m1 * m1 + 25.0 / 4.0 * eta) + chi2 * (113.0 / 12.0 * m2 * m2 + 25.0 / 4.0 * eta);
  const T sss = 79.0 / 8.0 * eta * chi1 * chi2;
  const T a5c = pi * (38645.0 / 756.0 - 65.0 / 9.0 * eta);
  const T a6c = 11583231236531.0 / 4694215680.0 - 640.0 / 3.0 * pi * pi - 6848.0 / 21.0 * kEulerGamma +
                (-15737765635.0 / 3048192.0 + 2255.0 / 12.0 * pi * pi) * eta + 76055.0 / 1728.0 * eta * eta -
                127825.0 / 1296.0 * eta * eta * eta;
  const T n = 3.0 / (128.0 * eta);
  S.tc = tc;
  S.P[0] = n;
  S.P[1] = 0.0 * n;
  S.P[2] = n * (3715.0 / 756.0 + 55.0 / 9.0 * eta);
  S.P[3] = n * (-16.0 * pi + 4.0 * bso);
  S.P[4] = n * (15293365.0 / 508032.0 + 27145.0 / 504.0 * eta + 3085.0 / 72.0 * eta * eta - 10.0 * sss);
  S.P[5] = n * a5c * (1.0 + 1.5 * kLn6);                // alpha5 (1 + 3 ln(v/v_lso)), v_lso = 6^-1/2
  S.P[6] = n * (a6c - 6848.0 / 21.0 * kLn4);             // alpha6 - (6848/21) ln(4 v)
  S.P[7] = n * pi * (77096675.0 / 254016.0 + 378515.0 / 1512.0 * eta - 74045.0 / 756.0 * eta * eta);
  for (int k = 0; k < 8; ++k) S.Pd[k] = double(k - 5) * S.P[k];
  for (int k = 0; k < 8; ++k) S.Pdd[k] = double(k - 5) * S.Pd[k];
  S.Q5 = n * 3.0 * a5c;
  S.Q6 = n * (-6848.0 / 21.0);
  // sky frame
  T sl, cl, sb, cb, sp, cp;
  sincos(lam, &sl, &cl);
  sincos(bet, &sb, &cb);
  sincos(psi, &sp, &cp);
  S.k[0] = -(cb * cl); S.k[1] = -(cb * sl); S.k[2] = -sb;
  const T u[3] = {sl, -cl, 0.0 * sl};
  const T v[3] = {-(sb * cl), -(sb * sl), cb};
  for (int i = 0; i < 3; ++i) { S.p[i] = cp * u[i] + sp * v[i]; S.q[i] = -(sp * u[i]) + cp * v[i]; }
  for (int i = 0; i < 3; ++i) S.kw[i] = to_dw(val(S.k[i]));
  for (int k = 0; k < 8; ++k) S.Pdw[k] = to_dw(val(S.Pd[k]));
  for (int k = 0; k < 8; ++k) S.Pw[k] = to_dw(val(S.P[k]));
  S.Q5w = to_dw(val(S.Q5));
  S.Q6w = to_dw(val(S.Q6));
  S.tcw = to_dw(val(S.tc));
  // modes: (2 pi M / m)^(1/3) = (2 pi M)^(1/3) m^(-1/3) and its log from one cube root and one
  // log per sample; the spin-weighted harmonics share the sines and cosines of iota and iota/2
  const T Fisco = 1.0 / (k6Pow15 * 2.0 * pi * M);
  const T cm1 = cbrt(2.0 * pi * M);
  const T lncm1 = log(cm1);
  T ci, si, c2h, s2h;
  sincos(iota, &si, &ci);
  sincos(0.5 * iota, &s2h, &c2h);
  for (int md = 0; md < kNModes; ++md) {
    ModeCoefT<T>& C = S.md[md];
    const int l = kModeL[md], m = kModeM[md];
    T hmag;          // |H_lm| / x^(p/2)
    double argt;     // arg(conj H_lm) in turns
    int p;
    if (md == 0) { hmag = 1.0 + 0.0 * q; argt = 0.0; p = 0; }
    else if (md == 1) { hmag = delta / 3.0; argt = -0.25; p = 1; }
    else if (md == 2) { hmag = 0.75 * ::sqrt(15.0 / 14.0) * delta; argt = 0.25; p = 1; }
    else if (md == 3) { hmag = ::sqrt(5.0 / 7.0) / 3.0 * (1.0 - 3.0 * eta); argt = 0.0; p = 2; }
    else { hmag = 8.0 / 9.0 * ::sqrt(5.0 / 7.0) * (1.0 - 3.0 * eta); argt = 0.5; p = 2; }
    C.cm = cm1 * kCbrtInv[m];
    C.icm = 1.0 / C.cm;
    C.lncm = lncm1 - kLnM3[m];
    C.amp = 2.0 * pi * M * M / D * sqrt(eta / (3.0 * m)) * hmag * (C.icm * C.icm * C.icm / sqrt(C.cm));
    const T icm2 = C.icm * C.icm;
    C.icm5 = icm2 * icm2 * C.icm;
    C.ampp = p == 0 ? C.amp : (p == 1 ? C.amp * C.cm : C.amp * C.cm * C.cm);
    const T ph = m * phic / (2.0 * pi) + (0.125 + argt);
    C.ph0 = ph - rint(ph);
    C.mfac = 0.0 * q + m / (4.0 * pi);
    C.tffac = 0.0 * q + m / (12.0 * pi);
    T yp, yn;
    sylm_pair(l, m, ci, si, c2h, s2h, &yp, &yn);
    const double sgn = (l % 2) ? -1.0 : 1.0;
    C.Pp = 0.5 * (yp + sgn * yn);
    C.Pc = 0.5 * (sgn * yn - yp);
    C.Pc2 = sgn * yn - yp;
    C.fend = double(m) * Fisco;
    C.ftap = 0.9 * double(m) * Fisco;
    C.Ppw = to_dw(val(C.Pp));
    C.Pcw = to_dw(val(C.Pc));
    C.tffacw = to_dw(val(C.tffac));
    C.ph0w = to_dw(val(C.ph0));
    C.p = p;
    C.active = (valid && (mask & (1u << md)) && val(hmag) != 0.0) ? 1 : 0;
  }
  const double a0 = val(S.md[0].amp);
  const int e0 = (a0 > 0.0 && isfinite(a0)) ? ilogb(a0) : 0;
  S.hsc = scalbn(1.0, -e0);
  S.ihsc = scalbn(1.0, e0);
  for (int md = 0; md < kNModes; ++md) {
    S.md[md].cmw = to_dw(val(S.md[md].cm));
    S.md[md].ampw = to_dw(val(S.md[md].amp) * S.hsc);
  }
  S.pair32 = (S.md[0].active && S.md[3].active) ? 1 : 0;
  S.k32 = make_double2(0.0, 0.0);
  if (S.pair32) {
    double sd, cd;
    sincospi(2.0 * (val(S.md[3].ph0) - val(S.md[0].ph0)), &sd, &cd);
    const double r = val(S.md[3].amp) / val(S.md[0].amp);
    S.k32 = make_double2(r * cd, r * sd);
  }
  S.k32w[0] = to_dw(S.k32.x);
  S.k32w[1] = to_dw(S.k32.y);
}

__device__ inline void sample_prep(const double* th, unsigned mask, SampleCoef& S) {
  sample_prep_t<double>(th, theta_valid(th), mask, S);
}

// Spacecraft offsets delta_i from the constellation centre and the centre x_c, at time t.
__device__ __forceinline__ void orbit_offsets(const DetDev& D, double t, double xc[3], double dl[3][3],
                                              const double2* __restrict__ tab) {
  double s, c;
  sincos_turns(fma(t, D.rate_t, D.alpha0_t), tab, &s, &c);
  xc[0] = D.R * c; xc[1] = D.R * s; xc[2] = 0.0;
  if (D.orbit == 0) {
    const double c2 = c * c - s * s, s2 = 2.0 * s * c;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      dl[i][0] = D.eRh * (c2 * D.cb[i] + s2 * D.sb[i]) - D.eR3h * D.cb[i];
      dl[i][1] = D.eRh * (s2 * D.cb[i] - c2 * D.sb[i]) - D.eR3h * D.sb[i];
      dl[i][2] = -D.eRs3 * (c * D.cb[i] + s * D.sb[i]);
    }
  } else {
    double s0, c0;
    sincos_turns(t * D.geo_rate_t, tab, &s0, &c0);
    const double ch = -0.5, sh = 0.86602540378443864676;  // cos, sin of 120 degrees
    double ci = c0, si = s0;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
#pragma unroll
      for (int j = 0; j < 3; ++j) dl[i][j] = D.rgeo * (ci * D.e1[j] + si * D.e2[j]);
      const double cn = ci * ch - si * sh, sn = si * ch + ci * sh;
      ci = cn; si = sn;
    }
  }
}

// sinc(u) with the same small-argument series as the definition: 1 - u^2/6 + u^4/120 - u^6/5040
__device__ __forceinline__ double sinc_small(double u) {
  const double u2 = u * u;
  return 1.0 - u2 / 6.0 + u2 * u2 / 120.0 - u2 * u2 * u2 / 5040.0;
}

// sinc(u) = sum_k (-1)^k u^(2k) / (2k+1)! (Horner in x = u^2), for |u| <= 1: through u^16, where
// the first dropped term is below 1/19! = 8.2e-18, under half an ulp of sinc(u) >= sin 1. Shorter
// sums serve smaller |u|: through u^12 for |u| <= 0.4 (dropped term < 2e-18) and through u^8 for
// |u| <= 0.1 (< 3e-18). The caller picks the length from the bin (|u| <= 2a, a = pi f L).
constexpr double kSincPolyA = 0.5;   // bins with a below this take a polynomial
constexpr double kSincPolyA12 = 0.2;
constexpr double kSincPolyA8 = 0.05;
template <int DEG>   // highest power of x kept: 8, 6 or 4; argument x = u^2
__device__ __forceinline__ double sinc_poly_x(double x) {
  double p = DEG >= 8 ? 1.0 / 355687428096000.0 : (DEG >= 6 ? 1.0 / 6227020800.0 : 1.0 / 362880.0);
  if (DEG >= 8) {
    p = fma(p, x, -1.0 / 1307674368000.0);        // 1/15!
    p = fma(p, x, 1.0 / 6227020800.0);            // 1/13!
  }
  if (DEG >= 6) {
    p = fma(p, x, -1.0 / 39916800.0);             // 1/11!
    p = fma(p, x, 1.0 / 362880.0);                // 1/9!
  }
  p = fma(p, x, -1.0 / 5040.0);                   // 1/7!
  p = fma(p, x, 1.0 / 120.0);                     // 1/5!
  p = fma(p, x, -1.0 / 6.0);                      // 1/3!
  return fma(p, x, 1.0);
}
template <int DEG>
__device__ __forceinline__ double sinc_poly_n(double u) { return sinc_poly_x<DEG>(u * u); }
__device__ __forceinline__ double sinc_poly(double u) { return sinc_poly_n<8>(u); }
// sinc(u) and d sinc/du = u sum_{k>=1} 2k (-1)^k u^(2k-2) / (2k+1)! through the same order as
// sinc_poly_n<DEG>
template <int DEG>
__device__ __forceinline__ void sinc_poly_d_n(double u, double* sv, double* dv) {
  const double x = u * u;
  *sv = sinc_poly_n<DEG>(u);
  double q = DEG >= 8 ? 1.0 / 22230464256000.0 : (DEG >= 6 ? 1.0 / 518918400.0 : 1.0 / 45360.0);
  if (DEG >= 8) {
    q = fma(q, x, -1.0 / 93405312000.0);          // 14/15!
    q = fma(q, x, 1.0 / 518918400.0);             // 12/13!
  }
  if (DEG >= 6) {
    q = fma(q, x, -1.0 / 3991680.0);              // 10/11!
    q = fma(q, x, 1.0 / 45360.0);                 // 8/9!
  }
  q = fma(q, x, -1.0 / 840.0);                    // 6/7!
  q = fma(q, x, 1.0 / 30.0);                      // 4/5!
  q = fma(q, x, -1.0 / 3.0);                      // 2/3!
  *dv = u * q;
}
__device__ __forceinline__ void sinc_poly_d(double u, double* sv, double* dv) { sinc_poly_d_n<8>(u, sv, dv); }

// Projections of the geometry on the sample's frame as linear forms in the orbit basis b
// (DetDev::Mo), formed once per (detector, sample) tile into shared memory (kProj doubles):
//   pc[15 l + 5 v + m]: v-component (v = k, p, q) of the unnormalised link vector
//                       n'_l = delta_r - delta_s, link l = (r, s) = (0,1), (1,2), (2,0);
//   pc[45 + 5 i + m]:   k.delta_i, spacecraft i = 0, 1 (the third-spacecraft phases).
// Since (k, p, q) is orthonormal, |n'|^2 = (k.n')^2 + (p.n')^2 + (q.n')^2.
//   pc[55], pc[56]:     R k_x, R k_y (the centre's Doppler term k.x_c = R (k_x cos alpha + k_y sin alpha)).
constexpr int kProj = 57;
__device__ __forceinline__ double proj_coef(const DetDev& D, const SampleCoef& S, int i) {
  if (i >= 55) return D.R * S.k[i - 55];
  const int m = i % 5;
  if (i < 45) {
    const int l = i / 15, v = (i / 5) % 3, r = l, s = (l + 1) % 3;
    const double* w = v == 0 ? S.k : (v == 1 ? S.p : S.q);
    return w[0] * (D.Mo[r][0][m] - D.Mo[s][0][m]) + w[1] * (D.Mo[r][1][m] - D.Mo[s][1][m]) +
           w[2] * (D.Mo[r][2][m] - D.Mo[s][2][m]);
  }
  const int e = (i - 45) / 5;
  return S.k[0] * D.Mo[e][0][m] + S.k[1] * D.Mo[e][1][m] + S.k[2] * D.Mo[e][2][m];
}
// Every thread of the CTA calls this at the start of a tile (a barrier on both sides).
__device__ __forceinline__ void proj_prologue(const DetDev& D, const SampleCoef& S, double* pc) {
  __syncthreads();
  for (int i = threadIdx.x; i < kProj; i += blockDim.x) pc[i] = proj_coef(D, S, i);
  __syncthreads();
}
// p[0..3] . b + p[4]. p points to shared memory, read through a volatile pointer so that the 55
// forms are loaded where they are used (broadcast loads) instead of being held in registers
// across the mode loop.
__device__ __forceinline__ double dot5(const volatile double* p, const double b[4]) {
  return fma(p[0], b[0], fma(p[1], b[1], fma(p[2], b[2], fma(p[3], b[3], p[4]))));
}
// Orbit at time t: (cos, sin) of the centre's angle alpha and the offsets' basis b.
__device__ __forceinline__ void orbit_basis(const DetDev& D, double t, const double2* __restrict__ tab, double* c,
                                            double* s, double b[4]) {
  sincos_turns(fma(t, D.rate_t, D.alpha0_t), tab, s, c);
  if (D.orbit == 0) {
    b[0] = *c * *c - *s * *s;
    b[1] = 2.0 * *s * *c;
    b[2] = *c;
    b[3] = *s;
  } else {
    sincos_turns(t * D.geo_rate_t, tab, &b[1], &b[0]);
    b[2] = 0.0;
    b[3] = 0.0;
  }
}

// Mode-summed link products of one bin: S_l = sum over modes of G_l s+_l and M_l = sum of G_l s-_l,
// for the links l = 0 (1,2), 1 (2,3), 2 (3,1). The TDI brackets follow once per bin (xyz_final):
// X' = P_X + z Q_X (and Y', Z' alike) with P_c = S_{c+2} - M_c and Q_c = M_{c+2} - S_c (link
// indices mod 3); z depends on the bin only. Each unit adds four products per link, once each,
// where summing into the brackets would add each product into two of them.
struct XYZAcc {
  double2 S[3], M[3];
};
__device__ __forceinline__ void xyz_zero(XYZAcc& a) {
#pragma unroll
  for (int i = 0; i < 3; ++i) a.S[i] = a.M[i] = make_double2(0.0, 0.0);
}
__device__ __forceinline__ void xyz_final(const XYZAcc& a, double2 z, double2 x[3]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const int lp = (c + 2) % 3;
    x[c] = cadd(csub(a.S[lp], a.M[c]), cmul(z, csub(a.M[lp], a.S[c])));
  }
}

// Per-bin inputs shared by all modes of one bin.
// a < b for non-negative doubles by the order of their bit patterns: an integer compare, exact
// (GB300 runs the double compare DSETP on its narrow FP64 pipe)
__device__ __forceinline__ bool dlt_pos(double a, double b) { return __double_as_longlong(a) < __double_as_longlong(b); }

struct BinIn {
  double f, f13, fm13, lnf3, fm76, invf;
  double a, sa, ca;    // a = pi f L
  double a2, a2x2;     // a^2, 2 a^2
  double hf;           // f / 2
  int sdeg;            // sinc polynomial class of the bin: 0, 1, 2 (degree 8, 12, 16 in u), 3 (none)
  int b;               // bin index (for the tables read per unit)
  double aturn;        // a / (2 pi) = f L / 2
  double2 z;           // e^{-2 i a}
  double frc;          // frac(f t_c) computed exactly (turns)
};

// One (sample, mode, bin) unit: adds this mode's TDI brackets X', Y', Z' (Sec. 2.1) to acc.
// X = Q X' with Q = TDI factor (-i a) e^{-ia}; here
//   X' = G31 V31 - G12 U12,  Y' = G12 V12 - G23 U23,  Z' = G23 V23 - G31 U31,
// G_l = e^{i pi f k.delta_t} (n_l.h~.n_l) per link pair l=(r,s) with third spacecraft t,
// U_l = s-_l + z s+_l, V_l = s+_l + z s-_l, s-+_l = sinc(a(1 -+ k.n_l)),
// n_l = (x_r - x_s)/|x_r - x_s|, geometry at the mode's t_f, and the centre Doppler phase
// e^{-2 pi i f k.x_c} folded into the mode's phase. Written as X' = P_X + z Q_X with
// P_X = G31 s+31 - G12 s-12, Q_X = G31 s-31 - G12 s+12 (and cyclically for Y', Z').
// C2 (nullable): a second mode with the same m, evaluated with this one's geometry (see k32).
__device__ __forceinline__ void mode_bin(const DetDev& D, const SampleCoef& S, const ModeCoef& C, const BinIn& B,
                                         XYZAcc& acc, const double2* __restrict__ tab, const double* __restrict__ pc,
                                         const ModeCoef* C2 = nullptr) {
  // --- waveform and time-frequency map (rows A2, A3)
  const double v = C.cm * B.f13;
  const double lnv = C.lncm + B.lnf3;
  const double iv5 = C.icm5 * D.fm53[B.b];   // v^-5 = cm^-5 f^(-5/3)
  double poly = S.P[7];
  double dpol = S.Pd[7];
#pragma unroll
  for (int k = 6; k >= 0; --k) {
    poly = fma(poly, v, S.P[k]);
    dpol = fma(dpol, v, S.Pd[k]);
  }
  const double q56 = fma(S.Q6, v, S.Q5);
  const double psi_pn = fma(iv5, poly, lnv * q56);
  const double dv = fma(iv5, dpol, fma(S.Q6 * v, lnv, q56));   // v dPsi_PN/dv = v^-5 sum_k (k-5) P_k v^k + Q5 + Q6 v (1 + ln v)
  const double tf = fma(C.tffac * B.invf, dv, S.tc);            // Eq. eq_tf
  // amp v^p f^(-7/6) = (amp cm^p) f^(-7/6 + p/3), times the Planck taper inside it
  double amp = C.ampp * (C.p == 0 ? B.fm76 : (C.p == 1 ? D.fm56[B.b] : D.fm12[B.b]));
  if (dlt_pos(C.ftap, B.f)) {
    const double span = C.fend - C.ftap;
    const double zt = span / (C.fend - B.f) - span / (B.f - C.ftap);
    amp *= (zt > 700.0) ? 0.0 : 1.0 / (1.0 + exp(zt));
  }
  // --- orbit at t_f (row A4): centre angle and the offsets' basis
  double co, so, ob[4];
  orbit_basis(D, tf, tab, &co, &so, ob);
  const double kxc = fma(pc[55], co, pc[56] * so);   // k.x_c
  const double ph = fma(-C.mfac, psi_pn, C.ph0 - B.frc) - B.f * kxc;
  const double phr = ph - rint(ph);
  // polarisation weights times the amplitude (x weight doubled, see Fx below); a paired second
  // mode makes them complex: Pp + kappa Pp2, Pc + kappa Pc2, kappa = k32 v^2
  double2 Ap = make_double2(amp * C.Pp, 0.0), Ac = make_double2(amp * C.Pc2, 0.0);
  if (C2) {
    const double v2 = v * v;
    const double kr = S.k32.x * v2, ki = S.k32.y * v2;
    Ap = make_double2(amp * fma(kr, C2->Pp, C.Pp), amp * (ki * C2->Pp));
    Ac = make_double2(amp * fma(kr, C2->Pc2, C.Pc2), amp * (ki * C2->Pc2));
  }
  // mode phase times the third spacecraft's phase e^{i pi f k.delta_t}, one sincos per spacecraft;
  // the offsets sum to zero, so delta_2's phase is minus the other two
  double2 E[3];
  {
    const double e0 = B.hf * dot5(pc + 45, ob), e1 = B.hf * dot5(pc + 50, ob);
    sincos_turns_r(phr + e0, tab, &E[0].y, &E[0].x);
    sincos_turns_r(phr + e1, tab, &E[1].y, &E[1].x);
    sincos_turns_r(phr - (e0 + e1), tab, &E[2].y, &E[2].x);
  }
  // --- links (row A5): pair l = (1,2), (2,3), (3,1); third spacecraft 3, 1, 2. Projections of
  // the unnormalised link vectors x_r - x_s: the three sum to zero, so the third is minus the
  // other two
  double knr[3], npr[3], nqr[3];
#pragma unroll
  for (int l = 0; l < 2; ++l) {
    knr[l] = dot5(pc + 15 * l, ob);
    npr[l] = dot5(pc + 15 * l + 5, ob);
    nqr[l] = dot5(pc + 15 * l + 10, ob);
  }
  knr[2] = -(knr[0] + knr[1]);
  npr[2] = -(npr[0] + npr[1]);
  nqr[2] = -(nqr[0] + nqr[1]);
#pragma unroll
  for (int l = 0; l < 3; ++l) {
    const int t = (l + 2) % 3;
    // k.n, n.e+.n, n.ex.n of the unit link vector
    const double inv = rsqrt(fma(knr[l], knr[l], fma(npr[l], npr[l], nqr[l] * nqr[l])));
    const double kn = knr[l] * inv;
    const double np = npr[l] * inv, nq = nqr[l] * inv;
    // F+ = (n.p)^2 - (n.q)^2, Fx = 2 (n.p)(n.q); the 2 is in Ac (built from 2 Pc)
    const double Fp = np * np - nq * nq, Fch = np * nq;
    const double2 gam = C2 ? make_double2(fma(Ap.x, Fp, -Ac.y * Fch), fma(Ap.y, Fp, Ac.x * Fch))
                           : make_double2(Ap.x * Fp, Ac.x * Fch);
    const double2 G = cmul(gam, E[t]);
    // sinc(a(1 -+ kn)): Taylor polynomial while a < kSincPolyA (most bins of a massive-binary
    // signal), else from sin(a -+ a kn) = sin a cos(a kn) -+ cos a sin(a kn)
    // below a = kSincPolyA (degree class B.sdeg < 3, chosen once per bin): u1^2 = a^2 (1 - kn)^2 =
    // a^2 + kn (a^2 kn - 2 a^2) and u2^2 = a^2 + kn (a^2 kn + 2 a^2), two FMAs each; where u1 or u2
    // is small the cancellation error is ~ulp(a^2), far below what sinc resolves
    double sm, spl;
    if (B.sdeg < 3) {
      const double x1 = fma(kn, fma(B.a2, kn, -B.a2x2), B.a2), x2 = fma(kn, fma(B.a2, kn, B.a2x2), B.a2);
      if (B.sdeg == 0) {
        sm = sinc_poly_x<4>(x1);
        spl = sinc_poly_x<4>(x2);
      } else if (B.sdeg == 1) {
        sm = sinc_poly_x<6>(x1);
        spl = sinc_poly_x<6>(x2);
      } else {
        sm = sinc_poly_x<8>(x1);
        spl = sinc_poly_x<8>(x2);
      }
    } else {
      const double u1 = B.a * (1.0 - kn), u2 = B.a * (1.0 + kn);
      double sak, cak;
      sincos_turns(B.aturn * kn, tab, &sak, &cak);
      const double s1 = B.sa * cak - B.ca * sak, s2 = B.sa * cak + B.ca * sak;
      const bool small1 = dlt_pos(fabs(u1), 1e-3), small2 = dlt_pos(fabs(u2), 1e-3);
      if (!small1 && !small2) {
        const double rr = 1.0 / (u1 * u2);
        sm = s1 * u2 * rr;
        spl = s2 * u1 * rr;
      } else {
        sm = small1 ? sinc_small(u1) : s1 / u1;
        spl = small2 ? sinc_small(u2) : s2 / u2;
      }
    }
    // --- the link's products for the TDI brackets (row A6; see XYZAcc)
    acc.S[l].x = fma(G.x, spl, acc.S[l].x);
    acc.S[l].y = fma(G.y, spl, acc.S[l].y);
    acc.M[l].x = fma(G.x, sm, acc.M[l].x);
    acc.M[l].y = fma(G.y, sm, acc.M[l].y);
  }
}

__device__ __forceinline__ void load_bin(const DetDev& D, int b, double tc, BinIn& B) {
  B.f = D.f[b];
  B.f13 = D.f13[b];
  B.fm13 = D.fm13[b];
  B.lnf3 = D.lnf3[b];
  B.fm76 = D.fm76[b];
  B.invf = B.fm13 * B.fm13 * B.fm13;
  B.a = kPi * B.f * D.L;
  B.a2 = B.a * B.a;
  B.a2x2 = 2.0 * B.a2;
  B.hf = 0.5 * B.f;
  B.sdeg = dlt_pos(B.a, kSincPolyA8) ? 0 : (dlt_pos(B.a, kSincPolyA12) ? 1 : (dlt_pos(B.a, kSincPolyA) ? 2 : 3));
  B.b = b;
  B.aturn = 0.5 * B.f * D.L;
  const double2 sc = D.sca[b];
  B.sa = sc.x; B.ca = sc.y;
  B.z = D.z[b];
  // frac(f t_c) without rounding the product: p + e = f t_c exactly (FMA two-product)
  const double pr = B.f * tc;
  const double er = fma(B.f, tc, -pr);
  B.frc = (pr - rint(pr)) + er;
}

// Adds every active mode of one sample at one bin to a; (2,2) and (3,2) go through one unit when
// both are active (pair32).
__device__ __forceinline__ void bin_modes(const DetDev& D, const SampleCoef& S, const BinIn& B, XYZAcc& a,
                                          const double2* __restrict__ tab, const double* __restrict__ pc) {
#pragma unroll 1
  for (int md = 0; md < kNModes; ++md) {
    if (md == 3 && S.pair32) continue;
    const ModeCoef& C = S.md[md];
    if (!C.active || !dlt_pos(B.f, C.fend)) continue;
    mode_bin(D, S, C, B, a, tab, pc, (md == 0 && S.pair32) ? &S.md[3] : nullptr);
  }
}

// Mode-summed TDI brackets X', Y', Z' of one sample at one bin.
__device__ __forceinline__ void bin_xyz(const DetDev& D, const SampleCoef& S, int b, double2 acc[3],
                                        const double2* __restrict__ tab, const double* __restrict__ pc) {
  BinIn B;
  load_bin(D, b, S.tc, B);
  XYZAcc a;
  xyz_zero(a);
  bin_modes(D, S, B, a, tab, pc);
  xyz_final(a, B.z, acc);
}

// Adds one bin's PSD-weighted products to the running sums: v[c] += Re(dg_c B_c),
// v[3+c] += gg_c |B_c|^2 (explicitly rounded, so every kernel that uses it adds identically).
__device__ __forceinline__ void accum_bin(const DetDev& D, int b, const double2 o[3], double v[6]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const double2 g = D.dg[c * D.nb + b];
    v[c] = __dadd_rn(v[c], __fma_rn(g.x, o[c].x, -__dmul_rn(g.y, o[c].y)));
    v[3 + c] = __dadd_rn(v[3 + c], __dmul_rn(D.gg[c * D.nb + b], __fma_rn(o[c].x, o[c].x, __dmul_rn(o[c].y, o[c].y))));
  }
}

// Block reduction of NV doubles per thread in a fixed tree order; result valid in thread 0.
template <int NV>
__device__ __forceinline__ void block_sum(double v[NV], double (*sh)[kTileBins / 32]) {
#pragma unroll
  for (int i = 0; i < NV; ++i)
    for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_down_sync(0xffffffffu, v[i], o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int i = 0; i < NV; ++i) sh[i][wid] = v[i];
  __syncthreads();
  if (threadIdx.x == 0)
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      double s = sh[i][0];
      for (int w = 1; w < kTileBins / 32; ++w) s += sh[i][w];
      v[i] = s;
    }
}

// Block sum of the six per-thread values of the forward kernels (<d|h>_c, <h|h>_c) through shared
// memory: every thread stores its six values in red[i][threadIdx.x]; thread t < 96 adds entries
// g, g + 16, ..., g + 112 of row i = t / 16 (g = t % 16) in that order into red[i][g]; thread i < 6
// then adds red[i][0..15] in order. About 6 additions per thread against 30 for a shuffle tree per
// value, and no lane-dependent shuffles. Rows are padded by kRedPad entries so that the six final
// readers hit different banks. Returns true in threads 0..5, with the block's sum of
// v[threadIdx.x] in *out.
constexpr int kRedPad = 2;
template <class T, class Add>
__device__ __forceinline__ bool block_sum6(const T v[6], Add add, T (*red)[kTileBins + kRedPad], T* out) {
  __syncthreads();   // the previous call's final readers are done with red
#pragma unroll
  for (int i = 0; i < 6; ++i) red[i][threadIdx.x] = v[i];
  __syncthreads();
  if (threadIdx.x < 6 * 16) {
    const int i = threadIdx.x >> 4, g = threadIdx.x & 15;
    T s = red[i][g];
#pragma unroll
    for (int k = 1; k < kTileBins / 16; ++k) s = add(s, red[i][g + 16 * k]);
    red[i][g] = s;   // only this thread reads or writes column g of row i in this step
  }
  __syncthreads();
  if (threadIdx.x >= 6) return false;
  T s = red[threadIdx.x][0];
#pragma unroll
  for (int g = 1; g < 16; ++g) s = add(s, red[threadIdx.x][g]);
  *out = s;
  return true;
}

// A/E/T combinations (without Q n_c): B_A = Z' - X', B_E = X' - 2Y' + Z', B_T = X' + Y' + Z'.
__device__ __forceinline__ void aet_from_xyz(const double2 x[3], double2 o[3]) {
  o[0] = csub(x[2], x[0]);
  o[1] = cadd(csub(x[0], cscale(x[1], 2.0)), x[2]);
  o[2] = cadd(cadd(x[0], x[1]), x[2]);
}

}  // namespace pe
