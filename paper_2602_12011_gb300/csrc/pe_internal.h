// pe_internal.h -- library-internal layouts shared by the host code and the CUDA kernels of
// libpespace_gb300. Nothing here is part of the public ABI (include/pespace_gb300.h).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "pespace_gb300.h"

namespace pe {

// Physical constants (the library's own copy).
constexpr double kPi = 3.14159265358979323846;
constexpr double kC = 299792458.0;                 // speed of light [m/s]
constexpr double kMsunS = 4.925490947641267e-6;    // G Msun / c^3 [s]
constexpr double kGpcS = 1.02927125054339e17;      // 1 Gpc / c [s]
constexpr double kAuS = 499.00478383615643;        // 1 au / c [s]
constexpr double kYearS = 31557600.0;              // Julian year [s]
constexpr double kEulerGamma = 0.57721566490153286061;

constexpr int kNModes = 5;      // (2,2) (2,1) (3,3) (3,2) (4,4)
constexpr int kMaxDet = 8;
constexpr int kTileBins = 128;  // frequency bins per (sub-)tile = threads per CTA of the hot kernels
// Arithmetic of the forward path (mode-mask flags PE_PREC_MIXED, PE_PREC_FP32).
constexpr int kPrecFP64 = 0, kPrecMixed = 1, kPrecFP32 = 2;
// Work items of the log-likelihood kernels are R consecutive 128-bin sub-tiles of one (detector,
// sample) pair, R in {1, 2, 4, 8} picked by the autotuner. The default (no tuned choice) keeps
// one sub-tile per item in FP64 (most CTAs for small batches) and four in the other precisions,
// which amortise their per-item staging over more bins. Each sub-tile keeps its own partial, so R
// never changes a result.
constexpr int kFwdMaxSubtiles = 8;
__host__ __device__ constexpr int fwd_default_subtiles(int prec) { return prec == kPrecFP64 ? 1 : 4; }
constexpr int kSinTab = 1024;   // entries of the (cos, sin) table used by sincos_turns

// Per-(sample, mode) coefficients (row A1 of the path). With v = (2 pi M f/m)^(1/3):
//   v = cm f^(1/3), 1/v = icm f^(-1/3), ln v = lncm + ln(f)/3,
//   |H~_lm(f)| = amp f^(-7/6) v^p w(f)   (w: Planck taper, 1 for f <= ftap, 0 for f >= fend),
//   arg H~_lm(f) = 2 pi [ ph0 - f t_c - (m/4pi) Psi_PN(v) ] (turns, before the orbit's
//   centre Doppler term), and the mode's tensor is H~ (Pp e+ + i Pc ex).
// Templated on the scalar so that the same code gives values (double) and, with device dual
// numbers, their derivatives with respect to theta.
template <class T>
struct ModeCoefT {
  T cm, icm, lncm;
  T icm5;       // icm^5 (v^-5 = icm5 f^(-5/3))
  T amp;
  T ampp;       // amp cm^p (amp v^p = ampp f^(p/3))
  T ph0;
  T mfac;       // m / (4 pi)
  T tffac;      // m / (12 pi)
  T Pp, Pc;
  T Pc2;        // 2 Pc (the FP64 unit folds the 2 of Fx = 2 (n.p)(n.q) into it)
  T fend, ftap;
  float2 Ppw, Pcw;   // Pp, Pc as double words (FP32 pairs) for the mixed-precision path
  float2 cmw;        // cm as a double word
  float2 ampw;       // amp times the sample's hsc as a double word
  float2 tffacw;     // tffac as a double word
  float2 ph0w;       // ph0 as a double word
  int p;        // power of v in |H_lm|: 0 (22), 1 (21, 33), 2 (32, 44)
  int active;   // 1 if the mode is in the mask and its amplitude is non-zero
};

// Per-sample coefficients. Psi_PN(v) = v^-5 sum_k P[k] v^k + ln v (Q5 + Q6 v) (TaylorF2 3.5PN,
// already multiplied by 3/(128 eta)).
template <class T>
struct SampleCoefT {
  T tc;
  T P[8];
  T Pd[8];              // (k - 5) P[k]: coefficients of v dPsi_PN/dv
  T Pdd[8];             // (k - 5)^2 P[k]: coefficients of v d(v dPsi_PN/dv)/dv (reverse sweeps)
  T Q5, Q6;
  T k[3], p[3], q[3];   // propagation direction and polarisation frame
  float2 kw[3];         // k as double words
  float2 Pdw[8];        // Pd, Q6 and tc as double words (the mixed path's t_f)
  float2 Q6w, tcw;
  float2 Pw[8], Q5w;    // P and Q5 as double words (the mixed surrogate's node phase)
  double hsc, ihsc;     // power of two near 1/amp of the (2,2) mode and its inverse: the mixed-
                        // precision path carries amplitudes times hsc, keeping them far from the
                        // FP32 range limits
  ModeCoefT<T> md[kNModes];
  // (3,2) shares m = 2 with (2,2), hence v, t_f, the taper and every geometric factor; its signal
  // is k32 v^2 times that of (2,2) with its own polarisation weights, k32 = (amp_32 / amp_22)
  // e^{2 pi i (ph0_32 - ph0_22)}. pair32 = 1 when both are active, and the units evaluate them
  // together.
  double2 k32;
  float2 k32w[2];       // k32 (re, im) as double words
  int valid;
  int pair32;
};

using ModeCoef = ModeCoefT<double>;
using SampleCoef = SampleCoefT<double>;

// Derivatives of the per-sample coefficients with respect to theta that the adjoint needs
// (the sparsity of the map theta -> coefficients is built in: P and Q depend on q, chi1, chi2;
// amp on Mtot, q, dL; cm and the taper on Mtot; the polarisation weights on iota; the sky
// frame on lambda, beta, psi).
struct ModeGrad {
  double dlnA_dM, dlnA_dq;   // d ln(amp)/d Mtot, d ln(amp)/d q
  double dcm_dM;             // d cm / d Mtot
  double dfend_dM;           // d fend / d Mtot (ftap = 0.9 fend)
  double dPp_di, dPc_di;     // d Pp/d iota, d Pc/d iota
};
struct SampleGrad {
  double dP_dq[8], dQ5_dq, dQ6_dq;
  double dPd_dq[8];     // (k - 5) dP_dq[k]
  double dP3_dc1, dP4_dc1, dP3_dc2, dP4_dc2;
  double dlnA_ddL;           // -1/dL
  double dk[3][3], dp[3][3], dq[3][3];   // [component][lambda, beta, psi]
  ModeGrad md[kNModes];
};

// Device view of one detector: grid, orbit constants and per-bin SoA tables.
struct DetDev {
  double T;          // observation time = 1/df [s]
  long long k0;      // first bin index
  int nb;            // number of bins
  int orbit;         // 0 heliocentric, 1 geocentric
  int tdi_gen;
  int pad_;
  double L;          // nominal arm [s]
  // orbit: centre R (cos alpha, sin alpha, 0), alpha in half-turns = alpha0_ht + t * rate_ht
  // (alpha0_t, rate_t: the same in turns)
  double R, alpha0_ht, rate_ht, alpha0_t, rate_t;
  // heliocentric (first order in e): offsets from the centre use eRh = e R / 2,
  // eR3h = 3 e R / 2, eRs3 = sqrt(3) e R and the spacecraft angles cb[i], sb[i].
  double eRh, eR3h, eRs3;
  double cb[3], sb[3];
  // geocentric: offsets r (cos phi_i e1 + sin phi_i e2), phi_0 in half-turns = t * geo_rate_ht
  double rgeo, geo_rate_ht, geo_rate_t;
  double e1[3], e2[3];
  // per-bin tables (length nb)
  const double* f;      // f_k = k / T
  const double* f13;    // f^(1/3)
  const double* fm13;   // f^(-1/3)
  const double* lnf3;   // ln(f)/3
  const double* fm76;   // f^(-7/6)
  const double* fm56;   // f^(-5/6) = f^(-7/6 + 1/3)
  const double* fm12;   // f^(-1/2) = f^(-7/6 + 2/3)
  const double* fm53;   // f^(-5/3)
  const double2* sca;   // (sin a, cos a), a = pi f L
  const double2* z;     // z = e^{-2 pi i f L}
  const double2* dg;    // [3][nb]: conj(d~_c) w_c Q n_c   (w_c = 4/(S_c T))
  const double* gg;     // [3][nb]: w_c |Q|^2 n_c^2
  const double* dd;     // [3]: <d|d>_c
  const double2* sct;   // [kSinTab]: (cos, sin)(2 pi j / kSinTab), the sincos table
  const float4* sctw;   // [kSinTab]: the same as double words (cos hi, cos lo, sin hi, sin lo)
  // mixed-precision path: per-bin double words of f, a = pi f L, a/(2 pi), sin a, cos a
  const float2* fw;
  const float2* aw;
  const float2* atw;
  const float2* saw;
  const float2* caw;
  const float2* f13w;   // f^(1/3) and f^(-7/6) as double words
  const float2* fm76w;
  const float4* zw;     // z as (re hi, re lo, im hi, im lo)
  const float4* dgw;    // [3][nb]: dg / dg_scale as (re hi, re lo, im hi, im lo)
  const float2* ggw;    // [3][nb]: gg / gg_scale
  double dg_scale, gg_scale;   // powers of two near max|dg|, max gg (keep the double words in range)
  // FP32 copies for the precision study (PE_PREC_FP32): f, f^(1/3), f^(-1/3), ln f/3, f^(-7/6),
  // (sin a, cos a), z, dg / dg_scale [3][nb], gg / gg_scale [3][nb]
  const float* ff;
  const float* f13f;
  const float* fm13f;
  const float* lnf3f;
  const float* fm76f;
  const float2* scaf;
  const float2* zf;
  const float2* dgf;
  const float* ggf;
  float rate_tf, alpha0_tf, geo_rate_tf, Rf, Lf;   // orbit constants and arm in FP32
  // spacecraft offsets as linear forms: delta_i[j] = sum_m Mo[i][j][m] b_m + Mo[i][j][4] over the
  // orbit basis b = (cos 2alpha, sin 2alpha, cos alpha, sin alpha) (heliocentric) or
  // (cos phi_0, sin phi_0, 0, 0) (geocentric, constant term 0)
  double Mo[3][3][5];
  float Mof[3][3][5];   // the same in FP32 (the mixed surrogate's node geometry)
  float2 Rw;            // R as a double word
  float2 ratew, alpha0w, geo_ratew;   // rate_t, alpha0_t, geo_rate_t as double words
  float tfw_max;        // |t_f| below which the mixed unit forms t_f and the orbit angles in double words
  // Q = TDI factor(z) (-i a) e^{-i a}; n_A = 1/sqrt2, n_E = 1/sqrt6, n_T = 1/sqrt3
};

struct DetSet {
  DetDev d[kMaxDet];
  int ndet;
};

}  // namespace pe
