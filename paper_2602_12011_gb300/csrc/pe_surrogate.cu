// pe_surrogate.cu -- the learned waveform surrogate: an MLP
// 11 -> 256 -> 256 -> 256 -> 2560 on BF16 tensor cores (pe_mlp.cu) predicts, per mode, a phase
// residual and an amplitude ratio at 256 log-spaced frequency nodes; at those nodes the full
// response is evaluated in FP64 and spline-interpolated onto the grid (the sparse-node idea the
// paper cites for lisabeta, Sec. 1), feeding the same A/E/T weighted sums.
//
// Per mode m, nodes f_j = f_min exp(j h), j = 0..255, from f_min = 1e-4 Hz to the taper end
// m F_isco(M) (detector independent). Targets come from the plain generator at the nodes:
//   phase residual r_j = (m/2) [Psi_PN(v_j) - Psi_PN^{<=2.5PN}(v_j)]  (the 3PN and 3.5PN terms;
//                        the series through 2.5PN, spins included, is evaluated exactly at the nodes)
//   amplitude ratio a_j = |H_lm(x_j)|  (to the Newtonian power law (2 pi M^2/D) sqrt(eta/3m) x^-7/4)
// At each node: t_f from the analytic derivative of the baseline plus the node-differenced
// residual, the orbit at t_f, the six links and TDI give the transfer functions T_X, T_Y, T_Z per
// unit mode amplitude, scaled by a_j, and the mode phase phi_nl (turns, centre Doppler included,
// -f t_c excluded). Per bin: natural-knot-free (not-a-knot) cubic splines in u = ln f of these 7
// quantities, H = A_N(f) w(f) e^{2 pi i (phi_nl - frac(f t_c))}, X' += H T_X ... The taper w and
// frac(f t_c) stay exact per bin. Samples outside the training box take the plain path.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <random>
#include <string>
#include <type_traits>
#include <vector>

#include "pe_device.cuh"
#include "pe_device_mixed.cuh"
#include "pe_kernels.h"
#include "pe_mlp.h"
#include "pe_plan.h"
#include "pe_surrogate.h"
#include "pe_fault.h"

namespace pe {

constexpr int kNodes = 256;
constexpr int kNout = kNModes * 2 * kNodes;   // [mode][kind][node], kind 0 phase residual, 1 amplitude ratio
constexpr int kNin = 64;                      // 11 features, zero padded
constexpr int kHid = 256;
constexpr int kQ = 7;                         // spline quantities per (detector, sample, mode)
constexpr int kNodeTab = 2 + 8;               // double2 entries of k_node_h's table per (sample, mode)
constexpr double kFmin = 1e-4;                // lowest node frequency [Hz]
constexpr double kLnFmin = -9.210340371976182;  // ln(kFmin), the nodes' origin in u = ln f
constexpr float kLnFminHi = static_cast<float>(kLnFmin);   // as a double word
constexpr float kLnFminLo = static_cast<float>(kLnFmin - static_cast<double>(kLnFminHi));
constexpr float kFminHi = static_cast<float>(kFmin);       // kFmin as a double word
constexpr float kFminLo = static_cast<float>(kFmin - static_cast<double>(kFminHi));
constexpr double kInv2Pi = 0.5 / kPi;                      // 1/(2 pi) as a double word
constexpr float kInv2PiHi = static_cast<float>(kInv2Pi);
constexpr float kInv2PiLo = static_cast<float>(kInv2Pi - static_cast<double>(kInv2PiHi));

// ---- features, targets ------------------------------------------------------------------------
// Normalised inputs: the 11 parameters, each affinely scaled to order one (log10 for the mass).
__global__ void k_features(const double* theta, int B, int Bpad, __nv_bfloat16* X) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= Bpad) return;
  float f[kNin];
  for (int i = 0; i < kNin; ++i) f[i] = 0.f;
  if (s < B) {
    const double* t = theta + (size_t)s * PE_NPARAM;
    f[0] = (float)((log10(fmax(t[0], 1.0)) - 6.5) / 0.5);
    f[1] = (float)((t[1] - 5.5) / 2.6);
    f[2] = (float)(t[2] / 0.57);
    f[3] = (float)(t[3] / 0.57);
    f[4] = (float)((t[4] - 25.5) / 14.1);
    f[5] = (float)(t[5] - 1.5708);
    f[6] = (float)((t[6] - 3.1416) / 1.81);
    f[7] = (float)((t[7] - 3.1416) / 1.81);
    f[8] = (float)(t[8] / 0.9);
    f[9] = (float)((t[9] - 1.5708) / 0.91);
    f[10] = (float)((t[10] - 3.4e6) / 1.2e6);
  }
  for (int i = 0; i < kNin; ++i) X[(size_t)s * kNin + i] = __float2bfloat16_rn(f[i]);
}

// node frequency of mode m for a sample with mass M [s]: f_j = f_min exp(j h)
__device__ __forceinline__ double node_h(double M, int m) {
  const double fend = m / (pow(6.0, 1.5) * 2.0 * kPi * M);
  return log(fend / kFmin) / (kNodes - 1);
}

__device__ __forceinline__ double hmag_of(int md, double q) {
  const double eta = q / ((1.0 + q) * (1.0 + q)), delta = (q - 1.0) / (q + 1.0);
  if (md == 0) return 1.0;
  if (md == 1) return delta / 3.0;
  if (md == 2) return 0.75 * sqrt(15.0 / 14.0) * delta;
  if (md == 3) return sqrt(5.0 / 7.0) / 3.0 * (1.0 - 3.0 * eta);
  return 8.0 / 9.0 * sqrt(5.0 / 7.0) * (1.0 - 3.0 * eta);
}

// Per-sample coefficients of the plain generator and of its analytic baseline.
__global__ void k_sur_prep(const double* theta, int B, unsigned mask, SampleCoef* S, SampleCoef* S0) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= B) return;
  const double* t = theta + (size_t)s * PE_NPARAM;
  SampleCoef a;
  sample_prep(t, mask, a);
  S[s] = a;
  // baseline: the same phase series truncated after 2.5PN (the 3PN and 3.5PN terms, with the
  // 3PN logarithm, are what the network learns)
  SampleCoef b = a;
  b.P[6] = b.Pd[6] = b.Pdd[6] = 0.0;
  b.P[7] = b.Pd[7] = b.Pdd[7] = 0.0;
  b.Q6 = 0.0;
  b.Pdw[6] = b.Pdw[7] = b.Pw[6] = b.Pw[7] = b.Q6w = make_float2(0.f, 0.f);
  // the surrogate's per-bin amplitude is the Newtonian power law (2 pi M^2/D) sqrt(eta/3m) x^-7/4;
  // the mode factor |H_lm| travels with the transfer functions, so store amp / |H_lm| here
  for (int md = 0; md < kNModes; ++md) {
    const double hm = hmag_of(md, t[1]);
    b.md[md].amp = (hm != 0.0) ? a.md[md].amp / hm : 0.0;
  }
  S0[s] = b;
}

__device__ __forceinline__ double psi_of(const SampleCoef& S, double v, double lnv, double* dv_out,
                                         double iv = 0.0) {
  if (iv == 0.0) iv = 1.0 / v;   // the caller may pass 1/v
  double iv5 = iv * iv;
  iv5 = iv5 * iv5 * iv;
  double poly = S.P[7], dpol = 2.0 * S.P[7];
#pragma unroll
  for (int k = 6; k >= 0; --k) {
    poly = fma(poly, v, S.P[k]);
    dpol = fma(dpol, v, (k - 5) * S.P[k]);
  }
  if (dv_out) *dv_out = fma(iv5, dpol, fma(S.Q6 * v, 1.0 + lnv, S.Q5));
  return fma(iv5, poly, lnv * fma(S.Q6, v, S.Q5));
}

// Plain-generator node values (raw): out[s][(md*2 + kind)*kNodes + j], for the samples whose mass
// ratio exceeds q_above (all of them for q_above < 1; the others' rows are left as they are).
__global__ void k_targets(const double* theta, int B, const SampleCoef* S, const SampleCoef* S0, float* out,
                          double q_above) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)B * kNModes * kNodes) return;
  const int j = (int)(i % kNodes);
  const int md = (int)((i / kNodes) % kNModes);
  const int s = (int)(i / ((long long)kNodes * kNModes));
  const double* t = theta + (size_t)s * PE_NPARAM;
  if (!(t[1] > q_above)) return;
  const int mm = (md == 0) ? 2 : (md == 1) ? 1 : (md == 2) ? 3 : (md == 3) ? 2 : 4;
  const double M = t[0] * kMsunS;
  const double f = kFmin * exp(j * node_h(M, mm));
  const double v = cbrt(2.0 * kPi * M * f / mm);
  const double lnv = log(v);
  const double r = 0.5 * mm * (psi_of(S[s], v, lnv, nullptr) - psi_of(S0[s], v, lnv, nullptr));
  const int p = S[s].md[md].p;
  const double a = hmag_of(md, t[1]) * (p >= 1 ? v : 1.0) * (p >= 2 ? v : 1.0);
  out[(size_t)s * kNout + (md * 2 + 0) * kNodes + j] = (float)r;
  out[(size_t)s * kNout + (md * 2 + 1) * kNodes + j] = (float)a;
}

// column mean/std over n rows (fixed order, FP64)
__global__ void k_colstats(const float* T, long long n, float* mean, float* stdv) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= kNout) return;
  double s = 0.0, s2 = 0.0;
  for (long long r = 0; r < n; ++r) {
    const double x = T[r * kNout + c];
    s += x;
    s2 += x * x;
  }
  const double mu = s / n;
  const double var = fmax(s2 / n - mu * mu, 0.0);
  const double sd = sqrt(var);
  mean[c] = (float)mu;
  stdv[c] = (float)(sd > 1e-6 * (fabs(mu) + 1e-30) && sd > 1e-30 ? sd : 1.0);
}

// The phase outputs of one mode share one scale (the largest per-node std of that mode), so the
// standardised loss weighs phase errors in radians, as the mismatch does; amplitude ratios keep
// their per-node scale.
__global__ void k_group_phase_scale(float* stdv) {
  const int md = threadIdx.x;
  if (md >= kNModes) return;
  float mx = 0.f;
  for (int j = 0; j < kNodes; ++j) mx = fmaxf(mx, stdv[(md * 2) * kNodes + j]);
  for (int j = 0; j < kNodes; ++j) stdv[(md * 2) * kNodes + j] = mx > 0.f ? mx : 1.f;
}

__global__ void k_standardize(float* T, long long n, const float* mean, const float* stdv) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n * kNout) return;
  const int c = (int)(i % kNout);
  T[i] = (T[i] - mean[c]) / stdv[c];
}

// Minibatch rows of the step ctr[0]: rows idx_all[ctr[0] b + r], r < b.
__global__ void k_gather_rows(const __nv_bfloat16* X, const float* T, const int* idx_all, const int* ctr, int b,
                              __nv_bfloat16* Xb, float* Tb) {
  const int* idx = idx_all + (size_t)ctr[0] * b;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < (long long)b * kNin) {
    const int r = (int)(i / kNin), c = (int)(i % kNin);
    Xb[i] = X[(size_t)idx[r] * kNin + c];
  }
  if (i < (long long)b * kNout) {
    const int r = (int)(i / kNout), c = (int)(i % kNout);
    Tb[i] = T[(size_t)idx[r] * kNout + c];
  }
}

// ---- node response and splines ---------------------------------------------------------------
__device__ __forceinline__ bool in_box(const double* t, const SurBox& bx) {
  return t[0] >= bx.mlo && t[0] <= bx.mhi && t[1] <= bx.qmax && fabs(t[2]) <= bx.chimax && fabs(t[3]) <= bx.chimax;
}

// Whether a (sample, detector) pair takes the node-spline path: the sample is in the training box
// and the detector's orbit is heliocentric. A geocentric orbit (TianQin: a turn in 3.65 days)
// turns the response ~85 times per unit of ln f where t_f runs months before coalescence, ~2.5
// turns per node interval of the 256 log-spaced nodes, which no spline on those nodes carries;
// such a detector's bins take the plain path (its share of log L is then exact).
__device__ __forceinline__ bool sur_pair(const double* t, const SurBox& bx, int orbit) {
  return orbit == 0 && in_box(t, bx);
}

// FP32 link transfer functions of one node (the mixed path): T_X, T_Y, T_Z per unit mode amplitude,
// the same algebra as below with every quantity a float. The transfer functions are O(1) sums of
// O(1) link terms (the TDI factor, which vanishes at low frequency, is in the data tables), so
// FP32 leaves them ~1e-7 relative -- what their FP32 spline coefficients keep anyway.
// c, s: cos, sin of the orbit angle (heliocentric basis) or of the geocentric phase.
__device__ __forceinline__ void node_links_f32(const DetDev& D, const SampleCoef& Sa, const ModeCoef& C, float ff,
                                               float c, float s, float2 T[3]) {
  float b[4];
  if (D.orbit == 0) {
    b[0] = c * c - s * s;
    b[1] = 2.f * s * c;
    b[2] = c;
    b[3] = s;
  } else {
    b[0] = c;
    b[1] = s;
    b[2] = b[3] = 0.f;
  }
  float dl[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      dl[i][j] = fmaf(D.Mof[i][j][0], b[0], fmaf(D.Mof[i][j][1], b[1], fmaf(D.Mof[i][j][2], b[2],
                      fmaf(D.Mof[i][j][3], b[3], D.Mof[i][j][4]))));
  const float k[3] = {Sa.kw[0].x, Sa.kw[1].x, Sa.kw[2].x};
  float p[3], qv[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    p[i] = trunc_to_float(__double_as_longlong(Sa.p[i]));
    qv[i] = trunc_to_float(__double_as_longlong(Sa.q[i]));
  }
  const float Pp = C.Ppw.x, Pc = C.Pcw.x;
  float sa, ca;
  sincospif(ff * D.Lf, &sa, &ca);   // a = pi f L
  const float2 z = make_float2(ca * ca - sa * sa, -2.f * sa * ca);   // e^{-2 i a}
  const float a = 3.14159265f * ff * D.Lf;
  float2 G[3], U[3], V[3];
#pragma unroll
  for (int l = 0; l < 3; ++l) {
    const int rr = l, ss = (l + 1) % 3, tt = (l + 2) % 3;
    float n0 = dl[rr][0] - dl[ss][0], n1 = dl[rr][1] - dl[ss][1], n2 = dl[rr][2] - dl[ss][2];
    const float inv = rsqrtf(n0 * n0 + n1 * n1 + n2 * n2);
    n0 *= inv; n1 *= inv; n2 *= inv;
    const float kn = k[0] * n0 + k[1] * n1 + k[2] * n2;
    const float np = p[0] * n0 + p[1] * n1 + p[2] * n2;
    const float nq = qv[0] * n0 + qv[1] * n1 + qv[2] * n2;
    const float gr = Pp * (np * np - nq * nq), gi = Pc * 2.f * np * nq;
    const float kd = k[0] * dl[tt][0] + k[1] * dl[tt][1] + k[2] * dl[tt][2];
    float se, ce;
    sincospif(ff * kd, &se, &ce);   // pi f k.delta_t
    G[l] = make_float2(ce * gr - se * gi, ce * gi + se * gr);
    const float u1 = a * (1.f - kn), u2 = a * (1.f + kn);
    const float sm = fabsf(u1) < 1e-3f ? fmaf(-u1 * u1, 1.f / 6.f, 1.f) : sinf(u1) / u1;
    const float sp = fabsf(u2) < 1e-3f ? fmaf(-u2 * u2, 1.f / 6.f, 1.f) : sinf(u2) / u2;
    U[l] = make_float2(fmaf(z.x, sp, sm), z.y * sp);
    V[l] = make_float2(fmaf(z.x, sm, sp), z.y * sm);
  }
  auto cm = [](float2 x, float2 y) { return make_float2(x.x * y.x - x.y * y.y, x.x * y.y + x.y * y.x); };
  auto cs = [](float2 x, float2 y) { return make_float2(x.x - y.x, x.y - y.y); };
  T[0] = cs(cm(G[2], V[2]), cm(G[0], U[0]));
  T[1] = cs(cm(G[0], V[0]), cm(G[1], U[1]));
  T[2] = cs(cm(G[1], V[1]), cm(G[2], U[2]));
}

// Per (detector I, sample s, mode md, node j): the 7 spline quantities.
// Y: de-standardised MLP outputs [Bpad][kNout]; hs, nv: the mode's node spacing h and node table
// (k_node_h); nodes out: [I][s][md][q][j]. Node j sits at f_j = kFmin e^{j h}, so
// v_j = v_0 e^{j h/3} and ln v_j = ln v_0 + j h/3, with e^{+-j h/3} a product of the table's
// e^{+-2^k h/3} over the binary digits of j (no exponential, division or log per node); the sines and cosines
// go through the library's table sincos in turns, sin(a -+ a k.n) is formed from sin a, cos a and
// one sincos of a k.n, and the pair of sincs shares one reciprocal.
// MIX: the phase, t_f, the orbit angle and the centre Doppler term stay FP64 as above; the link
// transfer functions are FP32 (node_links_f32), and quantities 1..6 are written as floats into the
// first half of their rows (k_spline's mixed path reads them so).
template <bool MIX>
__global__ void k_sur_nodes(DetSet ds, int B, const SampleCoef* S, const SampleCoef* S0, const float* Y,
                            const double* theta, SurBox bx, const double* hs, const double2* nv,
                            const float4* __restrict__ nvw, double* nodes) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long total = (long long)ds.ndet * B * kNModes * kNodes;
  if (i >= total) return;
  const int j = (int)(i % kNodes);
  const int md = (int)((i / kNodes) % kNModes);
  const int s = (int)((i / ((long long)kNodes * kNModes)) % B);
  const int I = (int)(i / ((long long)kNodes * kNModes * B));
  double* q = nodes + ((((size_t)I * B + s) * kNModes + md) * kQ) * kNodes + j;
  const SampleCoef& Sa = S[s];
  const ModeCoef& C = Sa.md[md];
  const DetDev& D = ds.d[I];
  if (!C.active || !sur_pair(theta + (size_t)s * PE_NPARAM, bx, D.orbit)) {
    for (int k = 0; k < kQ; ++k) q[k * kNodes] = 0.0;
    return;
  }
  const int mm = (md == 0) ? 2 : (md == 1) ? 1 : (md == 2) ? 3 : (md == 3) ? 2 : 4;
  const double h = hs[(size_t)s * kNModes + md];
  const double2* tab = nv + ((size_t)s * kNModes + md) * kNodeTab;
  const double2 v0 = tab[0], iv0 = tab[1];
  const float* y = Y + (size_t)s * kNout + (md * 2) * kNodes;
  if constexpr (MIX) {
    // The node phase, t_f, the orbit angle and the centre Doppler term in double words (relative
    // error ~1e-14: ~1e-9 turn at the phase's 1e5 turns, far below the spline's own error); the
    // residual's derivative in FP32 (it only corrects t_f); the link transfer functions in FP32.
    const float4* tw = nvw + ((size_t)s * kNModes + md) * kNodeTab;
    df e3 = df_make(1.f, 0.f), ie3 = e3;
#pragma unroll
    for (int k = 0; k < 8; ++k)
      if ((j >> k) & 1) {
        const float4 w = tw[2 + k];
        e3 = dfl_mul(e3, df_make(w.x, w.y));
        ie3 = dfl_mul(ie3, df_make(w.z, w.w));
      }
    const float4 t0 = tw[0], t1 = tw[1];   // (v, ln v), (1/v, h/3) at the first node
    const df f = dfl_mul(dfl_mul(dfl_mul(e3, e3), e3), df_make(kFminHi, kFminLo));
    const df invf = dfl_mulf(dfl_mul(dfl_mul(ie3, ie3), ie3), 1.0f / kFminHi);   // 1/kFmin = 1e4, exact
    const df v = dfl_mul(df_make(t0.x, t0.y), e3), iv = dfl_mul(df_make(t1.x, t1.y), ie3);
    const df lnv = dfl_add(df_make(t0.z, t0.w), dfl_mulf(df_make(t1.z, t1.w), (float)j));
    const SampleCoef& Sb = S0[s];
    df poly = Sb.Pw[7], dpol = Sb.Pdw[7];
#pragma unroll
    for (int k = 6; k >= 0; --k) {
      poly = dfl_add(dfl_mul(poly, v), Sb.Pw[k]);
      dpol = dfl_add(dfl_mul(dpol, v), Sb.Pdw[k]);
    }
    const df iv2 = dfl_mul(iv, iv);
    const df iv5 = dfl_mul(dfl_mul(iv2, iv2), iv);
    const df q5 = Sb.Q5w, q6v = dfl_mul(Sb.Q6w, v);
    const df D0 = dfl_add(dfl_mul(iv5, dpol), dfl_add(dfl_mul(q6v, dfl_add(df_make(1.f, 0.f), lnv)), q5));
    const df psi0 = dfl_add(dfl_mul(iv5, poly), dfl_mul(lnv, dfl_add(q6v, q5)));
    const float r = y[j];
    float dr;
    if (j == 0) dr = fmaf(-3.f, r, fmaf(4.f, y[1], -y[2]));
    else if (j == kNodes - 1) dr = fmaf(3.f, r, fmaf(-4.f, y[kNodes - 2], y[kNodes - 3]));
    else dr = y[j + 1] - y[j - 1];
    const float drdu = dr * (0.5f / trunc_to_float(__double_as_longlong(h)));
    const df inv2pi = df_make(kInv2PiHi, kInv2PiLo);
    const df tf = dfl_add(Sa.tcw, dfl_mul(invf, dfl_add(dfl_mul(C.tffacw, D0), dfl_mulf(inv2pi, drdu))));
    const cdf eo = df_cis_turns(dfl_add(dfl_mul(tf, D.ratew), D.alpha0w), D.sctw);
    const df kxc = dfl_mul(D.Rw, dfl_add(dfl_mul(Sa.kw[0], eo.re), dfl_mul(Sa.kw[1], eo.im)));
    const df ph = dfl_mul(dfl_add(dfl_mulf(psi0, 0.5f * mm), df_make(r, 0.f)), inv2pi);
    reinterpret_cast<df*>(q - j)[j] = dfl_sub(dfl_sub(C.ph0w, ph), dfl_mul(f, kxc));   // a double word
    float2 T[3];
    node_links_f32(D, Sa, C, f.x, eo.re.x, eo.im.x, T);   // heliocentric (geocentric nodes are skipped)
    const float ar = y[kNodes + j];
    double* row0 = q - j;   // this system's row of quantity 0
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      reinterpret_cast<float*>(row0 + (1 + 2 * c) * kNodes)[j] = T[c].x * ar;
      reinterpret_cast<float*>(row0 + (2 + 2 * c) * kNodes)[j] = T[c].y * ar;
    }
    return;
  }
  double e3 = 1.0, ie3 = 1.0;   // e^{+-j h/3} from the binary digits of j
#pragma unroll
  for (int k = 0; k < 8; ++k)
    if ((j >> k) & 1) {
      const double2 w = tab[2 + k];
      e3 *= w.x;
      ie3 *= w.y;
    }
  const double f = kFmin * (e3 * e3 * e3);
  const double invf = (1.0 / kFmin) * (ie3 * ie3 * ie3);
  const double v = v0.x * e3;
  const double lnv = fma((double)j, iv0.y, v0.y);
  double D0;
  const double psi0 = psi_of(S0[s], v, lnv, &D0, iv0.x * ie3);
  const double r = y[j];
  const double amp_ratio = y[kNodes + j];
  // residual derivative in u = ln f by node differences (one-sided at the ends)
  double drdu;
  if (j == 0) drdu = -3.0 * r + 4.0 * y[1] - y[2];
  else if (j == kNodes - 1) drdu = 3.0 * r - 4.0 * y[kNodes - 2] + y[kNodes - 3];
  else drdu = y[j + 1] - y[j - 1];
  drdu *= 0.5 / h;
  const double tf = fma(invf, fma(C.tffac, D0, drdu * (0.5 / kPi)), Sa.tc);
  double xc[3], dl[3][3];
  orbit_offsets(D, tf, xc, dl, D.sct);
  const double kxc = Sa.k[0] * xc[0] + Sa.k[1] * xc[1] + Sa.k[2] * xc[2];
  const double phi = C.ph0 - (0.5 * mm * psi0 + r) * (0.5 / kPi) - f * kxc;
  // link transfer functions per unit mode amplitude at the node frequency; a = pi f L
  const double at = 0.5 * f * D.L;   // a in turns
  double sa, ca;
  sincos_turns(at, D.sct, &sa, &ca);
  const double2 z = make_double2(ca * ca - sa * sa, -2.0 * sa * ca);   // e^{-2 i a}
  const double a = kPi * f * D.L;
  double2 G[3], U[3], V[3];
  for (int l = 0; l < 3; ++l) {
    const int rr = l, ss = (l + 1) % 3, tt = (l + 2) % 3;
    double n0 = dl[rr][0] - dl[ss][0], n1 = dl[rr][1] - dl[ss][1], n2 = dl[rr][2] - dl[ss][2];
    const double inv = rsqrt(n0 * n0 + n1 * n1 + n2 * n2);
    n0 *= inv; n1 *= inv; n2 *= inv;
    const double kn = Sa.k[0] * n0 + Sa.k[1] * n1 + Sa.k[2] * n2;
    const double np = Sa.p[0] * n0 + Sa.p[1] * n1 + Sa.p[2] * n2;
    const double nq = Sa.q[0] * n0 + Sa.q[1] * n1 + Sa.q[2] * n2;
    const double2 gam = make_double2(C.Pp * (np * np - nq * nq), C.Pc * 2.0 * np * nq);
    const double kd = Sa.k[0] * dl[tt][0] + Sa.k[1] * dl[tt][1] + Sa.k[2] * dl[tt][2];
    double se, ce;
    sincos_turns(0.5 * f * kd, D.sct, &se, &ce);   // pi f k.delta_t
    G[l] = cmul(make_double2(ce, se), gam);
    const double u1 = a * (1.0 - kn), u2 = a * (1.0 + kn);
    double sk, ck;
    sincos_turns(at * kn, D.sct, &sk, &ck);        // a k.n
    const double s1 = fma(sa, ck, -(ca * sk)), s2 = fma(sa, ck, ca * sk);
    const bool small1 = fabs(u1) < 1e-3, small2 = fabs(u2) < 1e-3;
    double sm, spl;
    if (!small1 && !small2) {
      const double ru = 1.0 / (u1 * u2);
      sm = s1 * u2 * ru;
      spl = s2 * u1 * ru;
    } else {
      sm = small1 ? sinc_small(u1) : s1 / u1;
      spl = small2 ? sinc_small(u2) : s2 / u2;
    }
    U[l] = make_double2(fma(z.x, spl, sm), z.y * spl);
    V[l] = make_double2(fma(z.x, sm, spl), z.y * sm);
  }
  const double2 TX = csub(cmul(G[2], V[2]), cmul(G[0], U[0]));
  const double2 TY = csub(cmul(G[0], V[0]), cmul(G[1], U[1]));
  const double2 TZ = csub(cmul(G[1], V[1]), cmul(G[2], U[2]));
  q[0 * kNodes] = phi;
  q[1 * kNodes] = TX.x * amp_ratio;
  q[2 * kNodes] = TX.y * amp_ratio;
  q[3 * kNodes] = TY.x * amp_ratio;
  q[4 * kNodes] = TY.y * amp_ratio;
  q[5 * kNodes] = TZ.x * amp_ratio;
  q[6 * kNodes] = TZ.y * amp_ratio;
}

// Not-a-knot cubic spline on the uniform nodes u_j = u_0 + j h of one quantity; writes, per
// interval j, (a, b, c, d) of y(u_j + t) = a + b t + c t^2 + d t^3 over coef[j][4].
// With uniform spacing the not-a-knot conditions give M_1 = r_1/6, M_{N-2} = r_{N-2}/6
// (r_j = 6 (y_{j+1} - 2 y_j + y_{j-1})/h^2); the interior (1, 4, 1) system j = 2 .. N-3 is solved
// by the Thomas algorithm, whose pivots c'_j = 1/(4 - c'_{j-1}), c'_2 = 1/4, are the same for every
// system (a compile-time table). Both sweeps are first-order affine recurrences,
// d'_j = c'_j (r_j - d'_{j-1}) and M_j = d'_j - c'_j M_{j+1}, so one warp solves a system: each lane
// composes the maps of 8 consecutive rows, a shuffle scan composes the lanes' maps, and each lane
// then runs its rows from its prefix (|c'_j| <= 1/4 + ..., ~0.27, so the composed maps only shrink).
// coef_t: FP32 copies of quantities 1..6 (the transfer functions), [system][6][kNodes - 1][4].
struct ThomasPivots {
  double c[kNodes];
};
constexpr ThomasPivots thomas_pivots() {
  ThomasPivots t{};
  double prev = 0.0;
  for (int j = 2; j <= kNodes - 3; ++j) {
    t.c[j] = 1.0 / (4.0 - prev);
    prev = t.c[j];
  }
  return t;
}
__constant__ ThomasPivots kThomas = thomas_pivots();

constexpr int kSplineWarps = 4;   // systems per CTA, one warp each
constexpr int kSplineNP = kNodes + kNodes / 8;   // padded length of the shared arrays
// shared arrays are indexed through pad(j) = j + j/8: in the sweeps lane L reads rows 8L + k, and
// the padding spreads the 32 lanes' rows over distinct banks
__device__ __forceinline__ int spad(int j) { return j + (j >> 3); }

// The second derivatives M_j of one system, by one warp, in arithmetic R (double, or float for the
// FP32 transfer-function splines of the mixed path): yy the node values and piv the pivots
// (padded, shared), M the result (padded, shared).
template <class R>
__device__ __forceinline__ void spline_solve_warp(const R* yy, const R* piv, R* M, R ih2, int lane) {
  constexpr int N = kNodes, lo = 2, hi = N - 3, RW = 8;   // RW rows per lane: 32 x 8 >= hi - lo + 1
  const R M1 = ih2 * (yy[spad(2)] - R(2) * yy[spad(1)] + yy[spad(0)]) / R(6);
  const R MN2 = ih2 * (yy[spad(N - 1)] - R(2) * yy[spad(N - 2)] + yy[spad(N - 3)]) / R(6);
  // forward sweep: this lane's rows j0 .. j0 + RW - 1 (rows beyond hi are identity maps)
  const int j0 = lo + RW * lane;
  R rr[RW];
  R A = R(1), Bc = R(0);   // composed map d -> A d + Bc of this lane's rows
#pragma unroll
  for (int k = 0; k < RW; ++k) {
    const int j = j0 + k;
    if (j <= hi) {
      R r = ih2 * (yy[spad(j + 1)] - R(2) * yy[spad(j)] + yy[spad(j - 1)]);
      if (j == lo) r -= M1;
      if (j == hi) r -= MN2;
      rr[k] = r;
      const R c = piv[spad(j)];
      A = -c * A;
      Bc = c * (r - Bc);
    }
  }
  // inclusive scan of the maps over the lanes (lane L after lanes < L), then the input of this
  // lane's first row is the composition of the lanes before it applied to d'_{lo-1} = 0
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const R Ap = __shfl_up_sync(0xffffffffu, A, off), Bp = __shfl_up_sync(0xffffffffu, Bc, off);
    if (lane >= off) {
      Bc = fma(A, Bp, Bc);
      A = A * Ap;
    }
  }
  R d = __shfl_up_sync(0xffffffffu, Bc, 1);
  if (lane == 0) d = R(0);
  R dd[RW];
#pragma unroll
  for (int k = 0; k < RW; ++k) {
    const int j = j0 + k;
    if (j <= hi) d = (rr[k] - d) * piv[spad(j)];
    dd[k] = d;
  }
  // back substitution M_j = d'_j - c'_j M_{j+1} from M_{hi+1} = 0: this lane's rows top down,
  // composed over the lanes above it
  A = R(1);
  Bc = R(0);
#pragma unroll
  for (int k = RW - 1; k >= 0; --k) {
    const int j = j0 + k;
    if (j <= hi) {
      const R c = piv[spad(j)];
      Bc = fma(-c, Bc, dd[k]);
      A = -c * A;
    }
  }
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const R Ap = __shfl_down_sync(0xffffffffu, A, off), Bp = __shfl_down_sync(0xffffffffu, Bc, off);
    if (lane + off < 32) {
      Bc = fma(A, Bp, Bc);
      A = A * Ap;
    }
  }
  R m = __shfl_down_sync(0xffffffffu, Bc, 1);
  if (lane == 31) m = R(0);
#pragma unroll
  for (int k = RW - 1; k >= 0; --k) {
    const int j = j0 + k;
    if (j <= hi) {
      m = fma(-piv[spad(j)], m, dd[k]);
      M[spad(j)] = m;
    }
  }
  __syncwarp();
  if (lane == 0) {
    M[spad(1)] = M1;
    M[spad(N - 2)] = MN2;
    M[spad(0)] = R(2) * M1 - M[spad(2)];
    M[spad(N - 1)] = R(2) * MN2 - M[spad(N - 3)];
  }
  __syncwarp();
}

// spline_solve_warp in double words (the mixed path's phase spline): yy the node values, piv the
// pivots as double words, M the result (padded, shared); k6 = 1/h^2. The same sweeps and scans,
// every operation an unnormalised double-word one (~1e-14 relative: ~1e-9 turn at 1e5 turns).
__device__ __forceinline__ df shfl_up_dw(df x, int off) {
  return df_make(__shfl_up_sync(0xffffffffu, x.x, off), __shfl_up_sync(0xffffffffu, x.y, off));
}
__device__ __forceinline__ df shfl_down_dw(df x, int off) {
  return df_make(__shfl_down_sync(0xffffffffu, x.x, off), __shfl_down_sync(0xffffffffu, x.y, off));
}
__device__ __forceinline__ df second_diff_dw(const df* yy, int j) {
  return dfl_add(dfl_sub(yy[spad(j + 1)], df_scale2(yy[spad(j)], 2.f)), yy[spad(j - 1)]);
}
__device__ __forceinline__ void spline_solve_warp_dw(const df* yy, const df* piv, df* M, df k6, int lane) {
  constexpr int N = kNodes, lo = 2, hi = N - 3, RW = 8;
  const df zero = df_make(0.f, 0.f), one = df_make(1.f, 0.f);
  const df M1 = dfl_mul(k6, second_diff_dw(yy, 1));
  const df MN2 = dfl_mul(k6, second_diff_dw(yy, N - 2));
  const int j0 = lo + RW * lane;
  df rr[RW];
  df A = one, Bc = zero;
#pragma unroll
  for (int k = 0; k < RW; ++k) {
    const int j = j0 + k;
    if (j <= hi) {
      df r = dfl_mulf(dfl_mul(k6, second_diff_dw(yy, j)), 6.f);
      if (j == lo) r = dfl_sub(r, M1);
      if (j == hi) r = dfl_sub(r, MN2);
      rr[k] = r;
      const df c = piv[spad(j)];
      A = df_neg(dfl_mul(c, A));
      Bc = dfl_mul(c, dfl_sub(r, Bc));
    }
  }
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const df Ap = shfl_up_dw(A, off), Bp = shfl_up_dw(Bc, off);
    if (lane >= off) {
      Bc = dfl_add(dfl_mul(A, Bp), Bc);
      A = dfl_mul(A, Ap);
    }
  }
  df d = shfl_up_dw(Bc, 1);
  if (lane == 0) d = zero;
  df dd[RW];
#pragma unroll
  for (int k = 0; k < RW; ++k) {
    const int j = j0 + k;
    if (j <= hi) d = dfl_mul(dfl_sub(rr[k], d), piv[spad(j)]);
    dd[k] = d;
  }
  A = one;
  Bc = zero;
#pragma unroll
  for (int k = RW - 1; k >= 0; --k) {
    const int j = j0 + k;
    if (j <= hi) {
      const df c = piv[spad(j)];
      Bc = dfl_sub(dd[k], dfl_mul(c, Bc));
      A = df_neg(dfl_mul(c, A));
    }
  }
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const df Ap = shfl_down_dw(A, off), Bp = shfl_down_dw(Bc, off);
    if (lane + off < 32) {
      Bc = dfl_add(dfl_mul(A, Bp), Bc);
      A = dfl_mul(A, Ap);
    }
  }
  df m = shfl_down_dw(Bc, 1);
  if (lane == 31) m = zero;
#pragma unroll
  for (int k = RW - 1; k >= 0; --k) {
    const int j = j0 + k;
    if (j <= hi) {
      m = dfl_sub(dd[k], dfl_mul(piv[spad(j)], m));
      M[spad(j)] = m;
    }
  }
  __syncwarp();
  if (lane == 0) {
    M[spad(1)] = M1;
    M[spad(N - 2)] = MN2;
    M[spad(0)] = dfl_sub(df_scale2(M1, 2.f), M[spad(2)]);
    M[spad(N - 1)] = dfl_sub(df_scale2(MN2, 2.f), M[spad(N - 3)]);
  }
  __syncwarp();
}

// mixed: the phase (quantity 0, double-word node values from k_sur_nodes<true>) is solved in double
// words and written as (c0, c1) and (c2, c3), two float4 per interval in the same 32 bytes (the
// mixed-precision unit's form), and the transfer functions (quantities 1..6, used only through
// their FP32 copies) are solved in FP32 and written to coef_t alone.
__global__ void __launch_bounds__(32 * kSplineWarps) k_spline(const double* nodes, long long nsys, const double* hs,
                                                               double* coef, float* coef_t, int mixed) {
  constexpr int N = kNodes;
  __shared__ double ys[kSplineWarps][kSplineNP], Ms[kSplineWarps][kSplineNP];
  __shared__ double piv[kSplineNP];   // the pivots in shared memory: the lanes read different rows at once
  __shared__ float pivf[kSplineNP];
  __shared__ float2 pivw[kSplineNP];
  for (int j = threadIdx.x; j < N; j += blockDim.x) {
    piv[spad(j)] = kThomas.c[j];
    pivf[spad(j)] = (float)kThomas.c[j];
    pivw[spad(j)] = to_dw(kThomas.c[j]);
  }
  __syncthreads();
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long i = (long long)blockIdx.x * kSplineWarps + w;
  if (i >= nsys) return;                                  // whole warps leave together
  const double* y = nodes + i * N;
  double* cf = coef + i * (N - 1) * 4;
  const int q = (int)(i % kQ);
  float* ct = q > 0 ? coef_t + ((i / kQ) * (kQ - 1) + (q - 1)) * (N - 1) * 4 : nullptr;
  const double h = hs[i / kQ];
  if (!(h > 0.0)) {
    for (int j = lane; j < 4 * (N - 1); j += 32) {
      if (!(mixed && q > 0)) cf[j] = 0.0;
      if (ct) ct[j] = 0.f;
    }
    return;
  }
  if (mixed && q > 0) {
    float* yy = reinterpret_cast<float*>(ys[w]);
    float* M = reinterpret_cast<float*>(Ms[w]);
    const float* yf = reinterpret_cast<const float*>(y);   // k_sur_nodes<true> wrote floats
    for (int j = lane; j < N; j += 32) yy[spad(j)] = yf[j];
    __syncwarp();
    const float hf = (float)h;
    spline_solve_warp<float>(yy, pivf, M, 6.f / (hf * hf), lane);
    const float ih = 1.f / hf, h6 = hf * (1.f / 6.f), ih6 = ih * (1.f / 6.f);
    for (int j = lane; j < N - 1; j += 32) {
      const float y0 = yy[spad(j)], y1 = yy[spad(j + 1)], m0 = M[spad(j)], m1 = M[spad(j + 1)];
      *reinterpret_cast<float4*>(ct + 4 * j) =
          make_float4(y0, (y1 - y0) * ih - h6 * (2.f * m0 + m1), 0.5f * m0, (m1 - m0) * ih6);
    }
    return;
  }
  if (mixed) {   // the phase, as double words (k_sur_nodes<true> wrote them), no FP64 arithmetic
    df* yy = reinterpret_cast<df*>(ys[w]);
    df* M = reinterpret_cast<df*>(Ms[w]);
    const df* yw = reinterpret_cast<const df*>(y);
    for (int j = lane; j < N; j += 32) yy[spad(j)] = yw[j];
    __syncwarp();
    const df hw = to_dw(h), ihw = to_dw(1.0 / h);
    spline_solve_warp_dw(yy, pivw, M, dfl_mul(ihw, ihw), lane);
    const df h6 = dfl_mulf(hw, 1.f / 6.f), ih6 = dfl_mulf(ihw, 1.f / 6.f);
    for (int j = lane; j < N - 1; j += 32) {
      const df y0 = yy[spad(j)], y1 = yy[spad(j + 1)], m0 = M[spad(j)], m1 = M[spad(j + 1)];
      const df c1 = dfl_sub(dfl_mul(dfl_sub(y1, y0), ihw), dfl_mul(h6, dfl_add(df_scale2(m0, 2.f), m1)));
      const df c2 = df_scale2(m0, 0.5f);
      const df c3 = dfl_mul(dfl_sub(m1, m0), ih6);
      float4* cw = reinterpret_cast<float4*>(cf + 4 * j);
      cw[0] = make_float4(y0.x, y0.y, c1.x, c1.y);
      cw[1] = make_float4(c2.x, c2.y, c3.x, c3.y);
    }
    return;
  }
  double* yy = ys[w];
  double* M = Ms[w];
  for (int j = lane; j < N; j += 32) yy[spad(j)] = y[j];
  __syncwarp();
  spline_solve_warp<double>(yy, piv, M, 6.0 / (h * h), lane);
  const double ih = 1.0 / h, h6 = h * (1.0 / 6.0), ih6 = ih * (1.0 / 6.0);
  for (int j = lane; j < N - 1; j += 32) {
    const double y0 = yy[spad(j)], y1 = yy[spad(j + 1)], m0 = M[spad(j)], m1 = M[spad(j + 1)];
    const double c0 = y0;
    const double c1 = (y1 - y0) * ih - h6 * (2.0 * m0 + m1);
    const double c2 = 0.5 * m0;
    const double c3 = (m1 - m0) * ih6;
    *reinterpret_cast<double4*>(cf + 4 * j) = make_double4(c0, c1, c2, c3);
    if (ct) *reinterpret_cast<float4*>(ct + 4 * j) = make_float4((float)c0, (float)c1, (float)c2, (float)c3);
  }
}

// Per (sample, mode): the node spacing h in ln f, and the node table of k_sur_nodes: (v, ln v) and
// (1/v, h/3) at the first node f = kFmin, then e^{+-2^k h/3} for k = 0..7 (each from exp, so a
// node's product of at most 8 of them is within ~8 ulp of e^{+-j h/3}).
__global__ void k_node_h(const double* theta, int B, double* hs, double2* nv, float4* nvw) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B * kNModes) return;
  const int s = i / kNModes, md = i % kNModes;
  const int mm = (md == 0) ? 2 : (md == 1) ? 1 : (md == 2) ? 3 : (md == 3) ? 2 : 4;
  const double M = theta[(size_t)s * PE_NPARAM] * kMsunS;
  const double h = node_h(M, mm);
  hs[i] = h;
  const double v = cbrt(2.0 * kPi * M * kFmin / mm);
  double2* t = nv + (size_t)i * kNodeTab;
  t[0] = make_double2(v, log(v));
  t[1] = make_double2(1.0 / v, h * (1.0 / 3.0));
  for (int k = 0; k < 8; ++k) {
    const double x = (double)(1 << k) * h * (1.0 / 3.0);
    t[2 + k] = make_double2(exp(x), exp(-x));
  }
  // the same entries as double words (hi, lo of .x, hi, lo of .y) for the mixed node kernel
  float4* tw = nvw + (size_t)i * kNodeTab;
  for (int k = 0; k < kNodeTab; ++k) {
    const float2 a = to_dw(t[k].x), b = to_dw(t[k].y);
    tw[k] = make_float4(a.x, a.y, b.x, b.y);
  }
}

// Spline evaluation of one mode at one bin: adds hsc H T_X, hsc H T_Y, hsc H T_Z to acc. The phase
// spline (cf, quantity 0; ~1e5 turns) is evaluated in FP64; the transfer functions T (cft, FP32
// copies of quantities 1..6, smooth and of order one relative to their own scale) and their
// products with H in FP32, with H carried times the sample's power of two hsc.
// h, ih: the mode's node spacing in ln f and its inverse (formed once per tile).
__device__ __forceinline__ void mode_bin_sur(const ModeCoef& C, double ampN, double hsc, const BinIn& B, double u,
                                             const double* cf, const float* cft, double h, double ih, float2 acc[3],
                                             const double2* __restrict__ tab) {
  const double uj = (u - kLnFmin) * ih;
  int j = (int)floor(uj);
  j = j < 0 ? 0 : (j > kNodes - 2 ? kNodes - 2 : j);
  const double t = (uj - j) * h;
  const double* c0 = cf + (size_t)j * 4;
  const double ph = fma(fma(fma(c0[3], t, c0[2]), t, c0[1]), t, c0[0]);
  const float tf = (float)t;
  float val[kQ - 1];
#pragma unroll
  for (int k = 0; k < kQ - 1; ++k) {
    const float4 c = *reinterpret_cast<const float4*>(cft + ((size_t)k * (kNodes - 1) + j) * 4);
    val[k] = fmaf(fmaf(fmaf(c.w, tf, c.z), tf, c.y), tf, c.x);
  }
  double w = 1.0;
  if (B.f > C.ftap) {
    const double span = C.fend - C.ftap;
    const double zt = span / (C.fend - B.f) - span / (B.f - C.ftap);
    w = (zt > 700.0) ? 0.0 : 1.0 / (1.0 + exp(zt));
  }
  double sph, cph;
  sincos_turns(ph - B.frc, tab, &sph, &cph);
  const double amp = ampN * hsc * B.fm76 * w;  // Newtonian power law; the mode factor |H_lm| is in T
  const float hr = (float)(amp * cph), hi = (float)(amp * sph);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    acc[c].x = fmaf(hr, val[2 * c], fmaf(-hi, val[2 * c + 1], acc[c].x));
    acc[c].y = fmaf(hr, val[2 * c + 1], fmaf(hi, val[2 * c], acc[c].y));
  }
}

// mode_bin_sur on the FP32 pipe. The phase spline (up to ~1e5 turns) is evaluated in double words
// from its double-word coefficients (k_spline with phase_dw), at t = u0 - j h in double words
// (relative error ~1e-14, ~1e-9 turn at the largest phases), minus frac(f t_c); the result is
// reduced exactly to a fraction of a turn in [-1/2, 1/2] (hi - rint(hi), exact in FP32, plus lo),
// and sin, cos of 2 pi r come from CUDA's sincospif, ~1 ulp of 1 -- the accuracy of the FP32
// transfer functions they multiply. The segment j is located in FP32: a bin within rounding of a
// node may take the neighbouring segment, whose cubic agrees there to the spline's C2 continuity.
// The amplitude is FP32: ampf = a_lm hsc (per tile), fm76 = f^(-7/6) (the high word of its
// double-word table), and the taper weight 1/(1 + e^z) where f > ftap, with the distances to the
// taper's ends taken in FP64 (exact) and z, e^z in FP32 (relative error ~1e-6 of the weight).
// u0w = ln f - ln kFmin and frcw = frac(f t_c) as double words (per bin); hw, ihf: the mode's node
// spacing as a double word and 1/h in FP32 (per tile).
__device__ __forceinline__ void mode_bin_sur_mix(const ModeCoef& C, float ampf, double f, float fm76, df u0w,
                                                 df frcw, const double* cf, const float* cft, df hw, float ihf,
                                                 float2 acc[3]) {
  int j = (int)floorf(u0w.x * ihf);
  j = j < 0 ? 0 : (j > kNodes - 2 ? kNodes - 2 : j);
  const df t = dfl_sub(u0w, dfl_mulf(hw, (float)j));
  const float4* cw = reinterpret_cast<const float4*>(cf) + 2 * j;
  const float4 c01 = cw[0], c23 = cw[1];
  df ph = dfl_add(df_make(c23.x, c23.y), dfl_mul(df_make(c23.z, c23.w), t));
  ph = dfl_add(df_make(c01.z, c01.w), dfl_mul(ph, t));
  ph = dfl_sub(dfl_add(df_make(c01.x, c01.y), dfl_mul(ph, t)), frcw);
  const float rr = __fadd_rn(__fsub_rn(ph.x, rintf(ph.x)), ph.y);
  const float tf = t.x;
  float val[kQ - 1];
#pragma unroll
  for (int k = 0; k < kQ - 1; ++k) {
    const float4 c = *reinterpret_cast<const float4*>(cft + ((size_t)k * (kNodes - 1) + j) * 4);
    val[k] = fmaf(fmaf(fmaf(c.w, tf, c.z), tf, c.y), tf, c.x);
  }
  float amp = ampf * fm76;
  if (dlt_pos(C.ftap, f)) {
    const float span = trunc_to_float(__double_as_longlong(C.fend - C.ftap));
    const float zt = __fdividef(span, trunc_to_float(__double_as_longlong(C.fend - f))) -
                     __fdividef(span, trunc_to_float(__double_as_longlong(f - C.ftap)));
    amp = (zt > 80.f) ? 0.f : amp / (1.f + __expf(zt));
  }
  float sph, cph;
  sincospif(2.0f * rr, &sph, &cph);
  const float hr = amp * cph, hi = amp * sph;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    acc[c].x = fmaf(hr, val[2 * c], fmaf(-hi, val[2 * c + 1], acc[c].x));
    acc[c].y = fmaf(hr, val[2 * c + 1], fmaf(hi, val[2 * c], acc[c].y));
  }
}

// The pair p with off[p] <= t < off[p + 1] (the last such p where pairs are empty), searched in
// [lo, P): a CTA's tiles only move forward, so it passes the pair of its previous tile.
__device__ __forceinline__ int find_pair_s(const long long* off, int P, long long t, int lo = 0) {
  if (off[lo + 1] > t) return lo;   // still in the previous tile's pair (or its empty successors' place)
  int hi = P;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (off[mid] <= t) lo = mid; else hi = mid;
  }
  return lo;
}

// Persistent kernel over the same tile list as the FP64 k_loglike_fwd (kTileBins bins per tile,
// one bin per thread, the same order of the sums), FP64 unit. mode 0: surrogate path (in-box
// samples on heliocentric detectors) or plain path (the others), partials [tile][6] as the plain
// kernel; mode 1: mismatch sums of the surrogate against the plain signal, partials [tile][6] =
// (<s|p>, <s|s>, <p|p>, 0, 0, 0). The mixed-precision variant is k_sur_inbox (in-box tiles) plus
// k_loglike_fwd itself (the other tiles).
constexpr int kSurInboxCtas = 8;    // resident CTAs per SM asked of the in-box kernel (k_sur_inbox)
// consecutive tiles (bins per thread) k_sur_inbox takes at a time; measured on 1024 in-box samples,
// whole call: 1 tile 1.16 ms, 2 tiles 1.29 ms (64 registers, 8 CTAs per SM), 1.45 ms (6 CTAs per SM)
constexpr int kSurInboxBins = 1;
__global__ void __launch_bounds__(kTileBins, 3) k_sur_fwd(DetSet ds, int B, const SampleCoef* __restrict__ coef,
                                                        const SampleCoef* __restrict__ coefN,
                                                        const double* __restrict__ theta, SurBox bx,
                                                        const double* __restrict__ spl, const float* __restrict__ splt,
                                                        const double* __restrict__ hs,
                                                        const int* __restrict__ nend, const long long* __restrict__ off,
                                                        double* part, int mode) {
  __shared__ double red[6][kTileBins + kRedPad];   // block_sum6 staging
  __shared__ double pc[kProj];
  __shared__ double ihs[kNModes];
  __shared__ double2 stab[kSinTab];
  for (int i = threadIdx.x; i < kSinTab; i += blockDim.x) stab[i] = ds.d[0].sct[i];
  __syncthreads();
  const int P = ds.ndet * B;
  const long long total = off[P];
  int p = 0;
  for (long long t = blockIdx.x; t < total; t += gridDim.x) {
    p = find_pair_s(off, P, t, p);
    const int I = p / B, s = p - I * B;
    const bool sur = sur_pair(theta + (size_t)s * PE_NPARAM, bx, ds.d[I].orbit);
    const int b0 = int(t - off[p]) * kTileBins + threadIdx.x;
    const int ne = nend[p];
    const DetDev& D = ds.d[I];
    const SampleCoef& S = coef[s];
    proj_prologue(D, S, pc);
    if (threadIdx.x < kNModes) ihs[threadIdx.x] = 1.0 / hs[(size_t)s * kNModes + threadIdx.x];
    __syncthreads();
    {
      double v[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
#pragma unroll 1
      for (int b = b0; b < b0 + kTileBins && b < ne; b += kTileBins) {
        BinIn Bn;
        load_bin(D, b, S.tc, Bn);
        float2 xs[3] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
        XYZAcc xpa;
        xyz_zero(xpa);
        const double u = 3.0 * Bn.lnf3;
        if (sur) {
#pragma unroll 1
          for (int md = 0; md < kNModes; ++md) {
            const ModeCoef& C = S.md[md];
            if (!C.active || !(Bn.f < C.fend)) continue;
            const size_t sys = ((size_t)I * B + s) * kNModes + md;
            mode_bin_sur(C, coefN[s].md[md].amp, S.hsc, Bn, u, spl + sys * kQ * (kNodes - 1) * 4,
                         splt + sys * (kQ - 1) * (kNodes - 1) * 4, hs[(size_t)s * kNModes + md], ihs[md], xs, stab);
          }
        }
        if (!sur || mode == 1) bin_modes(D, S, Bn, xpa, stab, pc);   // the plain path, as k_loglike_fwd
        double2 xp[3], xsd[3];
        xyz_final(xpa, Bn.z, xp);
#pragma unroll
        for (int c = 0; c < 3; ++c) xsd[c] = make_double2((double)xs[c].x * S.ihsc, (double)xs[c].y * S.ihsc);
        double2 os[3], op[3];
        aet_from_xyz(sur ? xsd : xp, os);
        if (mode == 0) {
          accum_bin(D, b, os, v);
        } else {
          aet_from_xyz(xp, op);
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            const double w = D.gg[c * D.nb + b];
            v[0] += w * (os[c].x * op[c].x + os[c].y * op[c].y);
            v[1] += w * (os[c].x * os[c].x + os[c].y * os[c].y);
            v[2] += w * (op[c].x * op[c].x + op[c].y * op[c].y);
          }
        }
      }
      double a;
      if (block_sum6(v, [](double x, double y) { return x + y; }, red, &a)) part[t * 6 + threadIdx.x] = a;
    }
  }
}

// The mixed-precision surrogate's in-box tiles (mode 0): mode_bin_sur_mix per (mode, bin), A/E/T
// and the weighted products in double words, each 128-bin tile summed in double words (the tail of
// k_loglike_fwd's mixed path) and scaled back to FP64 into its own partial. A CTA walks a contiguous
// run of the in-box tile list (offk), so that consecutive tiles of a pair reuse its spline
// coefficients from L1, and takes NB consecutive tiles of one pair at a time: each thread then
// carries NB independent bins through one mode loop (their coefficient loads and arithmetic
// overlap), and each tile still gets its own partial in the same fixed order.
// block_sum6's fixed-order sum of six double words per thread with two barriers instead of
// three: consecutive tiles alternate between two staging buffers, so a tile's writes cannot meet
// the previous tile's final readers (those finish before the next tile's first barrier, and the
// buffer they read is written again only a tile later).
__device__ __forceinline__ bool tile_sum6(const df v[6], float2 (*red)[kTileBins + kRedPad], df* out) {
#pragma unroll
  for (int i = 0; i < 6; ++i) red[i][threadIdx.x] = v[i];
  __syncthreads();
  if (threadIdx.x < 6 * 16) {
    const int i = threadIdx.x >> 4, g = threadIdx.x & 15;
    df s = red[i][g];
#pragma unroll
    for (int k = 1; k < kTileBins / 16; ++k) s = dfl_add(s, red[i][g + 16 * k]);
    red[i][g] = s;
  }
  __syncthreads();
  if (threadIdx.x >= 6) return false;
  df s = red[threadIdx.x][0];
#pragma unroll
  for (int g = 1; g < 16; ++g) s = dfl_add(s, red[threadIdx.x][g]);
  *out = s;
  return true;
}

template <int NB>
__global__ void __launch_bounds__(kTileBins, kSurInboxCtas) k_sur_inbox(DetSet ds, int B,
                                                                     const SampleCoef* __restrict__ coef,
                                                                     const SampleCoef* __restrict__ coefN,
                                                                     const double* __restrict__ spl,
                                                                     const float* __restrict__ splt,
                                                                     const double* __restrict__ hs,
                                                                     const int* __restrict__ nend,
                                                                     const long long* __restrict__ off,
                                                                     const long long* __restrict__ offk, double* part) {
  __shared__ float2 red[2][6][kTileBins + kRedPad];   // tile sums' staging, alternating per tile
  __shared__ float ampf[kNModes];                  // a_lm hsc in FP32
  __shared__ float2 hsw[kNModes];                  // node spacing h as a double word
  __shared__ float ihsf[kNModes];                  // 1/h in FP32
  const int P = ds.ndet * B;
  const long long total = offk[P];
  const long long chunk = (total + gridDim.x - 1) / gridDim.x;
  const long long tk0 = blockIdx.x * chunk;
  const long long tk1 = tk0 + chunk < total ? tk0 + chunk : total;
  int p = 0, pcur = -1, buf = 0;
  for (long long tk = tk0; tk < tk1;) {
    p = find_pair_s(offk, P, tk, p);
    const long long tend = offk[p + 1] < tk1 ? offk[p + 1] : tk1;   // this pair's tiles in the run
    const int nt = (NB == 2 && tk + 1 < tend) ? 2 : 1;                // uniform over the CTA
    const int I = p / B, s = p - I * B;
    const int ne = nend[p];
    const DetDev& D = ds.d[I];
    const SampleCoef& S = coef[s];
    if (p != pcur) {     // the pair's per-sample values, staged once per run of its tiles
      __syncthreads();   // the previous pair's readers are done
      if (threadIdx.x < kNModes) {
        const double hm = hs[(size_t)s * kNModes + threadIdx.x];
        ampf[threadIdx.x] = (float)(coefN[s].md[threadIdx.x].amp * S.hsc);
        hsw[threadIdx.x] = to_dw(hm);
        ihsf[threadIdx.x] = (float)(1.0 / hm);
      }
      __syncthreads();
      pcur = p;
    }
    // per bin in double words, no FP64 arithmetic: u0 = 3 (ln f / 3) - ln kFmin, and frac(f t_c)
    // from the double-word product (relative error ~2^-46: ~1e-8 turn at f t_c ~ 4e5 turns)
    int bb[NB];
    double f[NB];
    df u0w[NB], frcw[NB];
    float fm76[NB];
    float2 xs[NB][3];
#pragma unroll
    for (int k = 0; k < NB; ++k) {
      bb[k] = int(tk - offk[p] + k) * kTileBins + threadIdx.x;
      const int b = (k < nt && bb[k] < ne) ? bb[k] : 0;
      f[k] = (k < nt && bb[k] < ne) ? D.f[b] : 0.0;   // 0 keeps an absent bin out of every mode
      u0w[k] = dfl_sub(dfl_mulf(df_from_bits(D.lnf3[b]), 3.f), df_make(kLnFminHi, kLnFminLo));
      fm76[k] = D.fm76w[b].x;
      const df ftc = dfl_mul(D.fw[b], S.tcw);
      frcw[k] = two_sum(__fsub_rn(ftc.x, rintf(ftc.x)), ftc.y);
#pragma unroll
      for (int c = 0; c < 3; ++c) xs[k][c] = make_float2(0.f, 0.f);
    }
#pragma unroll   // the modes' (and the bins') coefficient loads overlap
    for (int md = 0; md < kNModes; ++md) {
      const ModeCoef& C = S.md[md];
      if (!C.active) continue;
      const size_t sys = ((size_t)I * B + s) * kNModes + md;
#pragma unroll
      for (int k = 0; k < NB; ++k)
        if (dlt_pos(0.0, f[k]) && dlt_pos(f[k], C.fend))
          mode_bin_sur_mix(C, ampf[md], f[k], fm76[k], u0w[k], frcw[k], spl + sys * kQ * (kNodes - 1) * 4,
                           splt + sys * (kQ - 1) * (kNodes - 1) * 4, hsw[md], ihsf[md], xs[k]);
    }
    const double ih = S.ihsc;
#pragma unroll
    for (int k = 0; k < NB; ++k) {
      if (k >= nt) break;   // uniform
      df v[6];
#pragma unroll
      for (int i = 0; i < 6; ++i) v[i] = df_make(0.f, 0.f);
      const int b = bb[k];
      if (b < ne) {
        cdf x[3], o[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) x[c] = cdf{df_make(xs[k][c].x, 0.f), df_make(xs[k][c].y, 0.f)};
        aet_from_xyz_dw(x, o);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const float4 g = D.dgw[c * D.nb + b];
          v[c] = df_sub_s(df_mul(df_make(g.x, g.y), o[c].re), df_mul(df_make(g.z, g.w), o[c].im));
          const df m2 = df_add_s(df_mul(o[c].re, o[c].re), df_mul(o[c].im, o[c].im));
          v[3 + c] = df_mul(D.ggw[c * D.nb + b], m2);
        }
      }
      df r;
      if (tile_sum6(v, red[buf], &r))
        part[(off[p] + (tk - offk[p]) + k) * 6 + threadIdx.x] =
            df_to(r) * (threadIdx.x < 3 ? D.dg_scale * ih : D.gg_scale * ih * ih);
      buf ^= 1;
    }
    tk += nt;
  }
}

__global__ void k_mismatch_reduce(int ndet, int B, const long long* off, const double* part, const SampleCoef* coef,
                                  double* mm) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= B) return;
  double a = 0.0, b = 0.0, c = 0.0;
  for (int I = 0; I < ndet; ++I) {
    const int p = I * B + s;
    for (long long t = off[p]; t < off[p + 1]; ++t) {
      a += part[t * 6 + 0];
      b += part[t * 6 + 1];
      c += part[t * 6 + 2];
    }
  }
  mm[s] = (coef[s].valid && b > 0.0 && c > 0.0) ? 1.0 - a / sqrt(b * c) : NAN;
}

// Tile counts of the in-box pairs (nin) and of the others (nout), from the pairs' active bins.
__global__ void k_split_nend(const double* theta, int ndet, int B, SurBox bx, unsigned geo_mask, const int* nend,
                             int* nin, int* nout) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= ndet * B) return;
  const bool sur = sur_pair(theta + (size_t)(p % B) * PE_NPARAM, bx, (geo_mask >> (p / B)) & 1u);
  nin[p] = sur ? nend[p] : 0;
  nout[p] = sur ? 0 : nend[p];
}

// used[s] = 1 where the sample took the node-spline path on at least one (heliocentric) detector.
__global__ void k_used(const double* theta, int B, SurBox bx, int any_helio, const SampleCoef* coef, int32_t* used) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < B) used[s] = (any_helio && coef[s].valid && in_box(theta + (size_t)s * PE_NPARAM, bx)) ? 1 : 0;
}

__global__ void k_destd(const float* Y, int B, const float* mean, const float* stdv, float* out) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)B * kNout) return;
  const int c = (int)(i % kNout);
  out[i] = Y[i] * stdv[c] + mean[c];
}

}  // namespace pe

// =============================================================================================
// Host side
// =============================================================================================
namespace {

using bf16 = __nv_bfloat16;

struct Layer {
  int in = 0, out = 0;
  float *W = nullptr, *b = nullptr, *mW = nullptr, *vW = nullptr, *mb = nullptr, *vb = nullptr, *gW = nullptr,
        *gb = nullptr;
  bf16 *Wb = nullptr, *WTb = nullptr;
};

template <class T>
cudaError_t dalloc(T** p, size_t n) {
  return pe::dmalloc(reinterpret_cast<void**>(p), n * sizeof(T) + 16);
}

}  // namespace

struct pe_surrogate_s {
  Layer L[4];
  float* mean = nullptr;
  float* stdv = nullptr;
  pe::SurBox box{1e5, 1e7, 10.0, 0.99, 8.0};
  int node_source = 0;   // 0: the network; 1: the plain generator at the nodes (no network)
  int trained = 0;
  int adam_t = 0;
  uint64_t seed = 0;
  std::vector<void*> owned;
  // batch work buffers
  int cap = 0;
  bf16 *X = nullptr, *H[3] = {nullptr, nullptr, nullptr}, *HT[3] = {nullptr, nullptr, nullptr}, *XT = nullptr;
  bf16 *dY = nullptr, *dYT = nullptr, *dZ = nullptr, *dZT = nullptr;
  float *Z[3] = {nullptr, nullptr, nullptr}, *Y = nullptr, *dYf = nullptr, *dH = nullptr, *dZf = nullptr, *Tb = nullptr;
  double* part = nullptr;
};

namespace {

pe_status sfail(pe_status st, const char* msg) { return pe::set_error(st, msg); }

// Status of the tensor-core GEMMs launched since the last check (their barrier waits are bounded
// and record a code instead of hanging).
pe_status gemm_status(const char* who) {
  const int code = pe::umma_take_error();
  if (code == 0) return PE_OK;
  char msg[160];
  snprintf(msg, sizeof(msg), "%s: tensor-core GEMM barrier wait timed out (code %d)", who, code);
  return sfail(PE_ECUDA, msg);
}


void free_batch(pe_surrogate_s* s) {
  void* ptrs[] = {s->X, s->H[0], s->H[1], s->H[2], s->HT[0], s->HT[1], s->HT[2], s->XT, s->dY, s->dYT, s->dZ,
                  s->dZT, s->Z[0], s->Z[1], s->Z[2], s->Y, s->dYf, s->dH, s->dZf, s->Tb, s->part};
  for (void* p : ptrs)
    if (p) pe::dfree(p);
  s->X = s->XT = s->dY = s->dYT = s->dZ = s->dZT = nullptr;
  for (int i = 0; i < 3; ++i) { s->H[i] = s->HT[i] = nullptr; s->Z[i] = nullptr; }
  s->Y = s->dYf = s->dH = s->dZf = s->Tb = nullptr;
  s->part = nullptr;
  s->cap = 0;
}

cudaError_t ensure_batch(pe_surrogate_s* s, int cap) {
  if (cap <= s->cap) return cudaSuccess;
  free_batch(s);
  cudaError_t e = cudaSuccess;
  const size_t c = (size_t)cap;
  if (e == cudaSuccess) e = dalloc(&s->X, c * pe::kNin);
  if (e == cudaSuccess) e = dalloc(&s->XT, c * pe::kNin);
  for (int i = 0; i < 3 && e == cudaSuccess; ++i) {
    e = dalloc(&s->H[i], c * pe::kHid);
    if (e == cudaSuccess) e = dalloc(&s->HT[i], c * pe::kHid);
    if (e == cudaSuccess) e = dalloc(&s->Z[i], c * pe::kHid);
  }
  if (e == cudaSuccess) e = dalloc(&s->Y, c * pe::kNout);
  if (e == cudaSuccess) e = dalloc(&s->Tb, c * pe::kNout);
  if (e == cudaSuccess) e = dalloc(&s->dYf, c * pe::kNout);
  if (e == cudaSuccess) e = dalloc(&s->dY, c * pe::kNout);
  if (e == cudaSuccess) e = dalloc(&s->dYT, c * pe::kNout);
  if (e == cudaSuccess) e = dalloc(&s->dH, c * pe::kHid);
  if (e == cudaSuccess) e = dalloc(&s->dZ, c * pe::kHid);
  if (e == cudaSuccess) e = dalloc(&s->dZT, c * pe::kHid);
  if (e == cudaSuccess) e = dalloc(&s->dZf, c * pe::kHid);
  if (e == cudaSuccess) e = dalloc(&s->part, (c * pe::kNout + 255) / 256 + 1);
  if (e == cudaSuccess) s->cap = cap;
  return e;
}

// refresh the bf16 copies (and transposed copies) of every weight matrix
cudaError_t refresh_bf16(pe_surrogate_s* s, cudaStream_t st) {
  for (int l = 0; l < 4; ++l) {
    Layer& L = s->L[l];
    cudaError_t e = pe::f32_to_bf16(L.W, L.Wb, (size_t)L.out * L.in, st);
    if (e == cudaSuccess) e = pe::transpose_bf16(L.Wb, L.WTb, L.out, L.in, st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// forward of Bp rows (Bp % 64 == 0) from s->X; output Y (standardised) in s->Y
cudaError_t mlp_forward(pe_surrogate_s* s, int Bp, cudaStream_t st) {
  cudaError_t e = pe::gemm_tn(s->X, s->L[0].Wb, s->Z[0], Bp, pe::kHid, pe::kNin, 1, s->L[0].b, s->H[0], st);
  if (e == cudaSuccess) e = pe::gemm_tn(s->H[0], s->L[1].Wb, s->Z[1], Bp, pe::kHid, pe::kHid, 1, s->L[1].b, s->H[1], st);
  if (e == cudaSuccess) e = pe::gemm_tn(s->H[1], s->L[2].Wb, s->Z[2], Bp, pe::kHid, pe::kHid, 1, s->L[2].b, s->H[2], st);
  if (e == cudaSuccess) e = pe::gemm_tn(s->H[2], s->L[3].Wb, s->Y, Bp, pe::kNout, pe::kHid, 2, s->L[3].b, nullptr, st);
  return e;
}

// Host copy of the intermediates of one forward + backward pass (the elementwise checks of the
// dense layers): fp32 buffers as they are, bf16 buffers widened to fp32.
struct MlpTrace {
  float* host = nullptr;
  size_t off = 0;
  cudaError_t err = cudaSuccess;
  void f32(const float* dev, size_t n) {
    if (err == cudaSuccess) err = cudaMemcpy(host + off, dev, n * sizeof(float), cudaMemcpyDeviceToHost);
    off += n;
  }
  void b16(const bf16* dev, size_t n) {
    std::vector<uint16_t> tmp(n);
    if (err == cudaSuccess) err = cudaMemcpy(tmp.data(), dev, n * sizeof(uint16_t), cudaMemcpyDeviceToHost);
    for (size_t i = 0; i < n && err == cudaSuccess; ++i) {
      const uint32_t bits = (uint32_t)tmp[i] << 16;
      std::memcpy(host + off + i, &bits, sizeof(float));
    }
    off += n;
  }
};

// backward from dY (bf16 + fp32 in s->dY, s->dYf) into every layer's gW, gb; with a trace, each
// layer's incoming cotangent dH and its dZ (fp32 and bf16) are copied out as they are formed
cudaError_t mlp_backward(pe_surrogate_s* s, int Bp, cudaStream_t st, MlpTrace* tr = nullptr) {
  cudaError_t e = pe::transpose_bf16(s->dY, s->dYT, Bp, pe::kNout, st);
  if (e == cudaSuccess) e = pe::transpose_bf16(s->H[2], s->HT[2], Bp, pe::kHid, st);
  // layer 3: gW3 [2560][256] = dY^T H2; gb3 = colsum dY; dH2 = dY W3
  if (e == cudaSuccess) e = pe::gemm_tn(s->dYT, s->HT[2], s->L[3].gW, pe::kNout, pe::kHid, Bp, 0, nullptr, nullptr, st);
  if (e == cudaSuccess) e = pe::colsum(s->dYf, s->L[3].gb, Bp, pe::kNout, st);
  if (e == cudaSuccess) e = pe::gemm_tn(s->dY, s->L[3].WTb, s->dH, Bp, pe::kHid, pe::kNout, 0, nullptr, nullptr, st);
  for (int l = 2; l >= 0 && e == cudaSuccess; --l) {
    const bf16* Hin = (l == 0) ? s->X : s->H[l - 1];
    bf16* HinT = (l == 0) ? s->XT : s->HT[l - 1];
    const int nin = (l == 0) ? pe::kNin : pe::kHid;
    e = pe::silu_bwd(s->dH, s->Z[l], s->dZ, s->dZf, (size_t)Bp * pe::kHid, st);
    if (tr && e == cudaSuccess) {
      tr->f32(s->dH, (size_t)Bp * pe::kHid);
      tr->f32(s->dZf, (size_t)Bp * pe::kHid);
      tr->b16(s->dZ, (size_t)Bp * pe::kHid);
      e = tr->err;
    }
    if (e == cudaSuccess) e = pe::transpose_bf16(s->dZ, s->dZT, Bp, pe::kHid, st);
    if (e == cudaSuccess) e = pe::transpose_bf16(Hin, HinT, Bp, nin, st);
    if (e == cudaSuccess) e = pe::gemm_tn(s->dZT, HinT, s->L[l].gW, pe::kHid, nin, Bp, 0, nullptr, nullptr, st);
    if (e == cudaSuccess) e = pe::colsum(s->dZf, s->L[l].gb, Bp, pe::kHid, st);
    if (e == cudaSuccess && l > 0)
      e = pe::gemm_tn(s->dZ, s->L[l].WTb, s->dH, Bp, pe::kHid, pe::kHid, 0, nullptr, nullptr, st);
  }
  return e;
}

int pad64(int b) { return (b + 63) / 64 * 64; }

}  // namespace

extern "C" {

pe_status pe_surrogate_create(uint64_t seed, pe_surrogate* out) {
  if (out == nullptr) return sfail(PE_EINVAL, "pe_surrogate_create: out is NULL");
  *out = nullptr;
  pe_surrogate_s* s = new (std::nothrow) pe_surrogate_s();
  if (!s) return sfail(PE_ENOMEM, "pe_surrogate_create: host allocation failed");
  s->seed = seed;
  const int dims[5] = {pe::kNin, pe::kHid, pe::kHid, pe::kHid, pe::kNout};
  std::mt19937_64 rng(seed);
  cudaError_t e = cudaSuccess;
  for (int l = 0; l < 4 && e == cudaSuccess; ++l) {
    Layer& L = s->L[l];
    L.in = dims[l];
    L.out = dims[l + 1];
    const size_t nw = (size_t)L.in * L.out;
    e = dalloc(&L.W, nw);
    if (e == cudaSuccess) e = dalloc(&L.b, L.out);
    if (e == cudaSuccess) e = dalloc(&L.mW, nw);
    if (e == cudaSuccess) e = dalloc(&L.vW, nw);
    if (e == cudaSuccess) e = dalloc(&L.mb, L.out);
    if (e == cudaSuccess) e = dalloc(&L.vb, L.out);
    if (e == cudaSuccess) e = dalloc(&L.gW, nw);
    if (e == cudaSuccess) e = dalloc(&L.gb, L.out);
    if (e == cudaSuccess) e = dalloc(&L.Wb, nw);
    if (e == cudaSuccess) e = dalloc(&L.WTb, nw);
    if (e != cudaSuccess) break;
    // He-uniform initialisation (the input layer only sees its 11 used features)
    const int fan = (l == 0) ? PE_NPARAM : L.in;
    const double lim = std::sqrt(6.0 / fan) * (l == 3 ? 0.1 : 1.0);
    std::uniform_real_distribution<double> U(-lim, lim);
    std::vector<float> w(nw), z(nw, 0.f), zb(L.out, 0.f);
    for (size_t i = 0; i < nw; ++i) w[i] = (l == 0 && (int)(i % L.in) >= PE_NPARAM) ? 0.f : (float)U(rng);
    e = pe::upload(L.W, w.data(), nw * sizeof(float));
    if (e == cudaSuccess) e = pe::upload(L.mW, z.data(), nw * sizeof(float));
    if (e == cudaSuccess) e = pe::upload(L.vW, z.data(), nw * sizeof(float));
    if (e == cudaSuccess) e = pe::upload(L.b, zb.data(), L.out * sizeof(float));
    if (e == cudaSuccess) e = pe::upload(L.mb, zb.data(), L.out * sizeof(float));
    if (e == cudaSuccess) e = pe::upload(L.vb, zb.data(), L.out * sizeof(float));
  }
  if (e == cudaSuccess) e = dalloc(&s->mean, pe::kNout);
  if (e == cudaSuccess) e = dalloc(&s->stdv, pe::kNout);
  if (e == cudaSuccess) {
    std::vector<float> zero(pe::kNout, 0.f), one(pe::kNout, 1.f);
    e = pe::upload(s->mean, zero.data(), pe::kNout * sizeof(float));
    if (e == cudaSuccess) e = pe::upload(s->stdv, one.data(), pe::kNout * sizeof(float));
  }
  if (e == cudaSuccess) e = refresh_bf16(s, 0);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    cudaGetLastError();
    pe_surrogate_destroy(s);
    return sfail(PE_ENOMEM, "pe_surrogate_create: device allocation failed");
  }
  if (pe::umma_prepare() != cudaSuccess) {
    cudaGetLastError();
    pe_surrogate_destroy(s);
    return sfail(PE_ECUDA, "pe_surrogate_create: the tensor-core GEMM cannot be set up on this device");
  }
  *out = s;
  return PE_OK;
}

pe_status pe_surrogate_destroy(pe_surrogate s) {
  if (!s) return PE_OK;
  cudaDeviceSynchronize();
  free_batch(s);
  for (int l = 0; l < 4; ++l) {
    Layer& L = s->L[l];
    void* ptrs[] = {L.W, L.b, L.mW, L.vW, L.mb, L.vb, L.gW, L.gb, L.Wb, L.WTb};
    for (void* p : ptrs)
      if (p) pe::dfree(p);
  }
  if (s->mean) pe::dfree(s->mean);
  if (s->stdv) pe::dfree(s->stdv);
  cudaGetLastError();
  delete s;
  return PE_OK;
}

pe_status pe_surrogate_set_node_source(pe_surrogate s, int source) {
  if (!s || (source != 0 && source != 1)) return sfail(PE_EINVAL, "pe_surrogate_set_node_source: bad arguments");
  s->node_source = source;
  return PE_OK;
}

pe_status pe_surrogate_set_box(pe_surrogate s, double mtot_lo, double mtot_hi, double q_max, double chi_max) {
  if (!s) return sfail(PE_EINVAL, "pe_surrogate_set_box: NULL handle");
  if (!(mtot_lo > 0.0 && mtot_hi >= mtot_lo && q_max >= 1.0 && chi_max >= 0.0 && chi_max < 1.0))
    return sfail(PE_EINVAL, "pe_surrogate_set_box: bad box");
  s->box = pe::SurBox{mtot_lo, mtot_hi, q_max, chi_max, s->box.qnet};
  return PE_OK;
}

pe_status pe_surrogate_set_network_qmax(pe_surrogate s, double q_net) {
  if (!s || !(q_net >= 1.0)) return sfail(PE_EINVAL, "pe_surrogate_set_network_qmax: bad arguments");
  s->box.qnet = q_net;
  return PE_OK;
}

pe_status pe_surrogate_targets(const double* theta_dev, int B, float* out_dev) {
  if (!theta_dev || !out_dev || B < 1) return sfail(PE_EINVAL, "pe_surrogate_targets: bad arguments");
  pe::SampleCoef *S = nullptr, *S0 = nullptr;
  cudaError_t e = dalloc(&S, B);
  if (e == cudaSuccess) e = dalloc(&S0, B);
  if (e == cudaSuccess) {
    pe::k_sur_prep<<<(B + 63) / 64, 64>>>(theta_dev, B, PE_MODE_ALL, S, S0);
    const long long n = (long long)B * pe::kNModes * pe::kNodes;
    pe::k_targets<<<(unsigned)((n + 255) / 256), 256>>>(theta_dev, B, S, S0, out_dev, 0.0);
    e = pe::launch_status();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
  }
  if (S) pe::dfree(S);
  if (S0) pe::dfree(S0);
  if (e != cudaSuccess) { cudaGetLastError(); return sfail(PE_ECUDA, "pe_surrogate_targets failed"); }
  return PE_OK;
}

pe_status pe_surrogate_train(pe_surrogate s, const double* theta_train_dev, int n_train, int epochs, int batch, double lr,
                             double* out_final_loss, float* out_loss_curve) {
  if (!s || !theta_train_dev || n_train < 64 || epochs < 1 || batch < 64 || batch % 64 || !(lr > 0.0))
    return sfail(PE_EINVAL, "pe_surrogate_train: bad arguments (n_train >= 64, batch % 64 == 0)");
  const size_t nt = (size_t)n_train;
  float* T = nullptr;
  bf16* Xall = nullptr;
  int* idx_d = nullptr;
  cudaError_t e = dalloc(&T, nt * pe::kNout);
  if (e == cudaSuccess) e = dalloc(&Xall, nt * pe::kNin);
  if (e == cudaSuccess) e = dalloc(&idx_d, nt);
  if (e == cudaSuccess) e = ensure_batch(s, batch);
  if (e != cudaSuccess) {
    cudaGetLastError();
    if (T) pe::dfree(T);
    if (Xall) pe::dfree(Xall);
    if (idx_d) pe::dfree(idx_d);
    return sfail(PE_ENOMEM, "pe_surrogate_train: allocation failed");
  }
  pe_status st = PE_OK;
  // targets from the plain generator (chunks of 32768 samples), standardised per output
  for (size_t c0 = 0; c0 < nt && st == PE_OK; c0 += 32768) {
    const int nb = (int)std::min<size_t>(32768, nt - c0);
    st = pe_surrogate_targets(theta_train_dev + c0 * PE_NPARAM, nb, T + c0 * pe::kNout);
  }
  if (st == PE_OK) {
    pe::k_colstats<<<(pe::kNout + 127) / 128, 128>>>(T, (long long)nt, s->mean, s->stdv);
    pe::k_group_phase_scale<<<1, 32>>>(s->stdv);
    const long long n = (long long)nt * pe::kNout;
    pe::k_standardize<<<(unsigned)((n + 255) / 256), 256>>>(T, (long long)nt, s->mean, s->stdv);
    pe::k_features<<<(n_train + 127) / 128, 128>>>(theta_train_dev, n_train, n_train, Xall);
    e = pe::launch_status();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) st = sfail(PE_ECUDA, "pe_surrogate_train: target preparation failed");
  }
  // One training step -- minibatch gather, forward, loss, backward, Adam, bf16 refresh, step
  // counters -- is captured once as a CUDA graph and replayed for every step: the per-epoch
  // permutation lives on the device, and the step's schedule (learning rate, Adam bias
  // corrections, minibatch offset) comes from device counters.
  std::mt19937_64 rng(s->seed ^ 0x9e3779b97f4a7c15ull);
  std::vector<int> perm(nt);
  for (size_t i = 0; i < nt; ++i) perm[i] = (int)i;
  const int steps = n_train / batch;
  const int total_steps = steps * epochs;
  const long long ng = (long long)batch * pe::kNout;
  int nblk = 0;
  int* ctr = nullptr;
  float* par = nullptr;
  cudaStream_t cs = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  if (st == PE_OK) {
    e = dalloc(&ctr, 4);
    if (e == cudaSuccess) e = dalloc(&par, 4);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    const int ctr0[4] = {0, 0, s->adam_t, 0};
    if (e == cudaSuccess) e = pe::upload(ctr, ctr0, sizeof(ctr0));
    if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaError_t c = pe::train_step_params(ctr, par, lr, total_steps, 0.9f, 0.999f, cs);
      if (c == cudaSuccess) {
        pe::k_gather_rows<<<(unsigned)((ng + 255) / 256), 256, 0, cs>>>(Xall, T, idx_d, ctr, batch, s->X, s->Tb);
        c = pe::launch_status();
      }
      if (c == cudaSuccess) c = mlp_forward(s, batch, cs);
      if (c == cudaSuccess) c = pe::mse(s->Y, s->Tb, s->dYf, s->dY, s->part, (size_t)ng, 1.0f / (float)ng, &nblk, cs);
      if (c == cudaSuccess) c = mlp_backward(s, batch, cs);
      for (int l = 0; l < 4 && c == cudaSuccess; ++l) {
        Layer& L = s->L[l];
        c = pe::adam(L.W, L.gW, L.mW, L.vW, (size_t)L.in * L.out, par, 0.9f, 0.999f, 1e-8f, cs);
        if (c == cudaSuccess) c = pe::adam(L.b, L.gb, L.mb, L.vb, L.out, par, 0.9f, 0.999f, 1e-8f, cs);
      }
      if (c == cudaSuccess) c = refresh_bf16(s, cs);
      if (c == cudaSuccess) c = pe::train_step_advance(ctr, cs);
      e = cudaStreamEndCapture(cs, &graph);
      if (e == cudaSuccess) e = c;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    if (e != cudaSuccess) st = sfail(PE_ECUDA, "pe_surrogate_train: capturing the training step failed");
  }
  std::vector<double> hpart;
  double last = 0.0;
  for (int ep = 0; ep < epochs && st == PE_OK; ++ep) {
    std::shuffle(perm.begin(), perm.end(), rng);
    e = pe::upload_async(idx_d, perm.data(), nt * sizeof(int), cs);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctr, 0, sizeof(int), cs);   // step within the epoch
    for (int k = 0; k < steps && e == cudaSuccess; ++k) e = cudaGraphLaunch(exec, cs);
    // loss of the epoch's last minibatch (its partial sums are left in s->part)
    hpart.resize(nblk);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hpart.data(), s->part, nblk * sizeof(double), cudaMemcpyDeviceToHost, cs);
    if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
    if (e != cudaSuccess) {
      st = sfail(PE_ECUDA, "pe_surrogate_train: training step failed");
      break;
    }
    double sum = 0.0;
    for (double x : hpart) sum += x;
    last = sum / (double)ng;
    if (out_loss_curve) out_loss_curve[ep] = (float)last;
  }
  if (st == PE_OK) s->adam_t += total_steps;
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  if (cs) cudaStreamDestroy(cs);
  if (ctr) pe::dfree(ctr);
  if (par) pe::dfree(par);
  if (st == PE_OK && cudaDeviceSynchronize() != cudaSuccess) st = sfail(PE_ECUDA, "pe_surrogate_train: training failed");
  pe::dfree(T);
  pe::dfree(Xall);
  pe::dfree(idx_d);
  if (st != PE_OK) { cudaGetLastError(); return st; }
  st = gemm_status("pe_surrogate_train");
  if (st != PE_OK) return st;
  s->trained = 1;
  if (out_final_loss) *out_final_loss = last;
  return PE_OK;
}

// De-standardised node values [B][2560] of theta (device), written to out_dev (device).
pe_status pe_surrogate_predict(pe_surrogate s, const double* theta_dev, int B, float* out_dev) {
  if (!s || !theta_dev || !out_dev || B < 1) return sfail(PE_EINVAL, "pe_surrogate_predict: bad arguments");
  const int Bp = pad64(B);
  cudaError_t e = ensure_batch(s, Bp);
  if (e == cudaSuccess) {
    pe::k_features<<<(Bp + 127) / 128, 128>>>(theta_dev, B, Bp, s->X);
    e = pe::launch_status();
  }
  if (e == cudaSuccess) e = mlp_forward(s, Bp, 0);
  if (e == cudaSuccess) {
    const long long n = (long long)B * pe::kNout;
    pe::k_destd<<<(unsigned)((n + 255) / 256), 256>>>(s->Y, B, s->mean, s->stdv, out_dev);
    e = pe::launch_status();
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) { cudaGetLastError(); return sfail(PE_ECUDA, "pe_surrogate_predict failed"); }
  return gemm_status("pe_surrogate_predict");
}

// Shared driver of the surrogate log-likelihood (mode 0) and the mismatch study (mode 1).
static pe_status sur_run(pe_surrogate s, const pe_detector* dets, int ndet, const double* theta_dev, int B,
                         unsigned mode_mask, int mode, double* out0, int32_t* used, cudaStream_t st) {
  pe::DetSet ds;
  pe_status s0 = pe::detset_from_handles(dets, ndet, &ds);
  if (s0 != PE_OK) return s0;
  if (B < 1 || B > (1 << 20) || !theta_dev || !out0) return sfail(PE_EINVAL, "surrogate: bad arguments");
  const bool mix = (mode_mask & PE_PREC_MIXED) != 0;
  if ((mode_mask & PE_MODE_ALL) == 0 || (mode_mask & ~(PE_MODE_ALL | PE_PREC_MIXED)))
    return sfail(PE_EINVAL, "surrogate: bad mode mask");
  if (mix && mode != 0) return sfail(PE_EINVAL, "surrogate: the mismatch study is FP64 only");
  mode_mask &= PE_MODE_ALL;
  const int P = ndet * B;
  long long max_tiles = 0;
  for (int i = 0; i < ndet; ++i) max_tiles += (long long)B * pe::tiles_of(ds.d[i].nb, pe::kTileBins);
  const int Bp = pad64(B);
  cudaError_t e = ensure_batch(s, Bp);
  std::vector<void*> bufs;
  auto aalloc = [&](auto** p, size_t n) {
    if (e != cudaSuccess) return;
    void* q = nullptr;
    e = pe::dmalloc_async(&q, n * sizeof(**p) + 16, st);
    if (e == cudaSuccess) { bufs.push_back(q); *p = static_cast<std::remove_pointer_t<decltype(p)>>(q); }
  };
  pe::SampleCoef *S = nullptr, *S0 = nullptr;
  int* nend = nullptr;
  long long* off = nullptr;
  double *part = nullptr, *nodes = nullptr, *spl = nullptr, *hs = nullptr, *hs_sys = nullptr;
  double2* nv = nullptr;
  float4* nvw = nullptr;
  float *Yd = nullptr, *splt = nullptr;
  const size_t nsys = (size_t)ndet * B * pe::kNModes;
  aalloc(&S, B);
  aalloc(&S0, B);
  aalloc(&nend, P);
  aalloc(&off, P + 1);
  int *nin = nullptr, *nout = nullptr;
  long long *offin = nullptr, *offout = nullptr;
  if (mix) {
    aalloc(&nin, P);
    aalloc(&nout, P);
    aalloc(&offin, P + 1);
    aalloc(&offout, P + 1);
  }
  aalloc(&part, (size_t)max_tiles * 6);
  aalloc(&nodes, nsys * pe::kQ * pe::kNodes);
  aalloc(&spl, nsys * pe::kQ * (pe::kNodes - 1) * 4);
  aalloc(&splt, nsys * (pe::kQ - 1) * (pe::kNodes - 1) * 4);
  aalloc(&hs, (size_t)B * pe::kNModes);
  aalloc(&hs_sys, nsys);
  aalloc(&nv, (size_t)B * pe::kNModes * pe::kNodeTab);
  aalloc(&nvw, (size_t)B * pe::kNModes * pe::kNodeTab);
  aalloc(&Yd, (size_t)B * pe::kNout);
  if (e == cudaSuccess) {
    // MLP inference (BF16 tensor cores) -> de-standardised node values
    pe::k_features<<<(Bp + 127) / 128, 128, 0, st>>>(theta_dev, B, Bp, s->X);
    e = pe::launch_status();
    if (e == cudaSuccess && s->node_source == 0) e = mlp_forward(s, Bp, st);
  }
  if (e == cudaSuccess) {
    const long long n = (long long)B * pe::kNout;
    pe::k_sur_prep<<<(B + 63) / 64, 64, 0, st>>>(theta_dev, B, mode_mask, S, S0);
    // node values: the network's, with the plain generator's own above the network's mass-ratio
    // bound (or everywhere for node source 1)
    const long long nt = (long long)B * pe::kNModes * pe::kNodes;
    if (s->node_source == 0) {
      pe::k_destd<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(s->Y, B, s->mean, s->stdv, Yd);
      if (s->box.qnet < s->box.qmax)
        pe::k_targets<<<(unsigned)((nt + 255) / 256), 256, 0, st>>>(theta_dev, B, S, S0, Yd, s->box.qnet);
    } else {
      pe::k_targets<<<(unsigned)((nt + 255) / 256), 256, 0, st>>>(theta_dev, B, S, S0, Yd, 0.0);
    }
    pe::k_node_h<<<(B * pe::kNModes + 127) / 128, 128, 0, st>>>(theta_dev, B, hs, nv, nvw);
    const long long nn = (long long)nsys * pe::kNodes;
    if (mix)
      pe::k_sur_nodes<true><<<(unsigned)((nn + 127) / 128), 128, 0, st>>>(ds, B, S, S0, Yd, theta_dev, s->box, hs,
                                                                          nv, nvw, nodes);
    else
      pe::k_sur_nodes<false><<<(unsigned)((nn + 127) / 128), 128, 0, st>>>(ds, B, S, S0, Yd, theta_dev, s->box, hs,
                                                                           nv, nvw, nodes);
    e = pe::launch_status();
    // the spline kernel reads the node spacing per system (I, s, md): replicate per detector
    for (int I = 0; I < ndet && e == cudaSuccess; ++I)
      e = cudaMemcpyAsync(hs_sys + (size_t)I * B * pe::kNModes, hs, (size_t)B * pe::kNModes * sizeof(double),
                          cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) {
      const long long ns = (long long)nsys * pe::kQ;
      pe::k_spline<<<(unsigned)((ns + pe::kSplineWarps - 1) / pe::kSplineWarps), 32 * pe::kSplineWarps, 0, st>>>(
          nodes, ns, hs_sys, spl, splt, mix ? 1 : 0);
      e = pe::launch_status();
    }
  }
  if (e == cudaSuccess) e = pe::launch_prep(theta_dev, B, mode_mask, ds, S, nend, nullptr, st);
  if (e == cudaSuccess) e = pe::launch_scan_tiles(nend, P, off, pe::kTileBins, st);
  pe::TuneChoice tcm = pe::default_choice(pe::kPrecMixed);
  if (mix) pe::lookup_tuned(ds, B, mode_mask | PE_PREC_MIXED, &tcm);
  if (e == cudaSuccess && mix) {
    unsigned geo_mask = 0;
    for (int I = 0; I < ndet; ++I)
      if (ds.d[I].orbit != 0) geo_mask |= 1u << I;
    pe::k_split_nend<<<(P + 127) / 128, 128, 0, st>>>(theta_dev, ndet, B, s->box, geo_mask, nend, nin, nout);
    e = pe::launch_status();
    if (e == cudaSuccess) e = pe::launch_scan_tiles(nin, P, offin, pe::kTileBins, st);
    // the fallback pairs' work items for the tuned mixed-precision forward kernel
    if (e == cudaSuccess) e = pe::launch_scan_tiles(nout, P, offout, tcm.subtiles * pe::kTileBins, st);
  }
  if (e == cudaSuccess) {
    int nsm = 1, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const long long g = std::max<long long>(1, std::min<long long>(max_tiles, (long long)nsm * 8));
    if (mix) {
      const long long g1 = std::max<long long>(1, std::min<long long>(max_tiles, (long long)nsm * pe::kSurInboxCtas));
      pe::k_sur_inbox<pe::kSurInboxBins><<<(unsigned)g1, pe::kTileBins, 0, st>>>(ds, B, S, S0, spl, splt, hs, nend,
                                                                                off, offin, part);
      e = pe::launch_status();
      // fallback tiles: the mixed-precision forward kernel of pe_loglike_batch with its tuned (or
      // default) choice, over the fallback pairs' work items; it writes each sub-tile's partial at
      // off[p] + its index, the same place as in the full list
      if (e == cudaSuccess)
        e = pe::launch_loglike_fwd_variant(tcm.variant, pe::kPrecMixed, ds, B, S, nend, off, offout, tcm.subtiles,
                                           part, pe::grid_for(tcm, max_tiles), st);
    } else {
      pe::k_sur_fwd<<<(unsigned)g, pe::kTileBins, 0, st>>>(ds, B, S, S0, theta_dev, s->box, spl, splt, hs, nend, off,
                                                           part, mode);
      e = pe::launch_status();
    }
  }
  if (e == cudaSuccess) {
    if (mode == 0) {
      e = pe::launch_reduce(ds, B, off, part, S, out0, nullptr, st);
      if (e == cudaSuccess && used) {
        int any_helio = 0;
        for (int I = 0; I < ndet; ++I) any_helio |= ds.d[I].orbit == 0 ? 1 : 0;
        pe::k_used<<<(B + 127) / 128, 128, 0, st>>>(theta_dev, B, s->box, any_helio, S, used);
        e = pe::launch_status();
      }
    } else {
      pe::k_mismatch_reduce<<<(B + 127) / 128, 128, 0, st>>>(ndet, B, off, part, S, out0);
      e = pe::launch_status();
    }
  }
  for (void* p : bufs) pe::dfree_async(p, st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    char msg[256];
    snprintf(msg, sizeof(msg), "surrogate path failed: %s", cudaGetErrorString(e));
    return sfail(PE_ECUDA, msg);
  }
  return PE_OK;
}

pe_status pe_surrogate_loglike_batch(pe_surrogate s, const pe_detector* dets, int ndet, const double* theta_dev, int B,
                                     unsigned mode_mask, double* out_logl_dev, int32_t* out_used_dev, void* stream) {
  if (!s) return sfail(PE_EINVAL, "pe_surrogate_loglike_batch: NULL handle");
  return sur_run(s, dets, ndet, theta_dev, B, mode_mask, 0, out_logl_dev, out_used_dev, static_cast<cudaStream_t>(stream));
}

pe_status pe_surrogate_mismatch(pe_surrogate s, pe_detector det, const double* theta_dev, int B, unsigned mode_mask,
                                double* out_mismatch_dev, void* stream) {
  if (!s) return sfail(PE_EINVAL, "pe_surrogate_mismatch: NULL handle");
  return sur_run(s, &det, 1, theta_dev, B, mode_mask, 1, out_mismatch_dev, nullptr, static_cast<cudaStream_t>(stream));
}

// Forward and backward of the network on given inputs and output cotangents (host arrays), for
// gradient checks: x [B][64] (fp32, rounded to bf16 on the device), dy [B][2560]; returns the raw
// (standardised-space) outputs y [B][2560] and the gradients of every layer, concatenated as
// gW0, gb0, gW1, gb1, gW2, gb2, gW3, gb3 (weights [out][in]). B must be a multiple of 64.
static pe_status mlp_debug_impl(pe_surrogate s, const float* x, int B, const float* dy, float* y, float* grads,
                                float* trace) {
  if (!s || !x || !dy || !y || !grads || B < 64 || B % 64) return sfail(PE_EINVAL, "pe_surrogate_mlp_debug: bad arguments");
  cudaError_t e = ensure_batch(s, B);
  float* tmp = nullptr;
  const size_t nx = (size_t)B * pe::kNin, ny = (size_t)B * pe::kNout, nh = (size_t)B * pe::kHid;
  MlpTrace tr;
  tr.host = trace;
  if (e == cudaSuccess) e = dalloc(&tmp, std::max(nx, ny));
  if (e == cudaSuccess) e = pe::upload(tmp, x, nx * sizeof(float));
  if (e == cudaSuccess) e = pe::f32_to_bf16(tmp, s->X, nx, 0);
  if (e == cudaSuccess) e = mlp_forward(s, B, 0);
  if (e == cudaSuccess) e = cudaMemcpy(y, s->Y, ny * sizeof(float), cudaMemcpyDeviceToHost);
  if (trace && e == cudaSuccess) {
    tr.b16(s->X, nx);
    for (int l = 0; l < 3; ++l) {
      tr.f32(s->Z[l], nh);
      tr.b16(s->H[l], nh);
    }
    tr.f32(s->Y, ny);
    e = tr.err;
  }
  if (e == cudaSuccess) e = pe::upload(s->dYf, dy, ny * sizeof(float));
  if (e == cudaSuccess) e = pe::f32_to_bf16(s->dYf, s->dY, ny, 0);
  if (e == cudaSuccess) e = mlp_backward(s, B, 0, trace ? &tr : nullptr);
  size_t o = 0;
  for (int l = 0; l < 4 && e == cudaSuccess; ++l) {
    const size_t nw = (size_t)s->L[l].in * s->L[l].out;
    e = cudaMemcpy(grads + o, s->L[l].gW, nw * sizeof(float), cudaMemcpyDeviceToHost);
    o += nw;
    if (e == cudaSuccess) e = cudaMemcpy(grads + o, s->L[l].gb, s->L[l].out * sizeof(float), cudaMemcpyDeviceToHost);
    o += s->L[l].out;
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (tmp) pe::dfree(tmp);
  if (e != cudaSuccess) { cudaGetLastError(); return sfail(PE_ECUDA, "pe_surrogate_mlp_debug failed"); }
  return gemm_status("pe_surrogate_mlp_debug");
}

pe_status pe_surrogate_mlp_debug(pe_surrogate s, const float* x, int B, const float* dy, float* y, float* grads) {
  return mlp_debug_impl(s, x, B, dy, y, grads, nullptr);
}

pe_status pe_surrogate_mlp_trace(pe_surrogate s, const float* x, int B, const float* dy, float* y, float* grads,
                                 float* trace) {
  if (!trace) return sfail(PE_EINVAL, "pe_surrogate_mlp_trace: trace is NULL");
  return mlp_debug_impl(s, x, B, dy, y, grads, trace);
}

// Weights and biases as fp32 host arrays, concatenated W0, b0, W1, b1, W2, b2, W3, b3 ([out][in]).
pe_status pe_surrogate_get_weights(pe_surrogate s, float* out, int64_t* count) {
  if (!s || !count) return sfail(PE_EINVAL, "pe_surrogate_get_weights: bad arguments");
  size_t n = 0;
  for (int l = 0; l < 4; ++l) n += (size_t)s->L[l].in * s->L[l].out + s->L[l].out;
  *count = (int64_t)n;
  if (!out) return PE_OK;
  size_t o = 0;
  for (int l = 0; l < 4; ++l) {
    const size_t nw = (size_t)s->L[l].in * s->L[l].out;
    if (cudaMemcpy(out + o, s->L[l].W, nw * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(out + o + nw, s->L[l].b, s->L[l].out * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess) {
      cudaGetLastError();
      return sfail(PE_ECUDA, "pe_surrogate_get_weights: copy failed");
    }
    o += nw + s->L[l].out;
  }
  return PE_OK;
}

// ---- checkpoint: "PESURR01" | u32 version | u32 dims[5] | SurBox | i32 adam_t | u64 seed |
//      per layer W, b, mW, vW, mb, vb (fp32) | mean, std (fp32) | u64 FNV-1a of all preceding bytes
static uint64_t fnv1a(const unsigned char* p, size_t n, uint64_t h = 1469598103934665603ull) {
  for (size_t i = 0; i < n; ++i) { h ^= p[i]; h *= 1099511628211ull; }
  return h;
}

pe_status pe_surrogate_save(pe_surrogate s, const char* path) {
  if (!s || !path) return sfail(PE_EINVAL, "pe_surrogate_save: bad arguments");
  std::vector<unsigned char> buf;
  auto put = [&](const void* p, size_t n) { buf.insert(buf.end(), (const unsigned char*)p, (const unsigned char*)p + n); };
  put("PESURR01", 8);
  const uint32_t ver = 2, dims[5] = {pe::kNin, pe::kHid, pe::kHid, pe::kHid, pe::kNout};   // 2: SurBox.qnet
  put(&ver, 4);
  put(dims, sizeof(dims));
  put(&s->box, sizeof(s->box));
  put(&s->adam_t, 4);
  put(&s->seed, 8);
  std::vector<float> h;
  auto dget = [&](const float* d, size_t n) -> bool {
    h.resize(n);
    if (cudaMemcpy(h.data(), d, n * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess) return false;
    put(h.data(), n * sizeof(float));
    return true;
  };
  bool ok = true;
  for (int l = 0; l < 4 && ok; ++l) {
    const Layer& L = s->L[l];
    const size_t nw = (size_t)L.in * L.out;
    ok = dget(L.W, nw) && dget(L.b, L.out) && dget(L.mW, nw) && dget(L.vW, nw) && dget(L.mb, L.out) && dget(L.vb, L.out);
  }
  ok = ok && dget(s->mean, pe::kNout) && dget(s->stdv, pe::kNout);
  if (!ok) { cudaGetLastError(); return sfail(PE_ECUDA, "pe_surrogate_save: device copy failed"); }
  const uint64_t cs = fnv1a(buf.data(), buf.size());
  put(&cs, 8);
  FILE* f = fopen(path, "wb");
  if (!f) return sfail(PE_EINVAL, "pe_surrogate_save: cannot open file");
  const size_t w = fwrite(buf.data(), 1, buf.size(), f);
  fclose(f);
  if (w != buf.size()) return sfail(PE_EINVAL, "pe_surrogate_save: short write");
  return PE_OK;
}

pe_status pe_surrogate_load(pe_surrogate s, const char* path) {
  if (!s || !path) return sfail(PE_EINVAL, "pe_surrogate_load: bad arguments");
  FILE* f = fopen(path, "rb");
  if (!f) return sfail(PE_EINVAL, "pe_surrogate_load: cannot open file");
  std::vector<unsigned char> buf;
  unsigned char tmp[65536];
  size_t r;
  while ((r = fread(tmp, 1, sizeof(tmp), f)) > 0) buf.insert(buf.end(), tmp, tmp + r);
  fclose(f);
  if (buf.size() < 8 + 4 + 20 + sizeof(pe::SurBox) + 12 + 8 || memcmp(buf.data(), "PESURR01", 8) != 0)
    return sfail(PE_EINVAL, "pe_surrogate_load: not a surrogate checkpoint");
  uint64_t cs;
  memcpy(&cs, buf.data() + buf.size() - 8, 8);
  if (fnv1a(buf.data(), buf.size() - 8) != cs) return sfail(PE_EINVAL, "pe_surrogate_load: checksum mismatch");
  size_t o = 8;
  uint32_t ver, dims[5];
  memcpy(&ver, buf.data() + o, 4); o += 4;
  memcpy(dims, buf.data() + o, sizeof(dims)); o += sizeof(dims);
  const uint32_t want[5] = {pe::kNin, pe::kHid, pe::kHid, pe::kHid, pe::kNout};
  if (ver != 2 || memcmp(dims, want, sizeof(dims)) != 0) return sfail(PE_EINVAL, "pe_surrogate_load: version/shape mismatch");
  memcpy(&s->box, buf.data() + o, sizeof(s->box)); o += sizeof(s->box);
  memcpy(&s->adam_t, buf.data() + o, 4); o += 4;
  memcpy(&s->seed, buf.data() + o, 8); o += 8;
  auto dput = [&](float* d, size_t n) -> bool {
    if (o + n * sizeof(float) > buf.size() - 8) return false;
    const bool ok = pe::upload(d, buf.data() + o, n * sizeof(float)) == cudaSuccess;
    o += n * sizeof(float);
    return ok;
  };
  bool ok = true;
  for (int l = 0; l < 4 && ok; ++l) {
    Layer& L = s->L[l];
    const size_t nw = (size_t)L.in * L.out;
    ok = dput(L.W, nw) && dput(L.b, L.out) && dput(L.mW, nw) && dput(L.vW, nw) && dput(L.mb, L.out) && dput(L.vb, L.out);
  }
  ok = ok && dput(s->mean, pe::kNout) && dput(s->stdv, pe::kNout);
  if (!ok || o != buf.size() - 8) { cudaGetLastError(); return sfail(PE_EINVAL, "pe_surrogate_load: truncated checkpoint"); }
  if (refresh_bf16(s, 0) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) {
    cudaGetLastError();
    return sfail(PE_ECUDA, "pe_surrogate_load: device refresh failed");
  }
  s->trained = 1;
  return PE_OK;
}

}  // extern "C"
