// pe_device_f32.cuh -- the (sample, mode, bin) unit of mode_bin (pe_device.cuh) entirely in FP32:
// the paper's low-precision option (Sec. 3.1, the float32 curves of Fig. fig_cost), kept for the
// precision study. Same definitions and the same order of operations as mode_bin (Sec. 2.1, Eq.
// eq_tf, eq_fd_resp, FD TDI); every quantity is a float, including the TaylorF2 phase (up to
// ~1e6 rad), t_f and frac(f t_c), so its error is that of FP32 arithmetic on those magnitudes.
// Amplitudes carry the sample's power of two hsc and the whitened tables their scales, as in the
// mixed path, to stay inside the FP32 range.
#pragma once
#include "pe_device.cuh"

namespace pe {

struct ModeF {
  float cm, icm, lncm, amp, ph0, mfac, tffac, Pp, Pc, fend, ftap;
  int p, active;
};
struct SampleF {
  float tc, P[8], Pd[8], Q5, Q6, k[3];
  ModeF md[kNModes];
};

// FP32 copy of one sample's coefficients (amplitudes times hsc), written by one thread.
__device__ inline void sample_to_f32(const SampleCoef& S, SampleF& F) {
  F.tc = (float)S.tc;
  for (int k = 0; k < 8; ++k) { F.P[k] = (float)S.P[k]; F.Pd[k] = (float)S.Pd[k]; }
  F.Q5 = (float)S.Q5;
  F.Q6 = (float)S.Q6;
  for (int i = 0; i < 3; ++i) F.k[i] = (float)S.k[i];
  for (int m = 0; m < kNModes; ++m) {
    const ModeCoef& C = S.md[m];
    ModeF& G = F.md[m];
    G.cm = (float)C.cm; G.icm = (float)C.icm; G.lncm = (float)C.lncm; G.amp = (float)(C.amp * S.hsc);
    G.ph0 = (float)C.ph0; G.mfac = (float)C.mfac; G.tffac = (float)C.tffac; G.Pp = (float)C.Pp; G.Pc = (float)C.Pc;
    G.fend = (float)C.fend; G.ftap = (float)C.ftap; G.p = C.p; G.active = C.active;
  }
}

// x - rint(x) for |x| < 2^22, by adding and subtracting 1.5 * 2^23 on the FP32 pipe
__device__ __forceinline__ float frac_f(float x) {
  return __fsub_rn(x, __fsub_rn(__fadd_rn(x, 12582912.0f), 12582912.0f));
}
// sin, cos of 2 pi x for x in turns: reduction to [-1/2, 1/2], then CUDA's sincospif
__device__ __forceinline__ void sc_turns_f(float x, float* s, float* c) { sincospif(2.0f * frac_f(x), s, c); }

__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

struct XYZAccF {
  float2 P[3], Q[3];
};

struct BinF {
  float f, f13, fm13, lnf3, fm76, invf, a, sa, ca, frc;
  float2 z;
};
__device__ __forceinline__ void load_bin_f32(const DetDev& D, int b, float tc, BinF& B) {
  B.f = D.ff[b];
  B.f13 = D.f13f[b];
  B.fm13 = D.fm13f[b];
  B.lnf3 = D.lnf3f[b];
  B.fm76 = D.fm76f[b];
  B.invf = B.fm13 * B.fm13 * B.fm13;
  B.a = 3.14159265f * B.f * D.Lf;
  const float2 sc = D.scaf[b];
  B.sa = sc.x;
  B.ca = sc.y;
  B.z = D.zf[b];
  const float pr = B.f * tc;
  B.frc = frac_f(pr);
}

__device__ __forceinline__ float dot5f(const volatile float* p, const float b[4]) {
  return fmaf(p[0], b[0], fmaf(p[1], b[1], fmaf(p[2], b[2], fmaf(p[3], b[3], p[4]))));
}

__device__ __forceinline__ void mode_bin_f32(const DetDev& D, const SampleF& S, const ModeF& C, const BinF& B,
                                             XYZAccF& acc, const float* __restrict__ pcf) {
  const float v = C.cm * B.f13;
  const float iv = C.icm * B.fm13;
  const float lnv = C.lncm + B.lnf3;
  float iv5 = iv * iv;
  iv5 = iv5 * iv5 * iv;
  float poly = S.P[7], dpol = 2.0f * S.P[7];
#pragma unroll
  for (int k = 6; k >= 0; --k) {
    poly = fmaf(poly, v, S.P[k]);
    dpol = fmaf(dpol, v, S.Pd[k]);
  }
  const float psi_pn = fmaf(iv5, poly, lnv * fmaf(S.Q6, v, S.Q5));
  const float dv = fmaf(iv5, dpol, fmaf(S.Q6 * v, 1.0f + lnv, S.Q5));
  const float tf = fmaf(C.tffac * B.invf, dv, S.tc);
  float w = 1.0f;
  if (B.f > C.ftap) {
    const float span = C.fend - C.ftap;
    const float zt = span / (C.fend - B.f) - span / (B.f - C.ftap);
    w = (zt > 80.0f) ? 0.0f : 1.0f / (1.0f + expf(zt));
  }
  float amp = C.amp * B.fm76 * w;
  if (C.p >= 1) amp *= v;
  if (C.p >= 2) amp *= v;
  float so, co, ob[4];
  sc_turns_f(fmaf(tf, D.rate_tf, D.alpha0_tf), &so, &co);
  if (D.orbit == 0) {
    ob[0] = co * co - so * so;
    ob[1] = 2.0f * so * co;
    ob[2] = co;
    ob[3] = so;
  } else {
    sc_turns_f(tf * D.geo_rate_tf, &ob[1], &ob[0]);
    ob[2] = 0.0f;
    ob[3] = 0.0f;
  }
  const float kxc = D.Rf * (S.k[0] * co + S.k[1] * so);
  const float ph = fmaf(-C.mfac, psi_pn, C.ph0 - B.frc) - B.f * kxc;
  float sph, cph;
  sc_turns_f(ph, &sph, &cph);
  const float2 H = make_float2(amp * cph, amp * sph);
  float2 E[3];
#pragma unroll
  for (int i = 0; i < 2; ++i) sincospif(B.f * dot5f(pcf + 45 + 5 * i, ob), &E[i].y, &E[i].x);
  {
    const float2 e01 = cmulf(E[0], E[1]);
    E[2] = make_float2(e01.x, -e01.y);
  }
  float2 G[3];
  float smv[3], spv[3];
#pragma unroll
  for (int l = 0; l < 3; ++l) {
    const int t = (l + 2) % 3;
    const float knr = dot5f(pcf + 15 * l, ob), npr = dot5f(pcf + 15 * l + 5, ob), nqr = dot5f(pcf + 15 * l + 10, ob);
    const float inv = rsqrtf(fmaf(knr, knr, fmaf(npr, npr, nqr * nqr)));
    const float kn = knr * inv, np = npr * inv, nq = nqr * inv;
    const float2 gam = make_float2(C.Pp * (np * np - nq * nq), C.Pc * 2.0f * np * nq);
    G[l] = cmulf(E[t], cmulf(gam, H));
    const float u1 = B.a * (1.0f - kn), u2 = B.a * (1.0f + kn);
    smv[l] = fabsf(u1) < 1e-3f ? 1.0f - u1 * u1 / 6.0f : sinf(u1) / u1;
    spv[l] = fabsf(u2) < 1e-3f ? 1.0f - u2 * u2 / 6.0f : sinf(u2) / u2;
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const int lp = (c + 2) % 3, lu = c;
    acc.P[c].x = fmaf(G[lp].x, spv[lp], fmaf(-G[lu].x, smv[lu], acc.P[c].x));
    acc.P[c].y = fmaf(G[lp].y, spv[lp], fmaf(-G[lu].y, smv[lu], acc.P[c].y));
    acc.Q[c].x = fmaf(G[lp].x, smv[lp], fmaf(-G[lu].x, spv[lu], acc.Q[c].x));
    acc.Q[c].y = fmaf(G[lp].y, smv[lp], fmaf(-G[lu].y, spv[lu], acc.Q[c].y));
  }
}

// A/E/T brackets (times hsc) of one sample at one bin in FP32.
__device__ __forceinline__ void bin_aet_f32(const DetDev& D, const SampleF& S, int b, float2 o[3],
                                            const float* __restrict__ pcf) {
  BinF B;
  load_bin_f32(D, b, S.tc, B);
  XYZAccF a;
#pragma unroll
  for (int i = 0; i < 3; ++i) a.P[i] = a.Q[i] = make_float2(0.f, 0.f);
#pragma unroll 1
  for (int md = 0; md < kNModes; ++md) {
    const ModeF& C = S.md[md];
    if (!C.active || !(B.f < C.fend)) continue;
    mode_bin_f32(D, S, C, B, a, pcf);
  }
  float2 x[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const float2 zq = cmulf(B.z, a.Q[i]);
    x[i] = make_float2(a.P[i].x + zq.x, a.P[i].y + zq.y);
  }
  o[0] = make_float2(x[2].x - x[0].x, x[2].y - x[0].y);
  o[1] = make_float2(x[0].x - 2.0f * x[1].x + x[2].x, x[0].y - 2.0f * x[1].y + x[2].y);
  o[2] = make_float2(x[0].x + x[1].x + x[2].x, x[0].y + x[1].y + x[2].y);
}

}  // namespace pe
