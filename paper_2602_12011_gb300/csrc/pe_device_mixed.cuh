// pe_device_mixed.cuh -- the (sample, mode, bin) unit of mode_bin (pe_device.cuh) with the
// response geometry on the FP32 pipe in double-word arithmetic (pe_df.cuh, ~1e-14 relative).
// GB300 issues FP32 at 64x its FP64 rate, so the FP64 pipe keeps only what needs FP64's range
// and 53-bit precision: the TaylorF2 phase (up to ~1e6 rad), its exact reduction to a fraction of
// a turn, t_f where it lies far (more than 2^23 s, heliocentric, or 2^21 s, geocentric) from the
// origin, and the likelihood accumulation across tiles. Everything else -- t_f and the orbit
// angles, the sines and cosines of the orbit, phase, third-spacecraft and sinc
// arguments, the projections k.n, n.e+.n, n.ex.n of the link vectors (per-tile linear forms in the
// orbit basis, converted to double words once per tile), the
// sincs, the mode tensor factors, the TDI brackets, the A/E/T combinations and the PSD-weighted
// per-bin products -- is double-word. Amplitudes enter multiplied by the sample's power of two hsc
// (near 1/amp of the (2,2) mode) and the whitened data tables divided by powers of two near their
// maxima, keeping every double word far from the FP32 overflow and underflow limits; the tile sums
// are scaled back when they are converted to FP64.
// Same definitions as mode_bin: arXiv:2602.12011 Sec. 2.1 (Eq. eq_tf, eq_fd_resp, FD TDI).
#pragma once
#include "pe_device.cuh"
#include "pe_df.cuh"

namespace pe {

// Mode-summed link products of one bin in double words (times hsc), as XYZAcc: S_l = sum G_l s+_l,
// M_l = sum G_l s-_l.
struct MixAcc {
  df Sr[3], Si[3], Mr[3], Mi[3];
};
__device__ __forceinline__ void mix_zero(MixAcc& a) {
#pragma unroll
  for (int i = 0; i < 3; ++i) a.Sr[i] = a.Si[i] = a.Mr[i] = a.Mi[i] = df_make(0.f, 0.f);
}
// X' = P + z Q with P_c = S_{c+2} - M_c, Q_c = M_{c+2} - S_c (times hsc), double words
__device__ __forceinline__ void mix_final(const MixAcc& a, const cdf& z, cdf x[3]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const int lp = (c + 2) % 3;
    const cdf q = {dfl_sub(a.Mr[lp], a.Sr[c]), dfl_sub(a.Mi[lp], a.Si[c])};
    const cdf zq = cdfl_mul(z, q);
    x[c].re = dfl_add(dfl_sub(a.Sr[lp], a.Mr[c]), zq.re);
    x[c].im = dfl_add(dfl_sub(a.Si[lp], a.Mi[c]), zq.im);
  }
}

// Per-bin double words: f, a = pi f L, a / (2 pi), sin a, cos a, f^(1/3), f^(-7/6), 1/f.
struct BinW {
  df f, a, at, sa, ca, f13, fm76, invf;
};
__device__ __forceinline__ void load_bin_w(const DetDev& D, int b, BinW& W) {
  W.f = D.fw[b];
  W.f13 = D.f13w[b];
  W.fm76 = D.fm76w[b];
  W.a = D.aw[b];
  W.at = D.atw[b];
  W.sa = D.saw[b];
  W.ca = D.caw[b];
  W.invf = df_rcp(W.f);
}

// sinc(u) for |u| < 1e-3: 1 + u^2 (-1/6 + u^2/120) (the u^2/120 term enters the low word of -1/6;
// the dropped u^6/5040 is below 2e-22)
__device__ __forceinline__ df df_sinc_small(df u) {
  const df u2 = dfl_mul(u, u);
  const df p = df_make(-0.166666672f, __fmaf_rn(u2.x, 1.0f / 120.0f, 4.96705388e-09f));
  return dfl_add_o(df_make(1.f, 0.f), dfl_mul(u2, p));
}

// p[0..3] . b + p[4] in double words (the projection forms of DetDev::Mo, see proj_coef)
// sinc(u) for |u| <= 1 in double words: 1 + x (c1 + x (c2 + x (c3 + x (c4 + x T)))), x = u^2,
// c_k = (-1)^k / (2k+1)! as double words; the tail T = c5 + x (c6 + x (c7 + x c8)) is below
// 2.5e-8 and is evaluated in float (its rounding stays below 1e-14 of the result); the first
// dropped term is below 1/19! = 8.2e-18. With x <= 1 each Horner step adds a term at least six
// times smaller than its constant, so the steps take the ordered add.
__device__ __forceinline__ df df_sinc_poly(df u) {
  const df x = dfl_mul(u, u);
  float T = __fmaf_rn(x.x, 1.0f / 355687428096000.0f, -1.0f / 1307674368000.0f);
  T = __fmaf_rn(T, x.x, 1.0f / 6227020800.0f);
  T = __fmaf_rn(T, x.x, -1.0f / 39916800.0f);
  df p = dfl_add_o(df_make(2.75573188e-06f, 3.79357122e-14f), dfl_mulf(x, T));       // 1/9!
  p = dfl_add_o(df_make(-0.000198412701f, 2.72559687e-12f), dfl_mul(x, p));           // -1/7!
  p = dfl_add_o(df_make(0.00833333377f, -4.34617203e-10f), dfl_mul(x, p));            // 1/5!
  p = dfl_add_o(df_make(-0.166666672f, 4.96705388e-09f), dfl_mul(x, p));              // -1/3!
  return dfl_add_o(df_make(1.f, 0.f), dfl_mul(x, p));
}

__device__ __forceinline__ df dw_dot5(const float2* p, const df b[4]) {
  return dfl_add(dfl_add(dfl_mul(p[0], b[0]), dfl_mul(p[1], b[1])),
                  dfl_add(dfl_add(dfl_mul(p[2], b[2]), dfl_mul(p[3], b[3])), p[4]));
}

// double -> double word of the fraction x - rint(x) (exact in FP64), for the sincos of a turn count
__device__ __forceinline__ df frac_dw(double x) { return df_from_bits(x - rint(x)); }

// C2 (nullable): a second mode with the same m, evaluated with this one's geometry (see k32).
__device__ __forceinline__ void mode_bin_mixed(const DetDev& D, const SampleCoef& S, const ModeCoef& C, const BinIn& B,
                                               const BinW& W, MixAcc& acc, const float4* __restrict__ tab,
                                               const float2* __restrict__ pcw, const ModeCoef* C2 = nullptr) {
  // --- waveform (row A2): the phase in FP64
  const double v = C.cm * B.f13;
  const double lnv = C.lncm + B.lnf3;
  const double iv5 = C.icm5 * D.fm53[B.b];   // v^-5 = cm^-5 f^(-5/3)
  double poly = S.P[7];
#pragma unroll
  for (int k = 6; k >= 0; --k) poly = fma(poly, v, S.P[k]);
  const double q56 = fma(S.Q6, v, S.Q5);
  const double psi_pn = fma(iv5, poly, lnv * q56);
  // time-frequency map (row A3): t_f = t_c + (m / 12 pi) f^-1 v dPsi/dv with
  // v dPsi/dv = v^-5 sum_k Pd_k v^k + Q6 v ln v + q56, in double words. t_f only places the orbit,
  // so what matters is the error of the orbit angles alpha = alpha0 + t_f / yr (turns) and, for a
  // geocentric orbit, t_f / P_geo: while |t_f| < D.tfw_max they stay within ~1e-13 turn of their
  // FP64 values; beyond (the lowest frequencies of light systems) t_f and the angles are formed
  // in FP64 and reduced exactly there.
  const df vw = dfl_mul(C.cmw, W.f13);
  df dpol = S.Pdw[7];
#pragma unroll
  for (int k = 6; k >= 0; --k) dpol = dfl_add(dfl_mul(dpol, vw), S.Pdw[k]);
  const df dv = dfl_add(dfl_mul(df_from_bits(iv5), dpol),
                        dfl_add(dfl_mul(dfl_mul(S.Q6w, vw), df_from_bits(lnv)), df_from_bits(q56)));
  const df tf = dfl_add(S.tcw, dfl_mul(dfl_mul(C.tffacw, W.invf), dv));
  df alpha, geo;   // orbit angles in turns (df_cis_turns reduces them exactly)
  if (fabsf(tf.x) < D.tfw_max) {
    alpha = dfl_add(dfl_mul(tf, D.ratew), D.alpha0w);
    geo = dfl_mul(tf, D.geo_ratew);
  } else {
    double dpol64 = S.Pd[7];
#pragma unroll 1
    for (int k = 6; k >= 0; --k) dpol64 = fma(dpol64, v, S.Pd[k]);
    const double tf64 = fma(C.tffac * B.invf, fma(iv5, dpol64, fma(S.Q6 * v, lnv, q56)), S.tc);
    alpha = frac_dw(fma(tf64, D.rate_t, D.alpha0_t));
    geo = frac_dw(tf64 * D.geo_rate_t);
  }
  // amplitude (times hsc) in double words: ampw f^(-7/6) v^p, times the taper where it is below 1
  df A = dfl_mul(C.ampw, W.fm76);
  if (C.p >= 1) {
    A = dfl_mul(A, vw);
    if (C.p >= 2) A = dfl_mul(A, vw);
  }
  if (dlt_pos(C.ftap, B.f)) {
    const double span = C.fend - C.ftap;
    const double zt = span / (C.fend - B.f) - span / (B.f - C.ftap);
    A = dfl_mul(A, df_from_bits((zt > 700.0) ? 0.0 : 1.0 / (1.0 + exp(zt))));
  }
  // polarisation weights times the amplitude; a paired second mode makes them complex:
  // Pp + kappa Pp2, Pc + kappa Pc2, kappa = k32 v^2
  cdf Ap = {dfl_mul(A, C.Ppw), df_make(0.f, 0.f)}, Ac = {dfl_mul(A, C.Pcw), df_make(0.f, 0.f)};
  if (C2) {
    const df v2 = dfl_mul(vw, vw);
    const df kr = dfl_mul(S.k32w[0], v2), ki = dfl_mul(S.k32w[1], v2);
    Ap = cdf{dfl_mul(A, dfl_add(C.Ppw, dfl_mul(kr, C2->Ppw))), dfl_mul(A, dfl_mul(ki, C2->Ppw))};
    Ac = cdf{dfl_mul(A, dfl_add(C.Pcw, dfl_mul(kr, C2->Pcw))), dfl_mul(A, dfl_mul(ki, C2->Pcw))};
  }
  // --- orbital angle alpha(t_f) (row A4), centre Doppler f k.x_c, x_c = R (cos a, sin a, 0);
  // df_cis_turns reduces the angle in turns exactly
  const cdf eo = df_cis_turns(alpha, tab);
  const df co = eo.re, so = eo.im;
  const df kxc = dfl_mul(D.Rw, dfl_add(dfl_mul(S.kw[0], co), dfl_mul(S.kw[1], so)));
  // mode phase: the FP64 part reduced to a fraction of a turn, minus f k.x_c in double words
  const df pf = dfl_sub(frac_dw(fma(-C.mfac, psi_pn, C.ph0 - B.frc)), dfl_mul(W.f, kxc));
  // --- the offsets' basis (DetDev::Mo)
  df ob[4];
  if (D.orbit == 0) {
    ob[0] = dfl_sub(dfl_mul(co, co), dfl_mul(so, so));
    ob[1] = df_scale2(dfl_mul(so, co), 2.0f);
    ob[2] = co;
    ob[3] = so;
  } else {
    const cdf e0 = df_cis_turns(geo, tab);
    ob[0] = e0.re;
    ob[1] = e0.im;
    ob[2] = ob[3] = df_make(0.f, 0.f);
  }
  // --- third-spacecraft phases pi f k.delta_t (the offsets sum to zero, so delta_2's phase is
  // minus the other two); each link takes the mode phase plus its third spacecraft's phase
  const df e0 = df_scale2(dfl_mul(W.f, dw_dot5(pcw + 45, ob)), 0.5f);
  const df e1 = df_scale2(dfl_mul(W.f, dw_dot5(pcw + 50, ob)), 0.5f);
  const df e01 = dfl_add(e0, e1);
  // --- links (row A5); the loop stays rolled (one copy of its body) for the instruction cache.
  // Projections of the unnormalised link vectors x_r - x_s: the three sum to zero, so the third
  // is minus the sum of the other two
  cdf G[3];
  df smv[3], spv[3];
  df sk = df_make(0.f, 0.f), sp = sk, sq = sk;
#pragma unroll 1
  for (int l = 0; l < 3; ++l) {
    df knr, npr, nqr;
    if (l < 2) {
      knr = dw_dot5(pcw + 15 * l, ob);
      npr = dw_dot5(pcw + 15 * l + 5, ob);
      nqr = dw_dot5(pcw + 15 * l + 10, ob);
      sk = dfl_add(sk, knr);
      sp = dfl_add(sp, npr);
      sq = dfl_add(sq, nqr);
    } else {
      knr = df_make(-sk.x, -sk.y);
      npr = df_make(-sp.x, -sp.y);
      nqr = df_make(-sq.x, -sq.y);
    }
    const df inv = df_rsqrt(dfl_add(dfl_mul(knr, knr), dfl_add(dfl_mul(npr, npr), dfl_mul(nqr, nqr))));
    const df kn = dfl_mul(knr, inv);
    const df np = dfl_mul(npr, inv);
    const df nq = dfl_mul(nqr, inv);
    const df Fp = dfl_sub(dfl_mul(np, np), dfl_mul(nq, nq));
    const df Fc = df_scale2(dfl_mul(np, nq), 2.0f);
    const cdf gam = C2 ? cdf{dfl_sub(dfl_mul(Ap.re, Fp), dfl_mul(Ac.im, Fc)), dfl_add(dfl_mul(Ap.im, Fp), dfl_mul(Ac.re, Fc))}
                       : cdf{dfl_mul(Ap.re, Fp), dfl_mul(Ac.re, Fc)};
    // third spacecraft t = (l + 2) % 3
    const cdf Et = df_cis_turns(l == 0 ? dfl_sub(pf, e01) : dfl_add(pf, l == 1 ? e0 : e1), tab);
    G[l] = cdfl_mul(gam, Et);
    // sinc(a(1 -+ kn)): Taylor polynomial while a < kSincPolyA (|u| <= 2a < 1), else from
    // sin(a -+ a kn) = sin a cos(a kn) -+ cos a sin(a kn)
    const df akn = dfl_mul(W.a, kn);
    const df u1 = dfl_sub(W.a, akn), u2 = dfl_add(W.a, akn);
    if (dlt_pos(B.a, kSincPolyA)) {
      smv[l] = df_sinc_poly(u1);
      spv[l] = df_sinc_poly(u2);
    } else {
      const cdf ea = df_cis_turns(dfl_mul(W.at, kn), tab);
      const df sak = ea.im, cak = ea.re;
      const df x1 = dfl_mul(W.sa, cak), x2 = dfl_mul(W.ca, sak);
      const df s1 = dfl_sub(x1, x2), s2 = dfl_add(x1, x2);
      const bool small1 = fabsf(u1.x) < 1e-3f, small2 = fabsf(u2.x) < 1e-3f;
      if (!small1 && !small2) {
        const df rr = df_rcp(dfl_mul(u1, u2));
        smv[l] = dfl_mul(dfl_mul(s1, u2), rr);
        spv[l] = dfl_mul(dfl_mul(s2, u1), rr);
      } else {
        smv[l] = small1 ? df_sinc_small(u1) : dfl_mul(s1, df_rcp(u1));
        spv[l] = small2 ? df_sinc_small(u2) : dfl_mul(s2, df_rcp(u2));
      }
    }
  }
  // --- the links' products for the TDI brackets (row A6; see MixAcc)
#pragma unroll
  for (int l = 0; l < 3; ++l) {
    acc.Sr[l] = dfl_add(acc.Sr[l], dfl_mul(G[l].re, spv[l]));
    acc.Si[l] = dfl_add(acc.Si[l], dfl_mul(G[l].im, spv[l]));
    acc.Mr[l] = dfl_add(acc.Mr[l], dfl_mul(G[l].re, smv[l]));
    acc.Mi[l] = dfl_add(acc.Mi[l], dfl_mul(G[l].im, smv[l]));
  }
}

// Mode-summed TDI brackets X', Y', Z' of one sample at one bin times the sample's hsc, mixed
// precision.
__device__ __forceinline__ void bin_xyz_mixed(const DetDev& D, const SampleCoef& S, int b, cdf x[3],
                                              const float4* __restrict__ tab, const float2* __restrict__ pcw) {
  BinIn B;
  load_bin(D, b, S.tc, B);
  BinW W;
  load_bin_w(D, b, W);
  MixAcc a;
  mix_zero(a);
#pragma unroll 1
  for (int md = 0; md < kNModes; ++md) {
    if (md == 3 && S.pair32) continue;
    const ModeCoef& C = S.md[md];
    if (!C.active || !dlt_pos(B.f, C.fend)) continue;
    mode_bin_mixed(D, S, C, B, W, a, tab, pcw, (md == 0 && S.pair32) ? &S.md[3] : nullptr);
  }
  const float4 zz = D.zw[b];
  mix_final(a, cdf{df_make(zz.x, zz.y), df_make(zz.z, zz.w)}, x);
}

// A/E/T combinations (without Q n_c) in double words: B_A = Z' - X', B_E = X' - 2Y' + Z',
// B_T = X' + Y' + Z'. At long wavelength (a = pi f L << 1) B_T cancels to O(a^3) of the brackets
// (the six links' O(1) terms sum to zero exactly), so it is summed exactly (df_sum3_exact): a
// rounded double-word sum would leave an error of ~2^-47 of the brackets, which for the TianQin
// arm at 1e-4 Hz is ~1e-2 of B_T itself.
__device__ __forceinline__ void aet_from_xyz_dw(const cdf x[3], cdf o[3]) {
  o[0].re = dfl_sub(x[2].re, x[0].re);
  o[0].im = dfl_sub(x[2].im, x[0].im);
  o[1].re = dfl_sub(dfl_add(x[0].re, x[2].re), df_scale2(x[1].re, 2.0f));
  o[1].im = dfl_sub(dfl_add(x[0].im, x[2].im), df_scale2(x[1].im, 2.0f));
  o[2].re = df_sum3_exact(x[0].re, x[1].re, x[2].re);
  o[2].im = df_sum3_exact(x[0].im, x[1].im, x[2].im);
}

}  // namespace pe
