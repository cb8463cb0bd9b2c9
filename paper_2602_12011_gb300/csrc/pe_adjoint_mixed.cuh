// pe_adjoint_mixed.cuh -- the reverse sweep of pe_adjoint.cuh (rows G1 of the gradient, Sec. 2.3 on
// automatic differentiation) with the response geometry, the link factors, the sincs, the TDI
// brackets and every per-link cotangent in double-word arithmetic (pe_df.cuh, ~1e-14 relative), as
// the mixed-precision forward unit (pe_device_mixed.cuh) has them. The FP64 pipe keeps the TaylorF2
// phase and t_f, the exact turn reductions, the PN-coefficient chain rule at the mode level and the
// accumulation across bins.
//
// Scales: the amplitude enters times the sample's power of two hsc (as in the forward unit) and the
// bracket cotangents times its inverse ihsc, so every geometric cotangent comes out at its true
// scale; the amplitude's own cotangent comes out times ihsc and meets the scaled amplitude again in
// d log A = ampb amp.
//
// Geometry. The offsets d_0, d_1 of spacecraft 0 and 1 from the centre are linear forms in the
// orbit basis (DetDev::Mo, staged per tile as double words); d_2 = -(d_0 + d_1). Link l's vector
// is x_r - x_s = alpha_l d_0 + beta_l d_1 and its third spacecraft's offset is gamma_l d_0 +
// delta_l d_1, with small integer weights, so the link loop indexes no array by l and the
// cotangents of d_0, d_1 collect in registers; they reach the orbit basis through the same forms.
#pragma once
#include "pe_adjoint.cuh"
#include "pe_device_mixed.cuh"

namespace pe {

// double-word accumulators of the sky-frame cotangents k, p, q of one bin
struct GradAccW {
  df k[3], p[3], q[3];
};
__device__ __forceinline__ void gaccw_zero(GradAccW& a) {
#pragma unroll
  for (int i = 0; i < 3; ++i) a.k[i] = a.p[i] = a.q[i] = df_make(0.f, 0.f);
}
__device__ __forceinline__ void gaccw_flush(const GradAccW& a, GradAcc& g) {
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    g.k[i] += df_to(a.k[i]);
    g.p[i] += df_to(a.p[i]);
    g.qv[i] += df_to(a.q[i]);
  }
}

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
__device__ __forceinline__ df dw_dot3(const float2* a, const df b[3]) {
  return dfl_add(dfl_add(dfl_mul(a[0], b[0]), dfl_mul(a[1], b[1])), dfl_mul(a[2], b[2]));
}

// sinc(u) and d sinc/du for |u| <= 1 in double words. With x = u^2: sinc = 1 + x P(x) (the series of
// df_sinc_poly) and d sinc/du = 2 u Q(x), Q(x) = sum_k k c_k x^(k-1), c_k = (-1)^k / (2k+1)!:
// Q = c1 + x (2 c2 + x (3 c3 + x (4 c4 + x T))), T = 5 c5 + x (6 c6 + x (7 c7 + x 8 c8)) in float
// (|T| < 1.3e-7); the first dropped term, 9 c9 x^8, is below 7.5e-17.
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
  df q = dfl_add(df_make(1.10229275e-05f, 1.5174285e-13f), dfl_mulf(x, T));   // 4 c4
  q = dfl_add(df_make(-0.0005952381f, 2.2728706e-11f), dfl_mul(x, q));          // 3 c3
  q = dfl_add(df_make(0.016666668f, -8.692344e-10f), dfl_mul(x, q));            // 2 c2
  q = dfl_add(df_make(-0.16666667f, 4.967054e-09f), dfl_mul(x, q));             // c1
  r.d = df_scale2(dfl_mul(u, q), 2.0f);
  return r;
}
// d sinc/du for |u| < 1e-3: u (-1/3 + u^2/30) (the dropped u^5/840 is below 1.2e-15 of the result)
__device__ __forceinline__ df df_dsinc_small(df u) {
  const df u2 = dfl_mul(u, u);
  const df p = df_make(-0.33333334f, __fmaf_rn(u2.x, 0.033333335f, 9.934108e-09f));
  return dfl_mul(u, p);
}

// Reverse sweep of one unit in double words; arguments as mode_bwd, plus: W, zw: the bin's
// double-word values and z; sX, sY, sZ: bracket cotangents times ihsc; gw: the bin's double-word
// k, p, q accumulators; tab: the double-word sincos table; kpq: the sample's k, p, q as double
// words [3][3]; mow: DetDev::Mo[0..1] as double words [2][3][5].
__device__ __forceinline__ void mode_bwd_mixed(const DetDev& D, const SampleCoef& S, const SampleGrad& SG, int md,
                                               const BinIn& B, const BinW& W, const cdf& zw, const cdf& sX,
                                               const cdf& sY, const cdf& sZ, GradAcc& g, GradAccW& gw,
                                               const float4* __restrict__ tab, const float2* __restrict__ kpq,
                                               const float2* __restrict__ mow, int md2 = -1) {
  const ModeCoef& C = S.md[md];
  const ModeGrad& CG = SG.md[md];
  // ---------------- FP64: waveform and t_f (rows A2, A3), as mode_bwd
  const double v = C.cm * B.f13;
  const double iv = C.icm * B.fm13;
  const double lnv = C.lncm + B.lnf3;
  double iv5 = iv * iv;
  iv5 = iv5 * iv5 * iv;
  double poly = S.P[7];
  double dpol = S.Pd[7];
  double ddpol = S.Pdd[7];
#pragma unroll
  for (int k = 6; k >= 0; --k) {
    poly = fma(poly, v, S.P[k]);
    dpol = fma(dpol, v, S.Pd[k]);
    ddpol = fma(ddpol, v, S.Pdd[k]);
  }
  const double psi_pn = fma(iv5, poly, lnv * fma(S.Q6, v, S.Q5));
  const double dv = fma(iv5, dpol, fma(S.Q6 * v, 1.0 + lnv, S.Q5));
  const double tf = fma(C.tffac * B.invf, dv, S.tc);
  double w = 1.0, zt = 0.0;
  const bool tap = dlt_pos(C.ftap, B.f);
  if (tap) {
    const double span = C.fend - C.ftap;
    zt = span / (C.fend - B.f) - span / (B.f - C.ftap);
    w = (zt > 700.0) ? 0.0 : 1.0 / (1.0 + exp(zt));
  }
  // ---------------- double words: amplitude times hsc (A0 before the taper, A after it)
  const df vw = dfl_mul(C.cmw, W.f13);
  df A0 = dfl_mul(C.ampw, W.fm76);
  if (C.p >= 1) A0 = dfl_mul(A0, vw);
  if (C.p >= 2) A0 = dfl_mul(A0, vw);
  const df A = tap ? dfl_mul(A0, df_from_bits(w)) : A0;
  // orbit (row A4): centre angle, the offsets' basis, spacecraft offsets d_0, d_1
  const cdf eo = df_cis_turns(frac_dw(fma(tf, D.rate_t, D.alpha0_t)), tab);
  const df co = eo.re, so = eo.im;
  df ob[4];
  cdf eg = {df_make(0.f, 0.f), df_make(0.f, 0.f)};
  if (D.orbit == 0) {
    ob[0] = dfl_sub(dfl_mul(co, co), dfl_mul(so, so));
    ob[1] = df_scale2(dfl_mul(so, co), 2.0f);
    ob[2] = co;
    ob[3] = so;
  } else {
    eg = df_cis_turns(frac_dw(tf * D.geo_rate_t), tab);
    ob[0] = eg.re;
    ob[1] = eg.im;
    ob[2] = ob[3] = df_make(0.f, 0.f);
  }
  df d0[3], d1[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    d0[j] = dw_dot5(mow + 5 * j, ob);
    d1[j] = dw_dot5(mow + 15 + 5 * j, ob);
  }
  // mode phase (FP64 part reduced to a fraction of a turn) minus f k.x_c; third-spacecraft phases
  // theta_t = f k.d_t / 2 in turns
  const df kxc = dfl_mul(D.Rw, dfl_add(dfl_mul(kpq[0], co), dfl_mul(kpq[1], so)));
  const df pf = dfl_sub(frac_dw(fma(-C.mfac, psi_pn, C.ph0 - B.frc)), dfl_mul(W.f, kxc));
  const df hf = df_scale2(W.f, 0.5f);
  const df th0 = dfl_mul(hf, dw_dot3(kpq, d0)), th1 = dfl_mul(hf, dw_dot3(kpq, d1));
  const df th01 = dfl_add(th0, th1);
  const df pif = dfl_mul(W.f, df_make(3.1415927f, -8.742278e-08f));   // pi f
  // polarisation weights Ap = Pp + kappa Pp2, Ac = Pc + kappa Pc2 (kappa = k32 v^2; 0 unpaired)
  cdf Ap = {C.Ppw, df_make(0.f, 0.f)}, Ac = {C.Pcw, df_make(0.f, 0.f)};
  if (md2 >= 0) {
    const df v2 = dfl_mul(vw, vw);
    const df kr = dfl_mul(S.k32w[0], v2), ki = dfl_mul(S.k32w[1], v2);
    const ModeCoef& C2 = S.md[md2];
    Ap = cdf{dfl_add(C.Ppw, dfl_mul(kr, C2.Ppw)), dfl_mul(ki, C2.Ppw)};
    Ac = cdf{dfl_add(C.Pcw, dfl_mul(kr, C2.Pcw)), dfl_mul(ki, C2.Pcw)};
  }
  // ---------------- links: forward and reverse, one pair at a time (seeds as in mode_bwd)
  const df zero = df_make(0.f, 0.f);
  df phtb = zero, ampb = zero;
  cdf Apb = {zero, zero}, Acb = {zero, zero};
  df d0b[3] = {zero, zero, zero}, d1b[3] = {zero, zero, zero};
#pragma unroll 1
  for (int l = 0; l < 3; ++l) {
    // x_r - x_s = al d_0 + be d_1; the third spacecraft t = (l + 2) % 3 sits at ga d_0 + de d_1
    const float al = (l == 2) ? -2.f : 1.f;
    const float be = (l == 0) ? -1.f : (l == 1 ? 2.f : -1.f);
    const float ga = (l == 0) ? -1.f : (l == 1 ? 1.f : 0.f);
    const float de = (l == 0) ? -1.f : (l == 1 ? 0.f : 1.f);
    const cdf& su = (l == 0) ? sX : (l == 1 ? sY : sZ);
    const cdf& Sv = (l == 0) ? sY : (l == 1 ? sZ : sX);
    const cdf Su = {df_neg(su.re), df_neg(su.im)};
    df n[3], dt[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      n[j] = dfl_add(df_scale2(d0[j], al), df_scale2(d1[j], be));
      dt[j] = dfl_add(df_scale2(d0[j], ga), df_scale2(d1[j], de));
    }
    const df inv = df_rsqrt(dfl_add(dfl_add(dfl_mul(n[0], n[0]), dfl_mul(n[1], n[1])), dfl_mul(n[2], n[2])));
#pragma unroll
    for (int j = 0; j < 3; ++j) n[j] = dfl_mul(n[j], inv);
    const df kn = dw_dot3(kpq, n), np = dw_dot3(kpq + 3, n), nq = dw_dot3(kpq + 6, n);
    const df Fp = dfl_sub(dfl_mul(np, np), dfl_mul(nq, nq));
    const df Fc = df_scale2(dfl_mul(np, nq), 2.0f);
    const cdf gam = (md2 >= 0) ? cdf{dfl_sub(dfl_mul(Ap.re, Fp), dfl_mul(Ac.im, Fc)),
                                     dfl_add(dfl_mul(Ap.im, Fp), dfl_mul(Ac.re, Fc))}
                               : cdf{dfl_mul(Ap.re, Fp), dfl_mul(Ac.re, Fc)};
    const cdf E = df_cis_turns(l == 0 ? dfl_sub(pf, th01) : dfl_add(pf, l == 1 ? th0 : th1), tab);
    const cdf K = {dfl_mul(A, gam.re), dfl_mul(A, gam.im)};
    const cdf G = cdf_mul_s(K, E);
    const df akn = dfl_mul(W.a, kn);
    const df u1 = dfl_sub(W.a, akn), u2 = dfl_add(W.a, akn);
    df sm, spl, dsm, dspl;   // sinc(u1), sinc(u2) and their derivatives
    if (dlt_pos(B.a, kSincPolyA)) {
      const df2 r1 = df_sinc_poly_d(u1), r2 = df_sinc_poly_d(u2);
      sm = r1.v;
      dsm = r1.d;
      spl = r2.v;
      dspl = r2.d;
    } else {
      const cdf ea = df_cis_turns(dfl_mul(W.at, kn), tab);
      const df x1 = dfl_mul(W.sa, ea.re), x2 = dfl_mul(W.ca, ea.im);
      const df y1 = dfl_mul(W.ca, ea.re), y2 = dfl_mul(W.sa, ea.im);
      const df s1 = dfl_sub(x1, x2), s2 = dfl_add(x1, x2);   // sin u1, sin u2
      const df c1 = dfl_add(y1, y2), c2 = dfl_sub(y1, y2);   // cos u1, cos u2
      if (fabsf(u1.x) < 1e-3f) {
        sm = df_sinc_small(u1);
        dsm = df_dsinc_small(u1);
      } else {
        const df r1 = df_rcp(u1);
        sm = dfl_mul(s1, r1);
        dsm = dfl_mul(dfl_sub(c1, sm), r1);
      }
      if (fabsf(u2.x) < 1e-3f) {
        spl = df_sinc_small(u2);
        dspl = df_dsinc_small(u2);
      } else {
        const df r2 = df_rcp(u2);
        spl = dfl_mul(s2, r2);
        dspl = dfl_mul(dfl_sub(c2, spl), r2);
      }
    }
    const cdf U = {dfl_add(dfl_mul(zw.re, spl), sm), dfl_mul(zw.im, spl)};
    const cdf V = {dfl_add(dfl_mul(zw.re, sm), spl), dfl_mul(zw.im, sm)};
    // reverse
    const cdf Gb = cdf_add_s(cdf_mul_conj(Su, U), cdf_mul_conj(Sv, V));
    const cdf Ub = cdf_mul_conj(Su, G), Vb = cdf_mul_conj(Sv, G);
    const df smb = dfl_add(Ub.re, dfl_add(dfl_mul(Vb.re, zw.re), dfl_mul(Vb.im, zw.im)));
    const df splb = dfl_add(dfl_add(dfl_mul(Ub.re, zw.re), dfl_mul(Ub.im, zw.im)), Vb.re);
    const df knb = dfl_mul(W.a, dfl_sub(dfl_mul(splb, dspl), dfl_mul(smb, dsm)));
    const cdf Eb = cdf_mul_conj(Gb, K), Kb = cdf_mul_conj(Gb, E);
    const df thb = dfl_sub(dfl_mul(E.re, Eb.im), dfl_mul(E.im, Eb.re));
    phtb = dfl_add(phtb, thb);
    const df kdb = dfl_mul(pif, thb);
    const cdf gamb = {dfl_mul(A, Kb.re), dfl_mul(A, Kb.im)};
    ampb = dfl_add(ampb, dfl_add(dfl_mul(Kb.re, gam.re), dfl_mul(Kb.im, gam.im)));
    Apb = cdf{dfl_add(Apb.re, dfl_mul(gamb.re, Fp)), dfl_add(Apb.im, dfl_mul(gamb.im, Fp))};
    Acb = cdf{dfl_add(Acb.re, dfl_mul(gamb.im, Fc)), dfl_sub(Acb.im, dfl_mul(gamb.re, Fc))};
    const df Fpb = dfl_add(dfl_mul(gamb.re, Ap.re), dfl_mul(gamb.im, Ap.im));
    const df Fcb = dfl_sub(dfl_mul(gamb.im, Ac.re), dfl_mul(gamb.re, Ac.im));
    const df npb = df_scale2(dfl_add(dfl_mul(np, Fpb), dfl_mul(nq, Fcb)), 2.0f);
    const df nqb = df_scale2(dfl_sub(dfl_mul(np, Fcb), dfl_mul(nq, Fpb)), 2.0f);
    df nb[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      gw.k[j] = dfl_add(gw.k[j], dfl_add(dfl_mul(knb, n[j]), dfl_mul(kdb, dt[j])));
      gw.p[j] = dfl_add(gw.p[j], dfl_mul(npb, n[j]));
      gw.q[j] = dfl_add(gw.q[j], dfl_mul(nqb, n[j]));
      nb[j] = dfl_add(dfl_add(dfl_mul(knb, kpq[j]), dfl_mul(npb, kpq[3 + j])), dfl_mul(nqb, kpq[6 + j]));
    }
    const df dot = dfl_add(dfl_add(dfl_mul(nb[0], n[0]), dfl_mul(nb[1], n[1])), dfl_mul(nb[2], n[2]));
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const df db = dfl_mul(dfl_sub(nb[j], dfl_mul(dot, n[j])), inv);   // cotangent of x_r - x_s
      const df kk = dfl_mul(kdb, kpq[j]);                                // of the third spacecraft's offset
      d0b[j] = dfl_add(d0b[j], dfl_add(df_scale2(db, al), df_scale2(kk, ga)));
      d1b[j] = dfl_add(d1b[j], dfl_add(df_scale2(db, be), df_scale2(kk, de)));
    }
  }
  // ---------------- the offsets' basis: obb[m] = sum_j d0b_j Mo[0][j][m] + d1b_j Mo[1][j][m]
  df obb[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    df a = zero;
#pragma unroll
    for (int j = 0; j < 3; ++j) a = dfl_add(a, dfl_add(dfl_mul(d0b[j], mow[5 * j + m]), dfl_mul(d1b[j], mow[15 + 5 * j + m])));
    obb[m] = a;
  }
  // ---------------- mode level: the phase cotangent in FP64; the orbit's reverse in double words
  // (the centre x_c = R (cos a, sin a, 0) and the offsets' basis), t_f's cotangent back in FP64
  const double phb = 2.0 * kPi * df_to(phtb);
  g.ph = fma(phb, 2.0 * C.mfac, g.ph);          // d ph0/d phi_c = m/(2 pi)
  g.tc = fma(-B.f, phb, g.tc);                   // frac(f t_c)
  const double psib = -C.mfac * phb;
  const df kxcb = df_from_bits(-B.f * phb);
  const df Rk = dfl_mul(D.Rw, kxcb);
  gw.k[0] = dfl_add(gw.k[0], dfl_mul(Rk, co));
  gw.k[1] = dfl_add(gw.k[1], dfl_mul(Rk, so));
  df cb_ = dfl_mul(Rk, kpq[0]), sb_ = dfl_mul(Rk, kpq[1]);
  double tfb;
  if (D.orbit == 0) {
    // ob = (cos 2a, sin 2a, cos a, sin a)
    cb_ = dfl_add(cb_, dfl_add(obb[2], df_scale2(dfl_add(dfl_mul(co, obb[0]), dfl_mul(so, obb[1])), 2.0f)));
    sb_ = dfl_add(sb_, dfl_add(obb[3], df_scale2(dfl_sub(dfl_mul(co, obb[1]), dfl_mul(so, obb[0])), 2.0f)));
    tfb = kPi * D.rate_ht * df_to(dfl_sub(dfl_mul(co, sb_), dfl_mul(so, cb_)));
  } else {
    // ob = (cos phi_0, sin phi_0, 0, 0)
    tfb = kPi * D.geo_rate_ht * df_to(dfl_sub(dfl_mul(eg.re, obb[1]), dfl_mul(eg.im, obb[0]))) +
          kPi * D.rate_ht * df_to(dfl_sub(dfl_mul(co, sb_), dfl_mul(so, cb_)));
  }
  g.tc += tfb;
  const double Db = tfb * C.tffac * B.invf;
  double vb = 0.0;
  if (C.amp != 0.0 && w != 0.0) {
    const double lnAb = df_to(dfl_mul(ampb, A));
    g.M = fma(lnAb, CG.dlnA_dM, g.M);
    g.q = fma(lnAb, CG.dlnA_dq, g.q);
    g.dL = fma(lnAb, SG.dlnA_ddL, g.dL);
    vb = lnAb * double(C.p) * iv;
    if (tap) {
      const double wb = df_to(dfl_mul(ampb, A0));
      const double zb = -wb * w * (1.0 - w);
      const double fe = C.fend, ft = C.ftap, As = fe - ft;
      const double dz = 0.1 / (fe - B.f) - As / ((fe - B.f) * (fe - B.f)) - 0.1 / (B.f - ft) -
                        0.9 * As / ((B.f - ft) * (B.f - ft));
      g.M = fma(zb * dz, CG.dfend_dM, g.M);
    }
  }
  vb += psib * dv * iv + Db * (iv5 * ddpol * iv + S.Q6 * (2.0 + lnv));
  g.M = fma(vb * B.f13, CG.dcm_dM, g.M);
  double pq = SG.dP_dq[7], dq = SG.dPd_dq[7];
#pragma unroll
  for (int k = 6; k >= 0; --k) {
    pq = fma(pq, v, SG.dP_dq[k]);
    dq = fma(dq, v, SG.dPd_dq[k]);
  }
  const double psiq = fma(iv5, pq, lnv * fma(SG.dQ6_dq, v, SG.dQ5_dq));
  const double Dq = fma(iv5, dq, fma(SG.dQ6_dq * v, 1.0 + lnv, SG.dQ5_dq));
  g.q += psib * psiq + Db * Dq;
  const double iv2 = iv * iv;
  g.c1 += psib * (SG.dP3_dc1 * iv2 + SG.dP4_dc1 * iv) - Db * (2.0 * SG.dP3_dc1 * iv2 + SG.dP4_dc1 * iv);
  g.c2 += psib * (SG.dP3_dc2 * iv2 + SG.dP4_dc2 * iv) - Db * (2.0 * SG.dP3_dc2 * iv2 + SG.dP4_dc2 * iv);
  const double Apbx = df_to(Apb.re), Acbx = df_to(Acb.re);
  g.io += Apbx * CG.dPp_di + Acbx * CG.dPc_di;
  if (md2 >= 0) {
    const ModeGrad& CG2 = SG.md[md2];
    const double Apby = df_to(Apb.im), Acby = df_to(Acb.im);
    const double Pp2 = S.md[md2].Pp, Pc2 = S.md[md2].Pc;
    const double2 kap = make_double2(S.k32.x * v * v, S.k32.y * v * v);
    g.io += (Apbx * kap.x + Apby * kap.y) * CG2.dPp_di + (Acbx * kap.x + Acby * kap.y) * CG2.dPc_di;
    const double2 kb = make_double2(Apbx * Pp2 + Acbx * Pc2, Apby * Pp2 + Acby * Pc2);
    const double lnrb = v * v * (kb.x * S.k32.x + kb.y * S.k32.y);
    g.M = fma(lnrb, CG2.dlnA_dM - CG.dlnA_dM, g.M);
    g.q = fma(lnrb, CG2.dlnA_dq - CG.dlnA_dq, g.q);
    const double vkb = 2.0 * lnrb / v;
    g.M = fma(vkb * B.f13, CG.dcm_dM, g.M);
  }
}

}  // namespace pe
