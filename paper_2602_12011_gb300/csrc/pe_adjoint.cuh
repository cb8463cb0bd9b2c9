// pe_adjoint.cuh -- hand-written reverse-mode derivative of one (sample, mode, bin) unit of the
// response (rows A2-A6, arXiv:2602.12011 Sec. 2.1), used by the gradient (row G1) and the Fisher
// matrix (row G2). The unit's forward intermediates are recomputed in registers (nothing per
// bin is stored), link by link, and the cotangents of its TDI brackets X', Y', Z' are pulled back
// to the source parameters.
//
// Conventions. For a real loss L and a complex intermediate z = x + iy the cotangent is
// zbar = dL/dx + i dL/dy, so dL = Re(conj(zbar) dz); for w = a b, abar = wbar conj(b).
#pragma once
#include "pe_device.cuh"

namespace pe {

// Adjoint accumulators of one thread: the theta components reached directly (Mtot, q, chi1,
// chi2, dL, iota, phi_c, t_c) and the sky-frame vectors k, p, q (contracted with their
// derivatives in lambda, beta, psi once per sample).
struct GradAcc {
  double M, q, c1, c2, dL, io, ph, tc;
  double k[3], p[3], qv[3];
};

__device__ __forceinline__ void gacc_zero(GradAcc& g) {
  g.M = g.q = g.c1 = g.c2 = g.dL = g.io = g.ph = g.tc = 0.0;
#pragma unroll
  for (int i = 0; i < 3; ++i) g.k[i] = g.p[i] = g.qv[i] = 0.0;
}

__device__ __forceinline__ double2 cconjmul(double2 a, double2 b) {  // a * conj(b)
  return make_double2(fma(a.x, b.x, a.y * b.y), fma(a.y, b.x, -a.x * b.y));
}

// d sinc(u)/du with the same small-argument series as sinc_small
__device__ __forceinline__ double dsinc(double u, double cosu, double sincu) {
  if (dlt_pos(fabs(u), 1e-3)) {
    const double u2 = u * u;
    return u * (-1.0 / 3.0 + u2 / 30.0 - u2 * u2 / 840.0);
  }
  return (cosu - sincu) / u;
}

// Reverse sweep of one unit. sX, sY, sZ: cotangents of this bin's brackets X', Y', Z'. md2 >= 0
// adds a second mode with the same m through this unit (complex polarisation weights
// Pp + kappa Pp2, Pc + kappa Pc2, kappa = k32 v^2; see SampleCoefT::k32), as the forward unit does.
__device__ __forceinline__ void mode_bwd(const DetDev& D, const SampleCoef& S, const SampleGrad& SG, int md,
                                         const BinIn& B, double2 sX, double2 sY, double2 sZ, GradAcc& g,
                                         const double2* __restrict__ tab, int md2 = -1) {
  const ModeCoef& C = S.md[md];
  const ModeGrad& CG = SG.md[md];
  // ---------------- forward recompute: waveform, t_f, amplitude, orbit, phase
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
  double vp = 1.0;
  if (C.p >= 1) vp *= v;
  if (C.p >= 2) vp *= v;
  const double amp0 = C.amp * B.fm76 * vp;
  const double amp = amp0 * w;
  // orbit
  double so, co;
  sincos_turns(fma(tf, D.rate_t, D.alpha0_t), tab, &so, &co);
  double xc[3] = {D.R * co, D.R * so, 0.0};
  double dl[3][3];
  double s0 = 0.0, c0 = 0.0, c2 = 0.0, s2 = 0.0;
  if (D.orbit == 0) {
    c2 = co * co - so * so;
    s2 = 2.0 * so * co;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      dl[i][0] = D.eRh * (c2 * D.cb[i] + s2 * D.sb[i]) - D.eR3h * D.cb[i];
      dl[i][1] = D.eRh * (s2 * D.cb[i] - c2 * D.sb[i]) - D.eR3h * D.sb[i];
      dl[i][2] = -D.eRs3 * (co * D.cb[i] + so * D.sb[i]);
    }
  } else {
    sincos_turns(tf * D.geo_rate_t, tab, &s0, &c0);
    const double ch = -0.5, sh = 0.86602540378443864676;
    double ci = c0, si = s0;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
#pragma unroll
      for (int j = 0; j < 3; ++j) dl[i][j] = D.rgeo * (ci * D.e1[j] + si * D.e2[j]);
      const double cn = ci * ch - si * sh, sn = si * ch + ci * sh;
      ci = cn; si = sn;
    }
  }
  const double kxc = S.k[0] * xc[0] + S.k[1] * xc[1] + S.k[2] * xc[2];
  const double ph = fma(-C.mfac, psi_pn, C.ph0 - B.frc) - B.f * kxc;
  const double phr = ph - rint(ph);
  // e^{2 pi i (ph + theta_t)}: the mode phase times the third spacecraft's phase
  // theta_t = f k.delta_t / 2 (turns); the offsets sum to zero, so theta_2 = -(theta_0 + theta_1)
  double2 Et[3];
  {
    const double th0 = 0.5 * B.f * (S.k[0] * dl[0][0] + S.k[1] * dl[0][1] + S.k[2] * dl[0][2]);
    const double th1 = 0.5 * B.f * (S.k[0] * dl[1][0] + S.k[1] * dl[1][1] + S.k[2] * dl[1][2]);
    sincos_turns_r(phr + th0, tab, &Et[0].y, &Et[0].x);
    sincos_turns_r(phr + th1, tab, &Et[1].y, &Et[1].x);
    sincos_turns_r(phr - (th0 + th1), tab, &Et[2].y, &Et[2].x);
  }
  // ---------------- links: forward and reverse, one pair at a time
  // seeds: pair 0 = (1,2): X' has -G U, Y' has +G V; pair 1 = (2,3): Y' -G U, Z' +G V;
  //        pair 2 = (3,1): Z' -G U, X' +G V.
  double ampb = 0.0, phtb = 0.0;   // cotangents of amp and of the summed angle 2 pi (ph + theta_t)
  double dlb[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i) dlb[i][0] = dlb[i][1] = dlb[i][2] = 0.0;
  // polarisation weights: Ap = Pp + kappa Pp2, Ac = Pc + kappa Pc2 (complex; kappa = 0 unpaired)
  double2 kap = make_double2(0.0, 0.0);
  double Pp2 = 0.0, Pc2 = 0.0;
  if (md2 >= 0) {
    kap = make_double2(S.k32.x * v * v, S.k32.y * v * v);
    Pp2 = S.md[md2].Pp;
    Pc2 = S.md[md2].Pc;
  }
  const double2 Ap = make_double2(fma(kap.x, Pp2, C.Pp), kap.y * Pp2);
  const double2 Ac = make_double2(fma(kap.x, Pc2, C.Pc), kap.y * Pc2);
  double2 Apb = make_double2(0.0, 0.0), Acb = make_double2(0.0, 0.0);
#pragma unroll
  for (int l = 0; l < 3; ++l) {
    const int r = l, s = (l + 1) % 3, t = (l + 2) % 3;
    double2 Su, Sv;
    if (l == 0) { Su = make_double2(-sX.x, -sX.y); Sv = sY; }
    else if (l == 1) { Su = make_double2(-sY.x, -sY.y); Sv = sZ; }
    else { Su = make_double2(-sZ.x, -sZ.y); Sv = sX; }
    double n[3] = {dl[r][0] - dl[s][0], dl[r][1] - dl[s][1], dl[r][2] - dl[s][2]};
    const double inv = rsqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    n[0] *= inv; n[1] *= inv; n[2] *= inv;
    const double kn = S.k[0] * n[0] + S.k[1] * n[1] + S.k[2] * n[2];
    const double np = S.p[0] * n[0] + S.p[1] * n[1] + S.p[2] * n[2];
    const double nq = S.q[0] * n[0] + S.q[1] * n[1] + S.q[2] * n[2];
    const double Fp = np * np - nq * nq, Fc = 2.0 * np * nq;
    const double2 gam = make_double2(fma(Ap.x, Fp, -Ac.y * Fc), fma(Ap.y, Fp, Ac.x * Fc));
    const double2 E = Et[t];
    const double se = E.y, ce = E.x;
    const double2 K = make_double2(amp * gam.x, amp * gam.y);
    const double2 G = cmul(K, E);
    const double u1 = B.a * (1.0 - kn), u2 = B.a * (1.0 + kn);
    double sm, spl, dsm, dspl;   // sinc(u1), sinc(u2) and their derivatives
    if (dlt_pos(B.a, kSincPolyA8)) {
      sinc_poly_d_n<4>(u1, &sm, &dsm);
      sinc_poly_d_n<4>(u2, &spl, &dspl);
    } else if (dlt_pos(B.a, kSincPolyA12)) {
      sinc_poly_d_n<6>(u1, &sm, &dsm);
      sinc_poly_d_n<6>(u2, &spl, &dspl);
    } else if (dlt_pos(B.a, kSincPolyA)) {
      sinc_poly_d(u1, &sm, &dsm);
      sinc_poly_d(u2, &spl, &dspl);
    } else {
      double sak, cak;
      sincos_turns(B.aturn * kn, tab, &sak, &cak);
      const double s1 = B.sa * cak - B.ca * sak, s2u = B.sa * cak + B.ca * sak;
      const double c1u = B.ca * cak + B.sa * sak, c2u = B.ca * cak - B.sa * sak;
      const bool small1 = dlt_pos(fabs(u1), 1e-3), small2 = dlt_pos(fabs(u2), 1e-3);
      if (!small1 && !small2) {
        const double rr = 1.0 / (u1 * u2);
        sm = s1 * u2 * rr;
        spl = s2u * u1 * rr;
      } else {
        sm = small1 ? sinc_small(u1) : s1 / u1;
        spl = small2 ? sinc_small(u2) : s2u / u2;
      }
      dsm = dsinc(u1, c1u, sm);
      dspl = dsinc(u2, c2u, spl);
    }
    const double2 U = make_double2(fma(B.z.x, spl, sm), B.z.y * spl);
    const double2 V = make_double2(fma(B.z.x, sm, spl), B.z.y * sm);
    // reverse
    const double2 Gb = cadd(cconjmul(Su, U), cconjmul(Sv, V));
    const double2 Ub = cconjmul(Su, G);
    const double2 Vb = cconjmul(Sv, G);
    const double smb = Ub.x + Vb.x * B.z.x + Vb.y * B.z.y;
    const double splb = Ub.x * B.z.x + Ub.y * B.z.y + Vb.x;
    const double u1b = smb * dsm;
    const double u2b = splb * dspl;
    const double knb = B.a * (u2b - u1b);
    const double2 Eb = cconjmul(Gb, K);
    const double2 Kb = cconjmul(Gb, E);
    const double thb = ce * Eb.y - se * Eb.x;
    phtb += thb;
    const double kdb = kPi * B.f * thb;
    const double2 gamb = make_double2(amp * Kb.x, amp * Kb.y);
    ampb = fma(Kb.x, gam.x, fma(Kb.y, gam.y, ampb));
    Apb = make_double2(fma(gamb.x, Fp, Apb.x), fma(gamb.y, Fp, Apb.y));
    Acb = make_double2(fma(gamb.y, Fc, Acb.x), fma(-gamb.x, Fc, Acb.y));
    const double Fpb = fma(gamb.x, Ap.x, gamb.y * Ap.y), Fcb = fma(gamb.y, Ac.x, -gamb.x * Ac.y);
    const double npb = 2.0 * (np * Fpb + nq * Fcb);
    const double nqb = 2.0 * (np * Fcb - nq * Fpb);
    double nb[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      g.k[i] = fma(knb, n[i], fma(kdb, dl[t][i], g.k[i]));
      g.p[i] = fma(npb, n[i], g.p[i]);
      g.qv[i] = fma(nqb, n[i], g.qv[i]);
      nb[i] = knb * S.k[i] + npb * S.p[i] + nqb * S.q[i];
    }
    const double dot = nb[0] * n[0] + nb[1] * n[1] + nb[2] * n[2];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const double db = (nb[i] - dot * n[i]) * inv;
      dlb[r][i] += db;
      dlb[s][i] -= db;
      dlb[t][i] = fma(kdb, S.k[i], dlb[t][i]);
    }
  }
  // ---------------- mode level: every link's angle holds 2 pi ph
  const double phb = 2.0 * kPi * phtb;
  g.ph = fma(phb, 2.0 * C.mfac, g.ph);          // d ph0/d phi_c = m/(2 pi)
  g.tc = fma(-B.f, phb, g.tc);                   // frac(f t_c)
  double psib = -C.mfac * phb;
  const double kxcb = -B.f * phb;
  double xcb[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) { g.k[i] = fma(kxcb, xc[i], g.k[i]); xcb[i] = kxcb * S.k[i]; }
  // orbit
  double cb_ = D.R * xcb[0], sb_ = D.R * xcb[1];
  double tfb;
  if (D.orbit == 0) {
    double c2b = 0.0, s2b = 0.0;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      c2b += D.eRh * (dlb[i][0] * D.cb[i] - dlb[i][1] * D.sb[i]);
      s2b += D.eRh * (dlb[i][0] * D.sb[i] + dlb[i][1] * D.cb[i]);
      cb_ -= D.eRs3 * dlb[i][2] * D.cb[i];
      sb_ -= D.eRs3 * dlb[i][2] * D.sb[i];
    }
    cb_ += 2.0 * (co * c2b + so * s2b);
    sb_ += 2.0 * (co * s2b - so * c2b);
    tfb = kPi * (co * sb_ - so * cb_) * D.rate_ht;
  } else {
    // d_i = rgeo (c_i e1 + s_i e2), (c_{i+1}, s_{i+1}) = rotation by 120 deg of (c_i, s_i)
    const double ch = -0.5, sh = 0.86602540378443864676;
    double cib = 0.0, sib = 0.0;
#pragma unroll
    for (int i = 2; i >= 0; --i) {
      // adjoint of the rotation that produced (c_{i+1}, s_{i+1}) from (c_i, s_i)
      const double cprev = cib * ch + sib * sh;
      const double sprev = -cib * sh + sib * ch;
      cib = cprev + D.rgeo * (dlb[i][0] * D.e1[0] + dlb[i][1] * D.e1[1] + dlb[i][2] * D.e1[2]);
      sib = sprev + D.rgeo * (dlb[i][0] * D.e2[0] + dlb[i][1] * D.e2[1] + dlb[i][2] * D.e2[2]);
    }
    tfb = kPi * (c0 * sib - s0 * cib) * D.geo_rate_ht + kPi * (co * sb_ - so * cb_) * D.rate_ht;
  }
  // t_f = t_c + (m/(12 pi f)) D(v)
  g.tc += tfb;
  const double Db = tfb * C.tffac * B.invf;
  // amplitude and taper
  double vb = 0.0;
  if (amp != 0.0) {
    const double lnAb = ampb * amp;
    g.M = fma(lnAb, CG.dlnA_dM, g.M);
    g.q = fma(lnAb, CG.dlnA_dq, g.q);
    g.dL = fma(lnAb, SG.dlnA_ddL, g.dL);
    vb = lnAb * double(C.p) * iv;
    if (tap) {
      const double wb = ampb * amp0;
      const double zb = -wb * w * (1.0 - w);
      const double fe = C.fend, ft = C.ftap, A = fe - ft;
      const double dz = 0.1 / (fe - B.f) - A / ((fe - B.f) * (fe - B.f)) - 0.1 / (B.f - ft) -
                        0.9 * A / ((B.f - ft) * (B.f - ft));
      g.M = fma(zb * dz, CG.dfend_dM, g.M);
    }
  }
  // Psi_PN(v), D(v): dPsi/dv = D/v, dD/dv = v^-5 ddpol / v + Q6 (2 + ln v)
  vb += psib * dv * iv + Db * (iv5 * ddpol * iv + S.Q6 * (2.0 + lnv));
  g.M = fma(vb * B.f13, CG.dcm_dM, g.M);
  // coefficient derivatives in q: Psi_q = v^-5 sum dP_k v^k + ln v (dQ5 + dQ6 v), D_q likewise
  double pq = SG.dP_dq[7], dq = SG.dPd_dq[7];
#pragma unroll
  for (int k = 6; k >= 0; --k) {
    pq = fma(pq, v, SG.dP_dq[k]);
    dq = fma(dq, v, SG.dPd_dq[k]);
  }
  const double psiq = fma(iv5, pq, lnv * fma(SG.dQ6_dq, v, SG.dQ5_dq));
  const double Dq = fma(iv5, dq, fma(SG.dQ6_dq * v, 1.0 + lnv, SG.dQ5_dq));
  g.q += psib * psiq + Db * Dq;
  // chi1, chi2 enter P3 (spin-orbit) and P4 (spin-spin): Psi += dP3 v^-2 + dP4 v^-1
  const double iv2 = iv * iv;
  g.c1 += psib * (SG.dP3_dc1 * iv2 + SG.dP4_dc1 * iv) - Db * (2.0 * SG.dP3_dc1 * iv2 + SG.dP4_dc1 * iv);
  g.c2 += psib * (SG.dP3_dc2 * iv2 + SG.dP4_dc2 * iv) - Db * (2.0 * SG.dP3_dc2 * iv2 + SG.dP4_dc2 * iv);
  // polarisation weights, and the paired mode: Ap = Pp + kappa Pp2, Ac = Pc + kappa Pc2
  g.io += Apb.x * CG.dPp_di + Acb.x * CG.dPc_di;
  if (md2 >= 0) {
    const ModeGrad& CG2 = SG.md[md2];
    g.io += (Apb.x * kap.x + Apb.y * kap.y) * CG2.dPp_di + (Acb.x * kap.x + Acb.y * kap.y) * CG2.dPc_di;
    const double2 kb = make_double2(Apb.x * Pp2 + Acb.x * Pc2, Apb.y * Pp2 + Acb.y * Pc2);   // kappa-bar
    // kappa = k32 v^2, k32 = (amp2 / amp1) e^{2 pi i (ph0_2 - ph0_1)}; the same m makes the phase
    // difference and the v-scale independent of theta, so only ln(amp2 / amp1) varies (M, q)
    const double lnrb = v * v * (kb.x * S.k32.x + kb.y * S.k32.y);
    g.M = fma(lnrb, CG2.dlnA_dM - CG.dlnA_dM, g.M);
    g.q = fma(lnrb, CG2.dlnA_dq - CG.dlnA_dq, g.q);
    const double vkb = 2.0 * lnrb / v;   // d kappa / d v = 2 kappa / v
    g.M = fma(vkb * B.f13, CG.dcm_dM, g.M);
  }
}

// Contract one thread's accumulators with the sample's sky-frame derivatives into grad[11].
__device__ __forceinline__ void gacc_to_theta(const GradAcc& g, const SampleGrad& SG, double out[PE_NPARAM]) {
  out[0] = g.M; out[1] = g.q; out[2] = g.c1; out[3] = g.c2; out[4] = g.dL; out[5] = g.io; out[6] = g.ph;
  for (int j = 0; j < 3; ++j) {
    double a = 0.0;
    for (int i = 0; i < 3; ++i) a += g.k[i] * SG.dk[i][j] + g.p[i] * SG.dp[i][j] + g.qv[i] * SG.dq[i][j];
    out[7 + j] = a;
  }
  out[10] = g.tc;
}

}  // namespace pe
