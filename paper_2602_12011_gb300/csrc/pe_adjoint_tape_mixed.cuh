// pe_adjoint_tape_mixed.cuh -- the tape gradient of pe_adjoint_tape.cuh in mixed precision
// (PE_PREC_MIXED; row G1, arXiv:2602.12011 Sec. 2.2-2.3). The forward pass is the mixed-precision
// unit (mode_bin_mixed: FP64 TaylorF2 phase and its exact turn reduction; double-word t_f,
// geometry, sincs and TDI brackets, same operations in the same order) writing the double words
// its reverse needs to the tape; the reverse sweep runs in double words from the tape, and only
// the phase and t_f cotangents and the PN chain rule at the mode level return to FP64. The
// per-tile contraction of the form cotangents with the orbit basis runs in double words too.
//
// The tape has the FP64 tape's layout (pe_adjoint_tape.cuh) with every field a double word
// (8 bytes, as a double): kTamp0 holds the amplitude times hsc before the taper, kTw after it.
#pragma once
#include "pe_adjoint_mixed.cuh"
#include "pe_adjoint_tape.cuh"

namespace pe {

// The same hinted accesses for double-word fields (tape_l2_policy, pe_adjoint_tape.cuh).
__device__ __forceinline__ void tst(df* a, df v, unsigned long long pol) {
  asm volatile("st.global.L2::cache_hint.v2.f32 [%0], {%1, %2}, %3;" ::"l"(__cvta_generic_to_global(a)), "f"(v.x),
               "f"(v.y), "l"(pol)
               : "memory");
}
__device__ __forceinline__ df tld(const df* a, unsigned long long pol) {
  df v;
  asm volatile("ld.global.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;"
               : "=f"(v.x), "=f"(v.y)
               : "l"(__cvta_generic_to_global(a)), "l"(pol)
               : "memory");
  return v;
}

// Forward pass of one unit: mode_bin_mixed plus the tape and the sincs' derivatives in k.n.
__device__ __forceinline__ void mode_fwd_tape_mixed(const DetDev& D, const SampleCoef& S, const ModeCoef& C,
                                                    const BinIn& B, const BinW& W, MixAcc& acc,
                                                    const float4* __restrict__ tab, const float2* __restrict__ pcw,
                                                    const ModeCoef* C2, df* tp, unsigned long long pol) {
  const double v = C.cm * B.f13;
  const double lnv = C.lncm + B.lnf3;
  const double iv5 = C.icm5 * D.fm53[B.b];
  double poly = S.P[7];
#pragma unroll
  for (int k = 6; k >= 0; --k) poly = fma(poly, v, S.P[k]);
  const double q56 = fma(S.Q6, v, S.Q5);
  const double psi_pn = fma(iv5, poly, lnv * q56);
  const df vw = dfl_mul(C.cmw, W.f13);
  df dpol = S.Pdw[7];
#pragma unroll
  for (int k = 6; k >= 0; --k) dpol = dfl_add(dfl_mul(dpol, vw), S.Pdw[k]);
  const df dv = dfl_add(dfl_mul(df_from_bits(iv5), dpol),
                        dfl_add(dfl_mul(dfl_mul(S.Q6w, vw), df_from_bits(lnv)), df_from_bits(q56)));
  const df tf = dfl_add(S.tcw, dfl_mul(dfl_mul(C.tffacw, W.invf), dv));
  df alpha, geo;
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
  df A = dfl_mul(C.ampw, W.fm76);
  if (C.p >= 1) {
    A = dfl_mul(A, vw);
    if (C.p >= 2) A = dfl_mul(A, vw);
  }
  tst(tp + (kTamp0 * kTileBins), A, pol);
  if (dlt_pos(C.ftap, B.f)) {
    const double span = C.fend - C.ftap;
    const double zt = span / (C.fend - B.f) - span / (B.f - C.ftap);
    A = dfl_mul(A, df_from_bits((zt > 700.0) ? 0.0 : 1.0 / (1.0 + exp(zt))));
  }
  tst(tp + (kTw * kTileBins), A, pol);
  tst(tp + (kTdv * kTileBins), dv, pol);
  cdf Ap = {dfl_mul(A, C.Ppw), df_make(0.f, 0.f)}, Ac = {dfl_mul(A, C.Pcw), df_make(0.f, 0.f)};
  if (C2) {
    const df v2 = dfl_mul(vw, vw);
    const df kr = dfl_mul(S.k32w[0], v2), ki = dfl_mul(S.k32w[1], v2);
    Ap = cdf{dfl_mul(A, dfl_add(C.Ppw, dfl_mul(kr, C2->Ppw))), dfl_mul(A, dfl_mul(ki, C2->Ppw))};
    Ac = cdf{dfl_mul(A, dfl_add(C.Pcw, dfl_mul(kr, C2->Pcw))), dfl_mul(A, dfl_mul(ki, C2->Pcw))};
  }
  const cdf eo = df_cis_turns(alpha, tab);
  const df co = eo.re, so = eo.im;
  const df kxc = dfl_mul(D.Rw, dfl_add(dfl_mul(S.kw[0], co), dfl_mul(S.kw[1], so)));
  const df pf = dfl_sub(frac_dw(fma(-C.mfac, psi_pn, C.ph0 - B.frc)), dfl_mul(W.f, kxc));
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
  tst(tp + (kTco * kTileBins), co, pol);
  tst(tp + (kTso * kTileBins), so, pol);
  tst(tp + (kTob0 * kTileBins), ob[0], pol);
  tst(tp + (kTob1 * kTileBins), ob[1], pol);
  const df e0 = df_scale2(dfl_mul(W.f, dw_dot5(pcw + 45, ob)), 0.5f);
  const df e1 = df_scale2(dfl_mul(W.f, dw_dot5(pcw + 50, ob)), 0.5f);
  const df e01 = dfl_add(e0, e1);
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
    const int t = (l == 0) ? 2 : l - 1;   // third spacecraft
    const cdf Et = df_cis_turns(l == 0 ? dfl_sub(pf, e01) : dfl_add(pf, l == 1 ? e0 : e1), tab);
    tst(tp + ((kTE + 2 * t) * kTileBins), Et.re, pol);
    tst(tp + ((kTE + 2 * t + 1) * kTileBins), Et.im, pol);
    G[l] = cdfl_mul(gam, Et);
    // sincs, and their derivatives in kn: d s-/dkn = -a sinc'(u1), d s+/dkn = a sinc'(u2)
    const df akn = dfl_mul(W.a, kn);
    const df u1 = dfl_sub(W.a, akn), u2 = dfl_add(W.a, akn);
    df dsm, dspl;
    if (dlt_pos(B.a, kSincPolyA)) {
      const df2 r1 = df_sinc_poly_d(u1), r2 = df_sinc_poly_d(u2);
      smv[l] = r1.v;
      spv[l] = r2.v;
      dsm = r1.d;
      dspl = r2.d;
    } else {
      const cdf ea = df_cis_turns(dfl_mul(W.at, kn), tab);
      const df sak = ea.im, cak = ea.re;
      const df x1 = dfl_mul(W.sa, cak), x2 = dfl_mul(W.ca, sak);
      const df s1 = dfl_sub(x1, x2), s2 = dfl_add(x1, x2);
      const df y1 = dfl_mul(W.ca, cak), y2 = dfl_mul(W.sa, sak);
      const df c1 = dfl_add(y1, y2), c2 = dfl_sub(y1, y2);   // cos u1, cos u2
      const bool small1 = fabsf(u1.x) < 1e-3f, small2 = fabsf(u2.x) < 1e-3f;
      if (!small1 && !small2) {
        const df rr = df_rcp(dfl_mul(u1, u2));
        smv[l] = dfl_mul(dfl_mul(s1, u2), rr);
        spv[l] = dfl_mul(dfl_mul(s2, u1), rr);
        dsm = dfl_mul(dfl_sub(c1, smv[l]), dfl_mul(u2, rr));
        dspl = dfl_mul(dfl_sub(c2, spv[l]), dfl_mul(u1, rr));
      } else {
        if (small1) {
          smv[l] = df_sinc_small(u1);
          dsm = df_dsinc_small(u1);
        } else {
          const df r1 = df_rcp(u1);
          smv[l] = dfl_mul(s1, r1);
          dsm = dfl_mul(dfl_sub(c1, smv[l]), r1);
        }
        if (small2) {
          spv[l] = df_sinc_small(u2);
          dspl = df_dsinc_small(u2);
        } else {
          const df r2 = df_rcp(u2);
          spv[l] = dfl_mul(s2, r2);
          dspl = dfl_mul(dfl_sub(c2, spv[l]), r2);
        }
      }
    }
    df* tl = tp + (kTL + 8 * l) * kTileBins;
    tst(tl + (0), kn, pol);
    tst(tl + (kTileBins), np, pol);
    tst(tl + (2 * kTileBins), nq, pol);
    tst(tl + (3 * kTileBins), inv, pol);
    tst(tl + (4 * kTileBins), smv[l], pol);
    tst(tl + (5 * kTileBins), spv[l], pol);
    tst(tl + (6 * kTileBins), df_neg(dfl_mul(W.a, dsm)), pol);
    tst(tl + (7 * kTileBins), dfl_mul(W.a, dspl), pol);
  }
#pragma unroll
  for (int l = 0; l < 3; ++l) {
    acc.Sr[l] = dfl_add(acc.Sr[l], dfl_mul(G[l].re, spv[l]));
    acc.Si[l] = dfl_add(acc.Si[l], dfl_mul(G[l].im, spv[l]));
    acc.Mr[l] = dfl_add(acc.Mr[l], dfl_mul(G[l].re, smv[l]));
    acc.Mi[l] = dfl_add(acc.Mi[l], dfl_mul(G[l].im, smv[l]));
  }

}

// Double-word copies of what the mode-level chain rule reads: the sample's PN coefficients and
// their derivatives, the orbit rates, and per mode the PN factors and the derivatives of the
// amplitude, v-scale and polarisation weights. Formed once per tile (one sample per tile) by
// chain_fill; the mixed reverse sweep then runs its chain rule on the FP32 pipe.
struct ChainW {
  df Pdd[8], dPq[8], dPdq[8];
  df Q6, dQ5q, dQ6q, dP3c1, dP4c1, dP3c2, dP4c2, dlnAdL;
  df rate, geo_rate;   // pi rate_ht, pi geo_rate_ht (turns of the orbit angles per second, times 2 pi)
  df mfac2[kNModes], mfac[kNModes], tffac[kNModes], lncm[kNModes];
  df dlnAdM[kNModes], dlnAdq[kNModes], dcmdM[kNModes], dPpdi[kNModes], dPcdi[kNModes];
};
constexpr int kChainW = (int)(sizeof(ChainW) / sizeof(df));
__device__ __forceinline__ double chain_value(const DetDev& D, const SampleCoef& S, const SampleGrad& SG, int i) {
  if (i < 8) return S.Pdd[i];
  if (i < 16) return SG.dP_dq[i - 8];
  if (i < 24) return SG.dPd_dq[i - 16];
  switch (i) {
    case 24: return S.Q6;
    case 25: return SG.dQ5_dq;
    case 26: return SG.dQ6_dq;
    case 27: return SG.dP3_dc1;
    case 28: return SG.dP4_dc1;
    case 29: return SG.dP3_dc2;
    case 30: return SG.dP4_dc2;
    case 31: return SG.dlnA_ddL;
    case 32: return kPi * D.rate_ht;
    case 33: return kPi * D.geo_rate_ht;
    default: break;
  }
  const int k = (i - 34) / kNModes, md = (i - 34) % kNModes;
  const ModeCoef& C = S.md[md];
  const ModeGrad& G = SG.md[md];
  switch (k) {
    case 0: return 2.0 * C.mfac;
    case 1: return C.mfac;
    case 2: return C.tffac;
    case 3: return C.lncm;
    case 4: return G.dlnA_dM;
    case 5: return G.dlnA_dq;
    case 6: return G.dcm_dM;
    case 7: return G.dPp_di;
    default: return G.dPc_di;
  }
}
// Every thread of the CTA calls this between barriers; entry i is formed by thread i.
__device__ __forceinline__ void chain_fill(const DetDev& D, const SampleCoef& S, const SampleGrad& SG, ChainW* cw) {
  if (threadIdx.x < kChainW) reinterpret_cast<df*>(cw)[threadIdx.x] = to_dw(chain_value(D, S, SG, threadIdx.x));
}
// Double-word accumulators of the theta components reached per unit (a bin's modes), converted to
// FP64 once per bin.
struct GradAccDW {
  df M, q, c1, c2, dL, io, ph, tc;
};
__device__ __forceinline__ void gaccdw_zero(GradAccDW& a) {
  a.M = a.q = a.c1 = a.c2 = a.dL = a.io = a.ph = a.tc = df_make(0.f, 0.f);
}
__device__ __forceinline__ void gaccdw_flush(const GradAccDW& a, GradAcc& g) {
  g.M += df_to(a.M); g.q += df_to(a.q); g.c1 += df_to(a.c1); g.c2 += df_to(a.c2);
  g.dL += df_to(a.dL); g.io += df_to(a.io); g.ph += df_to(a.ph); g.tc += df_to(a.tc);
}

// link_seeds in double words: bw are the A/E/T cotangents times ihsc, sa, ca the bin's sin a,
// cos a (the T cotangent cancels from the differences exactly, as there).
__device__ __forceinline__ void link_seeds_dw(const cdf bw[3], const df& sa, const df& ca, cdf* seeds) {
  const cdf& bA = bw[0];
  const cdf& bE = bw[1];
  const cdf& bT = bw[2];
  const cdf sX = {dfl_add(dfl_sub(bE.re, bA.re), bT.re), dfl_add(dfl_sub(bE.im, bA.im), bT.im)};
  const cdf sY = {dfl_sub(bT.re, df_scale2(bE.re, 2.0f)), dfl_sub(bT.im, df_scale2(bE.im, 2.0f))};
  const cdf sZ = {dfl_add(dfl_add(bA.re, bE.re), bT.re), dfl_add(dfl_add(bA.im, bE.im), bT.im)};
  const df s2 = df_scale2(sa, 2.0f);
  const cdf zm = {df_neg(dfl_mul(s2, sa)), dfl_mul(s2, ca)};
  const df e3r = dfl_mul(bE.re, df_make(3.f, 0.f)), e3i = dfl_mul(bE.im, df_make(3.f, 0.f));
#pragma unroll
  for (int l = 0; l < 3; ++l) {
    const cdf& sU = (l == 0) ? sX : (l == 1 ? sY : sZ);
    const cdf& sV = (l == 0) ? sY : (l == 1 ? sZ : sX);
    const cdf d = (l == 0) ? cdf{dfl_sub(bA.re, e3r), dfl_sub(bA.im, e3i)}
                : (l == 1) ? cdf{dfl_add(bA.re, e3r), dfl_add(bA.im, e3i)}
                           : cdf{df_scale2(bA.re, -2.0f), df_scale2(bA.im, -2.0f)};
    const cdf a = cdfl_mul(sV, zm), c = cdfl_mul(sU, zm);
    seeds[2 * l * kTileBins] = cdf{dfl_add(d.re, a.re), dfl_add(d.im, a.im)};
    seeds[(2 * l + 1) * kTileBins] = cdf{dfl_sub(d.re, c.re), dfl_sub(d.im, c.im)};
  }
}

// Reverse sweep of one unit from its double-word tape. seeds: the bin's link seeds
// (link_seeds_dw); cw: the tile's ChainW; lnf3: ln(f)/3 of the bin as a double word. Accumulates
// the theta components reached per unit into gw (double words; the taper's rare term into g) and
// writes the nine form cotangents (double words) to the slot's kTfb fields, as mode_bwd_tape.
__device__ __forceinline__ void mode_bwd_tape_mixed(const DetDev& D, const SampleCoef& S, const SampleGrad& SG,
                                                    int md, const BinIn& B, const BinW& W,
                                                    const cdf* __restrict__ seeds, const ChainW& cw, df lnf3,
                                                    GradAccDW& gw, GradAcc& g,
                                                    const float2* __restrict__ pcw, df* tp, int md2,
                                                    unsigned long long pol) {
  const ModeCoef& C = S.md[md];
  const ModeGrad& CG = SG.md[md];
  const df zero = df_make(0.f, 0.f);
  const df A0 = tld(tp + (kTamp0 * kTileBins), pol), A = tld(tp + (kTw * kTileBins), pol);
  // polarisation weights without the amplitude, as the forward pass forms them
  const df vw = dfl_mul(C.cmw, W.f13);
  cdf ap = {C.Ppw, zero}, ac = {C.Pcw, zero};
  if (md2 >= 0) {
    const df v2 = dfl_mul(vw, vw);
    const df kr = dfl_mul(S.k32w[0], v2), ki = dfl_mul(S.k32w[1], v2);
    const ModeCoef& C2 = S.md[md2];
    ap = cdf{dfl_add(C.Ppw, dfl_mul(kr, C2.Ppw)), dfl_mul(ki, C2.Ppw)};
    ac = cdf{dfl_add(C.Pcw, dfl_mul(kr, C2.Pcw)), dfl_mul(ki, C2.Pcw)};
  }
  const cdf Ap = {dfl_mul(A, ap.re), dfl_mul(A, ap.im)}, Ac = {dfl_mul(A, ac.re), dfl_mul(A, ac.im)};
  cdf Apb = {zero, zero}, Acb = {zero, zero};
  df th0b = zero, th1b = zero, th2b = zero;            // spacecraft-angle cotangents (radians)
  df f0k = zero, f0p = zero, f0q = zero, f1k = zero, f1p = zero, f1q = zero;   // link forms 0..5
#pragma unroll 1
  for (int l = 0; l < 3; ++l) {
    const int t = (l == 0) ? 2 : l - 1;
    const cdf P = seeds[2 * l * kTileBins], Q = seeds[(2 * l + 1) * kTileBins];
    const df* tl = tp + (kTL + 8 * l) * kTileBins;
    const df kn = tld(tl, pol), np = tld(tl + kTileBins, pol);
    const df nq = tld(tl + 2 * kTileBins, pol), inv = tld(tl + 3 * kTileBins, pol);
    const df sm = tld(tl + (4 * kTileBins), pol), spl = tld(tl + (5 * kTileBins), pol);
    const df dsm = tld(tl + (6 * kTileBins), pol), dspl = tld(tl + (7 * kTileBins), pol);
    const cdf E = {tld(tp + ((kTE + 2 * t) * kTileBins), pol), tld(tp + ((kTE + 2 * t + 1) * kTileBins), pol)};
    const df Fp = dfl_sub(dfl_mul(np, np), dfl_mul(nq, nq));
    const df Fc = df_scale2(dfl_mul(np, nq), 2.0f);
    const cdf gam = (md2 >= 0) ? cdf{dfl_sub(dfl_mul(Ap.re, Fp), dfl_mul(Ac.im, Fc)),
                                     dfl_add(dfl_mul(Ap.im, Fp), dfl_mul(Ac.re, Fc))}
                               : cdf{dfl_mul(Ap.re, Fp), dfl_mul(Ac.re, Fc)};
    const cdf G = cdf_mul_s(gam, E);
    const cdf Gb = {dfl_add(dfl_mul(sm, P.re), dfl_mul(spl, Q.re)), dfl_add(dfl_mul(sm, P.im), dfl_mul(spl, Q.im))};
    const df smb = dfl_add(dfl_mul(G.re, P.re), dfl_mul(G.im, P.im));
    const df splb = dfl_add(dfl_mul(G.re, Q.re), dfl_mul(G.im, Q.im));
    const df knb = dfl_add(dfl_mul(smb, dsm), dfl_mul(splb, dspl));
    const cdf gamb = cdf_mul_conj(Gb, E);
    const df thb = dfl_sub(dfl_mul(Gb.im, G.re), dfl_mul(Gb.re, G.im));   // Im(Gb conj G)
    if (t == 0) th0b = dfl_add(th0b, thb);
    else if (t == 1) th1b = dfl_add(th1b, thb);
    else th2b = dfl_add(th2b, thb);
    // gam = Fp Ap + i Fc Ac
    Apb = cdf{dfl_add(Apb.re, dfl_mul(gamb.re, Fp)), dfl_add(Apb.im, dfl_mul(gamb.im, Fp))};
    Acb = cdf{dfl_add(Acb.re, dfl_mul(gamb.im, Fc)), dfl_sub(Acb.im, dfl_mul(gamb.re, Fc))};
    const df Fpb = dfl_add(dfl_mul(gamb.re, Ap.re), dfl_mul(gamb.im, Ap.im));
    const df Fcb = dfl_sub(dfl_mul(gamb.im, Ac.re), dfl_mul(gamb.re, Ac.im));
    const df npb = df_scale2(dfl_add(dfl_mul(np, Fpb), dfl_mul(nq, Fcb)), 2.0f);
    const df nqb = df_scale2(dfl_sub(dfl_mul(np, Fcb), dfl_mul(nq, Fpb)), 2.0f);
    // (kn, np, nq) = (knr, npr, nqr) / |n'|
    const df dot = dfl_add(dfl_mul(knb, kn), dfl_add(dfl_mul(npb, np), dfl_mul(nqb, nq)));
    const df rk = dfl_mul(inv, dfl_sub(knb, dfl_mul(kn, dot)));
    const df rp = dfl_mul(inv, dfl_sub(npb, dfl_mul(np, dot)));
    const df rq = dfl_mul(inv, dfl_sub(nqb, dfl_mul(nq, dot)));
    // link 2's projections are minus the sum of links 0 and 1's
    if (l != 1) {
      const df sk = l == 0 ? rk : df_neg(rk), sp = l == 0 ? rp : df_neg(rp), sq = l == 0 ? rq : df_neg(rq);
      f0k = dfl_add(f0k, sk); f0p = dfl_add(f0p, sp); f0q = dfl_add(f0q, sq);
    }
    if (l != 0) {
      const df sk = l == 1 ? rk : df_neg(rk), sp = l == 1 ? rp : df_neg(rp), sq = l == 1 ? rq : df_neg(rq);
      f1k = dfl_add(f1k, sk); f1p = dfl_add(f1p, sp); f1q = dfl_add(f1q, sq);
    }
  }
  // spacecraft angles 2 pi (pf + e_t), e_2 = -(e_0 + e_1), e_t = (f/2) (form 6 + t)
  const df phb = dfl_mul(dfl_add(dfl_add(th0b, th1b), th2b), df_make(6.28318548f, -1.74845553e-07f));   // turns
  const df pif = dfl_mul(W.f, df_make(3.1415927f, -8.742278e-08f));            // pi f
  df fb[9];
  fb[0] = f0k; fb[1] = f0p; fb[2] = f0q; fb[3] = f1k; fb[4] = f1p; fb[5] = f1q;
  fb[6] = dfl_mul(pif, dfl_sub(th0b, th2b));
  fb[7] = dfl_mul(pif, dfl_sub(th1b, th2b));
  const df kxcb = df_neg(dfl_mul(W.f, phb));
  fb[8] = kxcb;
  df obb[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    df a = dfl_add(dfl_mul(fb[6], pcw[45 + m]), dfl_mul(fb[7], pcw[50 + m]));
#pragma unroll
    for (int f = 0; f < 6; ++f) a = dfl_add(a, dfl_mul(fb[f], pcw[5 * f + m]));
    obb[m] = a;
  }
  const df co = tld(tp + (kTco * kTileBins), pol), so = tld(tp + (kTso * kTileBins), pol);
  df tfb;
  if (D.orbit == 0) {
    const df cob = dfl_add(dfl_add(obb[2], dfl_mul(kxcb, pcw[55])),
                           df_scale2(dfl_add(dfl_mul(co, obb[0]), dfl_mul(so, obb[1])), 2.0f));
    const df sob = dfl_add(dfl_add(obb[3], dfl_mul(kxcb, pcw[56])),
                           df_scale2(dfl_sub(dfl_mul(co, obb[1]), dfl_mul(so, obb[0])), 2.0f));
    tfb = dfl_mul(cw.rate, dfl_sub(dfl_mul(co, sob), dfl_mul(so, cob)));
  } else {
    const df c0 = tld(tp + (kTob0 * kTileBins), pol), s0 = tld(tp + (kTob1 * kTileBins), pol);
    const df cob = dfl_mul(kxcb, pcw[55]), sob = dfl_mul(kxcb, pcw[56]);
    tfb = dfl_add(dfl_mul(cw.geo_rate, dfl_sub(dfl_mul(c0, obb[1]), dfl_mul(s0, obb[0]))),
                  dfl_mul(cw.rate, dfl_sub(dfl_mul(co, sob), dfl_mul(so, cob))));
  }
#pragma unroll
  for (int f = 0; f < 9; ++f) tst(tp + ((kTfb + f) * kTileBins), fb[f], pol);
  // ---------------- mode level, in double words (the taper's rare term in FP64)
  const df iv = df_rcp(vw);
  const df lnv = dfl_add(cw.lncm[md], lnf3);
  const df iv2 = dfl_mul(iv, iv);
  const df iv5 = dfl_mul(dfl_mul(iv2, iv2), iv);
  gw.ph = dfl_add(gw.ph, dfl_mul(phb, cw.mfac2[md]));   // d ph0/d phi_c = m/(2 pi)
  gw.tc = dfl_add(gw.tc, dfl_sub(tfb, dfl_mul(W.f, phb)));   // t_f = t_c + ..., frac(f t_c)
  const df psib = df_neg(dfl_mul(cw.mfac[md], phb));
  const df Db = dfl_mul(dfl_mul(tfb, cw.tffac[md]), W.invf);
  df vb = df_make(0.f, 0.f);
  if (A.x != 0.0f) {
    // cotangent of the amplitude (times ihsc), then of ln amp
    const df ampb = dfl_add(dfl_add(dfl_mul(Apb.re, ap.re), dfl_mul(Apb.im, ap.im)),
                            dfl_add(dfl_mul(Acb.re, ac.re), dfl_mul(Acb.im, ac.im)));
    const df lnAb = dfl_mul(ampb, A);
    gw.M = dfl_add(gw.M, dfl_mul(lnAb, cw.dlnAdM[md]));
    gw.q = dfl_add(gw.q, dfl_mul(lnAb, cw.dlnAdq[md]));
    gw.dL = dfl_add(gw.dL, dfl_mul(lnAb, cw.dlnAdL));
    vb = dfl_mul(dfl_mulf(lnAb, (float)C.p), iv);
    if (dlt_pos(C.ftap, B.f)) {
      const double span = C.fend - C.ftap;
      const double zt = span / (C.fend - B.f) - span / (B.f - C.ftap);
      const double w = (zt > 700.0) ? 0.0 : 1.0 / (1.0 + exp(zt));
      const double wb = df_to(dfl_mul(ampb, A0));
      const double zb = -wb * w * (1.0 - w);
      const double fe = C.fend, ft = C.ftap, As = fe - ft;
      const double dz = 0.1 / (fe - B.f) - As / ((fe - B.f) * (fe - B.f)) - 0.1 / (B.f - ft) -
                        0.9 * As / ((B.f - ft) * (B.f - ft));
      g.M = fma(zb * dz, CG.dfend_dM, g.M);
    }
  }
  // Psi_PN(v), D(v): dPsi/dv = D/v, dD/dv = v^-5 ddpol / v + Q6 (2 + ln v)
  df ddpol = cw.Pdd[7];
#pragma unroll
  for (int k = 6; k >= 0; --k) ddpol = dfl_add(dfl_mul(ddpol, vw), cw.Pdd[k]);
  const df dv = tld(tp + (kTdv * kTileBins), pol);
  const df dDdv = dfl_add(dfl_mul(dfl_mul(iv5, ddpol), iv), dfl_mul(cw.Q6, dfl_add(df_make(2.f, 0.f), lnv)));
  vb = dfl_add(vb, dfl_add(dfl_mul(dfl_mul(psib, dv), iv), dfl_mul(Db, dDdv)));
  gw.M = dfl_add(gw.M, dfl_mul(dfl_mul(vb, W.f13), cw.dcmdM[md]));
  // coefficient derivatives in q: Psi_q = v^-5 sum dP_k v^k + ln v (dQ5 + dQ6 v), D_q likewise
  df pq = cw.dPq[7], dq = cw.dPdq[7];
#pragma unroll
  for (int k = 6; k >= 0; --k) {
    pq = dfl_add(dfl_mul(pq, vw), cw.dPq[k]);
    dq = dfl_add(dfl_mul(dq, vw), cw.dPdq[k]);
  }
  const df q6v = dfl_mul(cw.dQ6q, vw);
  const df psiq = dfl_add(dfl_mul(iv5, pq), dfl_mul(lnv, dfl_add(q6v, cw.dQ5q)));
  const df Dq = dfl_add(dfl_mul(iv5, dq), dfl_add(dfl_mul(q6v, dfl_add(df_make(1.f, 0.f), lnv)), cw.dQ5q));
  gw.q = dfl_add(gw.q, dfl_add(dfl_mul(psib, psiq), dfl_mul(Db, Dq)));
  // chi1, chi2 enter P3 (spin-orbit) and P4 (spin-spin): Psi += dP3 v^-2 + dP4 v^-1
  const df pD2 = df_scale2(Db, 2.0f);
  const df t1 = dfl_sub(psib, pD2), t2 = dfl_sub(psib, Db);   // psib - 2 Db (v^-2), psib - Db (v^-1)
  gw.c1 = dfl_add(gw.c1, dfl_add(dfl_mul(dfl_mul(cw.dP3c1, iv2), t1), dfl_mul(dfl_mul(cw.dP4c1, iv), t2)));
  gw.c2 = dfl_add(gw.c2, dfl_add(dfl_mul(dfl_mul(cw.dP3c2, iv2), t1), dfl_mul(dfl_mul(cw.dP4c2, iv), t2)));
  // polarisation weights: cotangents of ap, ac are A Apb, A Acb (true scale)
  const df apbx = dfl_mul(A, Apb.re), acbx = dfl_mul(A, Acb.re);
  gw.io = dfl_add(gw.io, dfl_add(dfl_mul(apbx, cw.dPpdi[md]), dfl_mul(acbx, cw.dPcdi[md])));
  if (md2 >= 0) {
    const df apby = dfl_mul(A, Apb.im), acby = dfl_mul(A, Acb.im);
    const df v2 = dfl_mul(vw, vw);
    const cdf kap = {dfl_mul(S.k32w[0], v2), dfl_mul(S.k32w[1], v2)};
    const ModeCoef& C2 = S.md[md2];
    gw.io = dfl_add(gw.io, dfl_add(dfl_mul(dfl_add(dfl_mul(apbx, kap.re), dfl_mul(apby, kap.im)), cw.dPpdi[md2]),
                                   dfl_mul(dfl_add(dfl_mul(acbx, kap.re), dfl_mul(acby, kap.im)), cw.dPcdi[md2])));
    const cdf kb = {dfl_add(dfl_mul(apbx, C2.Ppw), dfl_mul(acbx, C2.Pcw)),
                    dfl_add(dfl_mul(apby, C2.Ppw), dfl_mul(acby, C2.Pcw))};   // kappa-bar
    // kappa = k32 v^2; only ln(amp2 / amp1) varies with theta (M, q)
    const df lnrb = dfl_mul(v2, dfl_add(dfl_mul(kb.re, S.k32w[0]), dfl_mul(kb.im, S.k32w[1])));
    gw.M = dfl_add(gw.M, dfl_mul(lnrb, dfl_sub(cw.dlnAdM[md2], cw.dlnAdM[md])));
    gw.q = dfl_add(gw.q, dfl_mul(lnrb, dfl_sub(cw.dlnAdq[md2], cw.dlnAdq[md])));
    // d kappa / d v = 2 kappa / v
    gw.M = dfl_add(gw.M, dfl_mul(dfl_mul(df_scale2(dfl_mul(lnrb, iv), 2.0f), W.f13), cw.dcmdM[md]));
  }
}

// Zeroes the contraction fields of a slot no unit used at this bin (double-word tape).
__device__ __forceinline__ void tape_clear_dw(df* tp, unsigned long long pol) {
  const df z = df_make(0.f, 0.f);
  tst(tp + (kTco * kTileBins), z, pol);
  tst(tp + (kTso * kTileBins), z, pol);
  tst(tp + (kTob0 * kTileBins), z, pol);
  tst(tp + (kTob1 * kTileBins), z, pol);
#pragma unroll
  for (int f = 0; f < 9; ++f) tst(tp + ((kTfb + f) * kTileBins), z, pol);
}

// tape_sum on the double-word tape, in double words; the result returns to FP64.
__device__ __forceinline__ double tape_sum_dw(const df* tape, int j, int e0, int e1, bool geo, unsigned act,
                                              unsigned long long pol) {
  int f, m;
  if (j < 30) { f = j / 5; m = j % 5; }
  else if (j < 40) { f = 6 + (j - 30) / 5; m = (j - 30) % 5; }
  else { f = 8; m = j - 38; }
  if (j < 40 && geo && (m == 2 || m == 3)) return 0.0;
  const int bf = m == 0 ? kTob0 : (m == 1 ? kTob1 : (m == 2 ? kTco : kTso));
  const int len = e1 - e0;
  if (len <= 0) return 0.0;
  const int st = j % len;
  auto term = [&](int i, df a) {
    int e = st + i;
    e = e0 + (e >= len ? e - len : e);
    const int slot = (act >> (2 * (e >> 7))) & 3, th = e & (kTileBins - 1);
    const df* col = tape + slot * kTapeF * kTileBins + th;
    const df fv = tld(col + ((kTfb + f) * kTileBins), pol);
    return (m == 4) ? dfl_add(a, fv) : dfl_add(a, dfl_mul(fv, tld(col + (bf * kTileBins), pol)));
  };
  df a0 = df_make(0.f, 0.f), a1 = a0, a2 = a0, a3 = a0;
  int i = 0;
  for (; i + 4 <= len; i += 4) {
    a0 = term(i, a0);
    a1 = term(i + 1, a1);
    a2 = term(i + 2, a2);
    a3 = term(i + 3, a3);
  }
  for (; i < len; ++i) a0 = term(i, a0);
  return df_to(dfl_add(dfl_add(a0, a1), dfl_add(a2, a3)));
}

}  // namespace pe
