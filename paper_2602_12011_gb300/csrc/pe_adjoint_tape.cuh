// pe_adjoint_tape.cuh -- FP64 gradient (row G1, arXiv:2602.12011 Sec. 2.2-2.3) of one (sample,
// mode, bin) unit with a tape: the forward pass evaluates the unit exactly as the likelihood's
// forward kernel does (mode_bin: the geometry as projections of the unnormalised link vectors on
// the sample's frame, linear forms in the orbit basis) and also writes the values its reverse
// sweep needs into a per-thread tape; the reverse sweep reads them back instead of recomputing the
// mode.
//
// Why a tape pays on this part: the FP64 pipe retires two operations per SM cycle, 64 times fewer
// than the FP32 pipe, so a value read back from memory costs a small fraction of its
// recomputation. A 128-thread CTA's tape (its 128 bins, up to four unit modes: 148 KB) lives in
// global memory, one region per resident CTA (46 MB for two CTAs on each of 152 SMs), held in L2
// by an evict-last hint on its accesses, so that two CTAs per SM keep two warps per scheduler
// issuing to the FP64 pipe; one CTA per SM with the tape in shared memory left the pipe waiting
// on its own dependent instructions a quarter of the time.
//
// The reverse sweep pulls the bracket cotangents back to the projections' values, then
//   (a) to the orbit basis, the orbit angle and t_f, through the forms' coefficients pc, and
//   (b) to the coefficients pc themselves (linear in the sky frame k, p, q): the cotangent of
//       coefficient m of a form is the sum over the tile's (bin, mode) entries of the form's
//       cotangent times basis element m. That contraction runs once per tile over the tape, and
//       its 42 sums are mapped to k, p, q through the offsets' forms Mo.
#pragma once
#include "pe_adjoint.cuh"

namespace pe {

// Tape of one unit mode: field f of thread i at tape[(slot * kTapeF + f) * kTileBins + i] of the
// CTA's region (coalesced: consecutive threads, consecutive addresses).
// Slots: (2,2) with a paired (3,2), or an unpaired (3,2) (the two exclude each other); (2,1);
// (3,3); (4,4).
constexpr int kTapeSlots = 4;
enum : int {
  kTco = 0, kTso = 1,     // cos, sin of the centre's orbit angle
  kTob0 = 2, kTob1 = 3,   // orbit basis b0, b1 (b2, b3 = cos, sin heliocentric; 0 geocentric)
  kTE = 4,                // e^{2 pi i (phase + theta_t)}, t = 0..2: (re, im) at kTE + 2 t
  kTamp0 = 10,            // amplitude before the taper
  kTw = 11,               // taper weight
  kTdv = 12,              // v dPsi_PN/dv
  kTL = 13,               // link l: kTL + 8 l + {0 kn, 1 np, 2 nq, 3 1/|n'|, 4 s-, 5 s+, 6 ds-/dkn, 7 ds+/dkn}
  kTapeF = 37,
  kTfb = 13,              // after the reverse sweep: the nine form cotangents (over the link fields)
};
constexpr int kTapeDoubles = kTapeSlots * kTapeF * kTileBins;   // per CTA
static_assert(kTL + 8 * 3 == kTapeF, "three links of eight fields close the unit's fields");
static_assert(kTfb + 9 <= kTapeF && kTfb > kTdv, "the form cotangents overwrite only link fields");
static_assert(kTileBins == 128, "tape_sum splits an entry index with a 7-bit shift");
// Tape slot of mode md (an unpaired (3,2) only occurs with (2,2) inactive).
__device__ __forceinline__ int tape_slot(int md) { return md == 4 ? 3 : (md == 3 ? 0 : md); }
// Pairs of the contraction: 30 link-form coefficients (forms 0..5 = k, p, q projections of links
// 0 and 1; coefficients m = 0..4), 10 spacecraft-offset coefficients (forms 6, 7) and the two of
// the centre's Doppler term k.x_c = pc55 cos + pc56 sin.
constexpr int kTapeSums = 42;

// Tape accesses with an L2 eviction-priority hint: the tape's lines are written and read back
// within one tile, while the per-bin tables stream past them, so they are marked to be evicted
// last (createpolicy.fractional.L2::evict_last; a hint only, no lasting state).
__device__ __forceinline__ unsigned long long tape_l2_policy() {
  unsigned long long p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ void tst(double* a, double v, unsigned long long pol) {
  asm volatile("st.global.L2::cache_hint.f64 [%0], %1, %2;" ::"l"(__cvta_generic_to_global(a)), "d"(v), "l"(pol)
               : "memory");
}
__device__ __forceinline__ double tld(const double* a, unsigned long long pol) {
  double v;
  asm volatile("ld.global.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(__cvta_generic_to_global(a)), "l"(pol)
               : "memory");
  return v;
}

// q(x) with d sinc(u)/du = u q(u^2): the derivative of sinc_poly_x<DEG>'s series term by term,
// q(x) = sum_{k=1..DEG} (-1)^k 2k x^(k-1) / (2k+1)!
template <int DEG>
__device__ __forceinline__ double dsinc_poly_x(double x) {
  double q = DEG >= 8 ? 16.0 / 355687428096000.0 : (DEG >= 6 ? 12.0 / 6227020800.0 : 8.0 / 362880.0);
  if (DEG >= 8) {
    q = fma(q, x, -14.0 / 1307674368000.0);
    q = fma(q, x, 12.0 / 6227020800.0);
  }
  if (DEG >= 6) {
    q = fma(q, x, -10.0 / 39916800.0);
    q = fma(q, x, 8.0 / 362880.0);
  }
  q = fma(q, x, -6.0 / 5040.0);
  q = fma(q, x, 4.0 / 120.0);
  return fma(q, x, -2.0 / 6.0);
}

// Forward pass of one unit: mode_bin's arithmetic (same operations, same order) plus the tape.
// tp points at this thread's column of the mode's slot.
__device__ __forceinline__ void mode_fwd_tape(const DetDev& D, const SampleCoef& S, const ModeCoef& C, const BinIn& B,
                                              XYZAcc& acc, const double2* __restrict__ tab,
                                              const double* __restrict__ pc, const ModeCoef* C2, double* tp,
                                              unsigned long long pol) {
  const double v = C.cm * B.f13;
  const double lnv = C.lncm + B.lnf3;
  const double iv5 = C.icm5 * D.fm53[B.b];
  double poly = S.P[7];
  double dpol = S.Pd[7];
#pragma unroll
  for (int k = 6; k >= 0; --k) {
    poly = fma(poly, v, S.P[k]);
    dpol = fma(dpol, v, S.Pd[k]);
  }
  const double q56 = fma(S.Q6, v, S.Q5);
  const double psi_pn = fma(iv5, poly, lnv * q56);
  const double dv = fma(iv5, dpol, fma(S.Q6 * v, lnv, q56));
  const double tf = fma(C.tffac * B.invf, dv, S.tc);
  const double amp0 = C.ampp * (C.p == 0 ? B.fm76 : (C.p == 1 ? D.fm56[B.b] : D.fm12[B.b]));
  double w = 1.0;
  if (dlt_pos(C.ftap, B.f)) {
    const double span = C.fend - C.ftap;
    const double zt = span / (C.fend - B.f) - span / (B.f - C.ftap);
    w = (zt > 700.0) ? 0.0 : 1.0 / (1.0 + exp(zt));
  }
  const double amp = amp0 * w;
  double co, so, ob[4];
  orbit_basis(D, tf, tab, &co, &so, ob);
  const double kxc = fma(pc[55], co, pc[56] * so);
  const double ph = fma(-C.mfac, psi_pn, C.ph0 - B.frc) - B.f * kxc;
  const double phr = ph - rint(ph);
  double2 Ap = make_double2(amp * C.Pp, 0.0), Ac = make_double2(amp * C.Pc2, 0.0);
  if (C2) {
    const double v2 = v * v;
    const double kr = S.k32.x * v2, ki = S.k32.y * v2;
    Ap = make_double2(amp * fma(kr, C2->Pp, C.Pp), amp * (ki * C2->Pp));
    Ac = make_double2(amp * fma(kr, C2->Pc2, C.Pc2), amp * (ki * C2->Pc2));
  }
  double2 E[3];
  {
    const double e0 = B.hf * dot5(pc + 45, ob), e1 = B.hf * dot5(pc + 50, ob);
    sincos_turns_r(phr + e0, tab, &E[0].y, &E[0].x);
    sincos_turns_r(phr + e1, tab, &E[1].y, &E[1].x);
    sincos_turns_r(phr - (e0 + e1), tab, &E[2].y, &E[2].x);
  }
  tst(tp + (kTco * kTileBins), co, pol);
  tst(tp + (kTso * kTileBins), so, pol);
  tst(tp + (kTob0 * kTileBins), ob[0], pol);
  tst(tp + (kTob1 * kTileBins), ob[1], pol);
#pragma unroll
  for (int t = 0; t < 3; ++t) {
    tst(tp + ((kTE + 2 * t) * kTileBins), E[t].x, pol);
    tst(tp + ((kTE + 2 * t + 1) * kTileBins), E[t].y, pol);
  }
  tst(tp + (kTamp0 * kTileBins), amp0, pol);
  tst(tp + (kTw * kTileBins), w, pol);
  tst(tp + (kTdv * kTileBins), dv, pol);
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
    const double inv = rsqrt(fma(knr[l], knr[l], fma(npr[l], npr[l], nqr[l] * nqr[l])));
    const double kn = knr[l] * inv;
    const double np = npr[l] * inv, nq = nqr[l] * inv;
    const double Fp = np * np - nq * nq, Fch = np * nq;
    const double2 gam = C2 ? make_double2(fma(Ap.x, Fp, -Ac.y * Fch), fma(Ap.y, Fp, Ac.x * Fch))
                           : make_double2(Ap.x * Fp, Ac.x * Fch);
    const double2 G = cmul(gam, E[t]);
    // sincs and their derivatives in kn: u1 = a (1 - kn), u2 = a (1 + kn), so
    // d s-/dkn = -a sinc'(u1) = (a^2 kn - a^2) q(u1^2) and d s+/dkn = (a^2 kn + a^2) q(u2^2) on the
    // polynomial branch
    double sm, spl, dsm, dspl;
    if (B.sdeg < 3) {
      const double x1 = fma(kn, fma(B.a2, kn, -B.a2x2), B.a2), x2 = fma(kn, fma(B.a2, kn, B.a2x2), B.a2);
      const double w1 = fma(B.a2, kn, -B.a2), w2 = fma(B.a2, kn, B.a2);
      if (B.sdeg == 0) {
        sm = sinc_poly_x<4>(x1);
        spl = sinc_poly_x<4>(x2);
        dsm = w1 * dsinc_poly_x<4>(x1);
        dspl = w2 * dsinc_poly_x<4>(x2);
      } else if (B.sdeg == 1) {
        sm = sinc_poly_x<6>(x1);
        spl = sinc_poly_x<6>(x2);
        dsm = w1 * dsinc_poly_x<6>(x1);
        dspl = w2 * dsinc_poly_x<6>(x2);
      } else {
        sm = sinc_poly_x<8>(x1);
        spl = sinc_poly_x<8>(x2);
        dsm = w1 * dsinc_poly_x<8>(x1);
        dspl = w2 * dsinc_poly_x<8>(x2);
      }
    } else {
      const double u1 = B.a * (1.0 - kn), u2 = B.a * (1.0 + kn);
      double sak, cak;
      sincos_turns(B.aturn * kn, tab, &sak, &cak);
      const double s1 = B.sa * cak - B.ca * sak, s2 = B.sa * cak + B.ca * sak;
      const double c1u = B.ca * cak + B.sa * sak, c2u = B.ca * cak - B.sa * sak;
      const bool small1 = dlt_pos(fabs(u1), 1e-3), small2 = dlt_pos(fabs(u2), 1e-3);
      if (!small1 && !small2) {
        const double rr = 1.0 / (u1 * u2);
        sm = s1 * u2 * rr;
        spl = s2 * u1 * rr;
      } else {
        sm = small1 ? sinc_small(u1) : s1 / u1;
        spl = small2 ? sinc_small(u2) : s2 / u2;
      }
      dsm = -B.a * dsinc(u1, c1u, sm);
      dspl = B.a * dsinc(u2, c2u, spl);
    }
    acc.S[l].x = fma(G.x, spl, acc.S[l].x);
    acc.S[l].y = fma(G.y, spl, acc.S[l].y);
    acc.M[l].x = fma(G.x, sm, acc.M[l].x);
    acc.M[l].y = fma(G.y, sm, acc.M[l].y);
    double* tl = tp + (kTL + 8 * l) * kTileBins;
    tst(tl + (0), kn, pol);
    tst(tl + (kTileBins), np, pol);
    tst(tl + (2 * kTileBins), nq, pol);
    tst(tl + (3 * kTileBins), inv, pol);
    tst(tl + (4 * kTileBins), sm, pol);
    tst(tl + (5 * kTileBins), spl, pol);
    tst(tl + (6 * kTileBins), dsm, pol);
    tst(tl + (7 * kTileBins), dspl, pol);
  }
}

// The seeds of the link sweeps of one bin. Link l contributes -G U to one bracket (cotangent
// sU) and +G V to the next (cotangent sV), U = s- + z s+, V = s+ + z s-; with Su = -sU:
// Gb = s- P_l + s+ Q_l, d/ds- = Re(G conj P_l), d/ds+ = Re(G conj Q_l), where
// P_l = Su + sV conj z and Q_l = Su conj z + sV depend on the bin only. Pairs: link 0 = (1,2):
// X' and Y'; link 1 = (2,3): Y', Z'; link 2 = (3,1): Z', X'. From the A/E/T cotangents bb
// (sX = -bA + bE + bT, sY = -2 bE + bT, sZ = bA + bE + bT) the differences sV - sU are bA - 3 bE,
// bA + 3 bE and -2 bA: the T cotangent, which dwarfs the others at long wavelength (the T
// channel's noise falls as a^4), cancels exactly, and with conj z - 1 = -2 sin a (sin a - i cos a)
// P_l = (sV - sU) + sV (conj z - 1), Q_l = (sV - sU) - sU (conj z - 1). sa, ca: sin a, cos a.
// Writes P_l, Q_l to pq[(2 l) * kTileBins], pq[(2 l + 1) * kTileBins].
__device__ __forceinline__ void link_seeds(const double2 bb[3], double sa, double ca, double2* pq) {
  const double2 sX = make_double2(-bb[0].x + bb[1].x + bb[2].x, -bb[0].y + bb[1].y + bb[2].y);
  const double2 sY = make_double2(-2.0 * bb[1].x + bb[2].x, -2.0 * bb[1].y + bb[2].y);
  const double2 sZ = make_double2(bb[0].x + bb[1].x + bb[2].x, bb[0].y + bb[1].y + bb[2].y);
  const double2 zm = make_double2(-2.0 * sa * sa, 2.0 * sa * ca);
#pragma unroll
  for (int l = 0; l < 3; ++l) {
    const double2 sU = (l == 0) ? sX : (l == 1 ? sY : sZ);
    const double2 sV = (l == 0) ? sY : (l == 1 ? sZ : sX);
    const double2 d = (l == 0) ? make_double2(bb[0].x - 3.0 * bb[1].x, bb[0].y - 3.0 * bb[1].y)
                    : (l == 1) ? make_double2(bb[0].x + 3.0 * bb[1].x, bb[0].y + 3.0 * bb[1].y)
                               : make_double2(-2.0 * bb[0].x, -2.0 * bb[0].y);
    pq[2 * l * kTileBins] = cadd(d, cmul(sV, zm));
    pq[(2 * l + 1) * kTileBins] = csub(d, cmul(sU, zm));
  }
}

// Reverse sweep of one unit from its tape. seeds: the bin's link seeds (link_seeds). Accumulates the
// theta components reached per unit (Mtot, q, chi1, chi2, dL, iota, phi_c, t_c) into g and writes
// the nine form cotangents to the slot's kTfb fields: links 0 and 1's (k, p, q) projections, the
// two spacecraft-offset phases and the centre's Doppler term.
__device__ __forceinline__ void mode_bwd_tape(const DetDev& D, const SampleCoef& S, const SampleGrad& SG, int md,
                                              const BinIn& B, const double2* __restrict__ seeds, GradAcc& g,
                                              const double* __restrict__ pc, double* tp, int md2,
                                              unsigned long long pol) {
  const ModeCoef& C = S.md[md];
  const ModeGrad& CG = SG.md[md];
  const double v = C.cm * B.f13;
  const double iv = C.icm * B.fm13;
  const double lnv = C.lncm + B.lnf3;
  const double iv5 = C.icm5 * D.fm53[B.b];
  const double amp0 = tld(tp + (kTamp0 * kTileBins), pol), w = tld(tp + (kTw * kTileBins), pol);
  const double amp = amp0 * w;
  // polarisation weights without the amplitude: ap = Pp + kappa Pp', ac = 2 Pc + kappa 2 Pc'
  double2 kap = make_double2(0.0, 0.0);
  double Pp2 = 0.0, Pc22 = 0.0;
  if (md2 >= 0) {
    kap = make_double2(S.k32.x * v * v, S.k32.y * v * v);
    Pp2 = S.md[md2].Pp;
    Pc22 = S.md[md2].Pc2;
  }
  const double2 ap = make_double2(fma(kap.x, Pp2, C.Pp), kap.y * Pp2);
  const double2 ac = make_double2(fma(kap.x, Pc22, C.Pc2), kap.y * Pc22);
  const double2 Ap = make_double2(amp * ap.x, amp * ap.y), Ac = make_double2(amp * ac.x, amp * ac.y);
  double2 Apb = make_double2(0.0, 0.0), Acb = make_double2(0.0, 0.0);
  double thb[3];                    // cotangents of the spacecraft angles 2 pi (phase + theta_t)
  double krb[3], prb[3], qrb[3];    // cotangents of the unnormalised projections, per link
#pragma unroll
  for (int l = 0; l < 3; ++l) {
    const int t = (l + 2) % 3;
    const double2 P = seeds[2 * l * kTileBins], Q = seeds[(2 * l + 1) * kTileBins];
    const double* tl = tp + (kTL + 8 * l) * kTileBins;
    const double kn = tld(tl + (0), pol), np = tld(tl + (kTileBins), pol), nq = tld(tl + (2 * kTileBins), pol), inv = tld(tl + (3 * kTileBins), pol);
    const double sm = tld(tl + (4 * kTileBins), pol), spl = tld(tl + (5 * kTileBins), pol);
    const double dsm = tld(tl + (6 * kTileBins), pol), dspl = tld(tl + (7 * kTileBins), pol);
    const double2 E = make_double2(tld(tp + ((kTE + 2 * t) * kTileBins), pol), tld(tp + ((kTE + 2 * t + 1) * kTileBins), pol));
    const double Fp = np * np - nq * nq, Fch = np * nq;
    const double2 gam = make_double2(fma(Ap.x, Fp, -Ac.y * Fch), fma(Ap.y, Fp, Ac.x * Fch));
    const double2 G = cmul(gam, E);
    const double2 Gb = make_double2(fma(sm, P.x, spl * Q.x), fma(sm, P.y, spl * Q.y));
    const double smb = fma(G.x, P.x, G.y * P.y);
    const double splb = fma(G.x, Q.x, G.y * Q.y);
    const double knb = fma(smb, dsm, splb * dspl);
    const double2 gamb = cconjmul(Gb, E);
    thb[t] = fma(Gb.y, G.x, -Gb.x * G.y);   // Im(Gb conj G): the angle's cotangent (G = gam E)
    // gam = Fp Ap + i Fch Ac
    Apb = make_double2(fma(gamb.x, Fp, Apb.x), fma(gamb.y, Fp, Apb.y));
    Acb = make_double2(fma(gamb.y, Fch, Acb.x), fma(-gamb.x, Fch, Acb.y));
    const double Fpb = fma(gamb.x, Ap.x, gamb.y * Ap.y), Fchb = fma(gamb.y, Ac.x, -gamb.x * Ac.y);
    const double npb = fma(2.0 * np, Fpb, nq * Fchb);
    const double nqb = fma(-2.0 * nq, Fpb, np * Fchb);
    // (kn, np, nq) = (knr, npr, nqr) / |n'|
    const double dot = fma(knb, kn, fma(npb, np, nqb * nq));
    krb[l] = inv * fma(-kn, dot, knb);
    prb[l] = inv * fma(-np, dot, npb);
    qrb[l] = inv * fma(-nq, dot, nqb);
  }
  // link 2's projections are minus the sum of links 0 and 1's
  double fb[9];
  fb[0] = krb[0] - krb[2]; fb[1] = prb[0] - prb[2]; fb[2] = qrb[0] - qrb[2];
  fb[3] = krb[1] - krb[2]; fb[4] = prb[1] - prb[2]; fb[5] = qrb[1] - qrb[2];
  // spacecraft angles 2 pi (phr + e_t), e_2 = -(e_0 + e_1), e_t = (f/2) (form 6 + t)
  const double phb = 2.0 * kPi * (thb[0] + thb[1] + thb[2]);   // cotangent of the phase (turns)
  fb[6] = kPi * B.f * (thb[0] - thb[2]);
  fb[7] = kPi * B.f * (thb[1] - thb[2]);
  const double kxcb = -B.f * phb;
  fb[8] = kxcb;
  // orbit basis through the forms' coefficients
  double obb[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    double a = fb[7] * pc[50 + m];
    a = fma(fb[6], pc[45 + m], a);
#pragma unroll
    for (int f = 5; f >= 0; --f) a = fma(fb[f], pc[5 * f + m], a);
    obb[m] = a;
  }
  const double co = tld(tp + (kTco * kTileBins), pol), so = tld(tp + (kTso * kTileBins), pol);
  double tfb;
  if (D.orbit == 0) {
    // b = (cos 2a, sin 2a, cos a, sin a)
    const double cob = fma(2.0 * co, obb[0], fma(2.0 * so, obb[1], fma(kxcb, pc[55], obb[2])));
    const double sob = fma(-2.0 * so, obb[0], fma(2.0 * co, obb[1], fma(kxcb, pc[56], obb[3])));
    tfb = kPi * D.rate_ht * (co * sob - so * cob);
  } else {
    // b = (cos phi_0, sin phi_0, 0, 0); the centre keeps its heliocentric angle
    const double c0 = tld(tp + (kTob0 * kTileBins), pol), s0 = tld(tp + (kTob1 * kTileBins), pol);
    const double cob = kxcb * pc[55], sob = kxcb * pc[56];
    tfb = kPi * D.geo_rate_ht * (c0 * obb[1] - s0 * obb[0]) + kPi * D.rate_ht * (co * sob - so * cob);
  }
#pragma unroll
  for (int f = 0; f < 9; ++f) tst(tp + ((kTfb + f) * kTileBins), fb[f], pol);
  // ---------------- mode level
  g.ph = fma(phb, 2.0 * C.mfac, g.ph);          // d ph0/d phi_c = m/(2 pi)
  g.tc = fma(-B.f, phb, g.tc);                   // frac(f t_c)
  const double psib = -C.mfac * phb;
  g.tc += tfb;                                   // t_f = t_c + (m/(12 pi f)) D(v)
  const double Db = tfb * C.tffac * B.invf;
  double vb = 0.0;
  if (dlt_pos(0.0, amp)) {
    const double ampb = fma(Apb.x, ap.x, fma(Apb.y, ap.y, fma(Acb.x, ac.x, Acb.y * ac.y)));
    const double lnAb = ampb * amp;
    g.M = fma(lnAb, CG.dlnA_dM, g.M);
    g.q = fma(lnAb, CG.dlnA_dq, g.q);
    g.dL = fma(lnAb, SG.dlnA_ddL, g.dL);
    vb = lnAb * double(C.p) * iv;
    if (dlt_pos(C.ftap, B.f)) {
      const double wb = ampb * amp0;
      const double zb = -wb * w * (1.0 - w);
      const double fe = C.fend, ft = C.ftap, A = fe - ft;
      const double dz = 0.1 / (fe - B.f) - A / ((fe - B.f) * (fe - B.f)) - 0.1 / (B.f - ft) -
                        0.9 * A / ((B.f - ft) * (B.f - ft));
      g.M = fma(zb * dz, CG.dfend_dM, g.M);
    }
  }
  double ddpol = S.Pdd[7];
#pragma unroll
  for (int k = 6; k >= 0; --k) ddpol = fma(ddpol, v, S.Pdd[k]);
  // Psi_PN(v), D(v): dPsi/dv = D/v, dD/dv = v^-5 ddpol / v + Q6 (2 + ln v)
  const double dv = tld(tp + (kTdv * kTileBins), pol);
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
  // polarisation weights: cotangents of ap, ac are amp Apb, amp Acb; ac carries 2 Pc
  const double2 apb = make_double2(amp * Apb.x, amp * Apb.y), acb = make_double2(amp * Acb.x, amp * Acb.y);
  g.io += apb.x * CG.dPp_di + 2.0 * acb.x * CG.dPc_di;
  if (md2 >= 0) {
    const ModeGrad& CG2 = SG.md[md2];
    g.io += (apb.x * kap.x + apb.y * kap.y) * CG2.dPp_di + 2.0 * (acb.x * kap.x + acb.y * kap.y) * CG2.dPc_di;
    const double2 kb = make_double2(apb.x * Pp2 + acb.x * Pc22, apb.y * Pp2 + acb.y * Pc22);   // kappa-bar
    // kappa = k32 v^2; only ln(amp2 / amp1) varies with theta (M, q), see mode_bwd
    const double lnrb = v * v * (kb.x * S.k32.x + kb.y * S.k32.y);
    g.M = fma(lnrb, CG2.dlnA_dM - CG.dlnA_dM, g.M);
    g.q = fma(lnrb, CG2.dlnA_dq - CG.dlnA_dq, g.q);
    const double vkb = 2.0 * lnrb / v;
    g.M = fma(vkb * B.f13, CG.dcm_dM, g.M);
  }
}

// Zeroes the contraction fields (form cotangents and basis) of a slot no unit used at this bin.
__device__ __forceinline__ void tape_clear(double* tp, unsigned long long pol) {
  tst(tp + (kTco * kTileBins), 0.0, pol);
  tst(tp + (kTso * kTileBins), 0.0, pol);
  tst(tp + (kTob0 * kTileBins), 0.0, pol);
  tst(tp + (kTob1 * kTileBins), 0.0, pol);
#pragma unroll
  for (int f = 0; f < 9; ++f) tst(tp + ((kTfb + f) * kTileBins), 0.0, pol);
}

// One of the 42 contraction sums over entries [e0, e1) of the tile's tape (entry e = slot * 128 +
// thread): sum j pairs a form's cotangent with one basis element (j < 30: link forms, coefficient
// j % 5; 30..39: spacecraft forms; 40, 41: the centre term's cos, sin). Each sum starts at entry
// e0 + j (neighbouring lanes read neighbouring threads' columns) and runs in a fixed order.
// act: the tile's active slots, two bits each in order (entry e is in slot (act >> 2 (e >> 7)) & 3):
// slots no unit of the tile used hold only zeros and are skipped.
__device__ __forceinline__ double tape_sum(const double* tape, int j, int e0, int e1, bool geo, unsigned act,
                                           unsigned long long pol) {
  int f, m;
  if (j < 30) { f = j / 5; m = j % 5; }
  else if (j < 40) { f = 6 + (j - 30) / 5; m = (j - 30) % 5; }
  else { f = 8; m = j - 38; }          // cos, sin: the centre's angle in either orbit
  if (j < 40 && geo && (m == 2 || m == 3)) return 0.0;
  const int bf = m == 0 ? kTob0 : (m == 1 ? kTob1 : (m == 2 ? kTco : kTso));
  const int len = e1 - e0;
  if (len <= 0) return 0.0;
  const int st = j % len;
  // four interleaved partial sums (a fixed order) keep four independent FMA chains in flight
  auto term = [&](int i, double a) {
    int e = st + i;
    e = e0 + (e >= len ? e - len : e);
    const int slot = (act >> (2 * (e >> 7))) & 3, th = e & (kTileBins - 1);
    const double* col = tape + slot * kTapeF * kTileBins + th;
    const double fv = tld(col + ((kTfb + f) * kTileBins), pol);
    return (m == 4) ? a + fv : fma(fv, tld(col + (bf * kTileBins), pol), a);
  };
  double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
  int i = 0;
  for (; i + 4 <= len; i += 4) {
    a0 = term(i, a0);
    a1 = term(i + 1, a1);
    a2 = term(i + 2, a2);
    a3 = term(i + 3, a3);
  }
  for (; i < len; ++i) a0 = term(i, a0);
  const double r = (a0 + a1) + (a2 + a3);
  return r;
}

// Maps the contraction sums (cotangents of the coefficients pc) to the sky frame: component c of
// k (vec 0), p (1) or q (2). pc[15 l + 5 vec + m] = w_vec . (Mo[l] - Mo[l+1])[., m] (links 0, 1),
// pc[45 + 5 e + m] = k . Mo[e][., m], pc55 = R k_x, pc56 = R k_y.
__device__ __forceinline__ double tape_to_frame(const DetDev& D, const double* pcb, int vec, int c) {
  double a = 0.0;
#pragma unroll 1
  for (int l = 0; l < 2; ++l)
    for (int m = 0; m < 5; ++m) a = fma(pcb[15 * l + 5 * vec + m], D.Mo[l][c][m] - D.Mo[l + 1][c][m], a);
  if (vec == 0) {
#pragma unroll 1
    for (int e = 0; e < 2; ++e)
      for (int m = 0; m < 5; ++m) a = fma(pcb[30 + 5 * e + m], D.Mo[e][c][m], a);
    if (c < 2) a = fma(pcb[40 + c], D.R, a);
  }
  return a;
}

}  // namespace pe
