// pe_grad.cu -- kernels of the gradient (row G1) and Fisher matrix (row G2) of the Whittle
// log-likelihood (arXiv:2602.12011 Sec. 2.2 and the automatic-differentiation discussion of
// Sec. 2.3), built on the hand-written reverse sweep in pe_adjoint.cuh:
//   k_prep_grad     per-sample coefficients (values) plus their derivatives in theta, the
//                   latter by device dual numbers over the 11 parameters
//   k_grad_fwd_tape FP64, persistent, two 128-thread CTAs per SM (mixed: three): per bin the forward mode sum
//                   writing each unit's tape (the CTA's region of global memory), the cotangents of the A/E/T
//                   sums dL/dB_c = conj(dg_c) - gg_c B_c, one reverse sweep per mode from the
//                   tape, and per tile the contraction of the form cotangents (pe_adjoint_tape.cuh)
//   k_grad_fwd_mixed the same in mixed precision with a double-word tape
//                   (pe_adjoint_tape_mixed.cuh)
//   k_grad_reduce   fixed-order per-sample sums of the tile partials -> logL, grad[11]
//   k_fisher_fwd    per bin six reverse sweeps (Re/Im of X', Y', Z') -> Jacobian J, then
//                   F += sum_c gg_c (J_Re B_c^T J_Re B_c + J_Im B_c^T J_Im B_c)
//   k_fisher_reduce fixed-order per-sample sums -> F[11][11]
#include <cuda_runtime.h>

#include "pe_adjoint.cuh"
#include "pe_adjoint_mixed.cuh"
#include "pe_adjoint_tape.cuh"
#include "pe_adjoint_tape_mixed.cuh"
#include "pe_grad.h"
#include "pe_fault.h"

namespace pe {

constexpr int kGradW = 23;   // per-tile partials: dh[3], hh[3], M q c1 c2 dL io ph tc, k[3] p[3] q[3]
constexpr int kGradV = 14;   // of which reduced by shuffles: dh[3], hh[3], M q c1 c2 dL io ph tc
constexpr int kFisherW = 66; // unique entries of the symmetric 11 x 11 matrix
constexpr int kFisherThreads = 32;

__global__ void k_prep_grad(const double* theta, int B, unsigned mask, DetSet ds, SampleCoef* coef,
                            SampleGrad* sgrad, int* nend, int* status) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= B) return;
  const double* th = theta + (size_t)s * PE_NPARAM;
  const bool valid = theta_valid(th);
  SampleCoef S;
  sample_prep_t<double>(th, valid, mask, S);
  coef[s] = S;
  SampleGrad G;
  {
    Dn td[PE_NPARAM];
    for (int i = 0; i < PE_NPARAM; ++i) td[i] = dvar(th[i], i);
    SampleCoefT<Dn> SD;
    sample_prep_t<Dn>(td, valid, mask, SD);
    for (int k = 0; k < 8; ++k) G.dP_dq[k] = SD.P[k].d[1];
    for (int k = 0; k < 8; ++k) G.dPd_dq[k] = double(k - 5) * G.dP_dq[k];
    G.dQ5_dq = SD.Q5.d[1];
    G.dQ6_dq = SD.Q6.d[1];
    G.dP3_dc1 = SD.P[3].d[2];
    G.dP4_dc1 = SD.P[4].d[2];
    G.dP3_dc2 = SD.P[3].d[3];
    G.dP4_dc2 = SD.P[4].d[3];
    G.dlnA_ddL = -1.0 / th[4];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        G.dk[i][j] = SD.k[i].d[7 + j];
        G.dp[i][j] = SD.p[i].d[7 + j];
        G.dq[i][j] = SD.q[i].d[7 + j];
      }
    for (int md = 0; md < kNModes; ++md) {
      const ModeCoefT<Dn>& C = SD.md[md];
      ModeGrad& M = G.md[md];
      const double a = C.amp.v;
      M.dlnA_dM = (a != 0.0) ? C.amp.d[0] / a : 0.0;
      M.dlnA_dq = (a != 0.0) ? C.amp.d[1] / a : 0.0;
      M.dcm_dM = C.cm.d[0];
      M.dfend_dM = C.fend.d[0];
      M.dPp_di = C.Pp.d[5];
      M.dPc_di = C.Pc.d[5];
    }
  }
  sgrad[s] = G;
  double fmax = 0.0;
  for (int md = 0; md < kNModes; ++md)
    if (S.md[md].active) fmax = fmax > S.md[md].fend ? fmax : S.md[md].fend;
  for (int I = 0; I < ds.ndet; ++I) {
    const DetDev& D = ds.d[I];
    int n = 0;
    if (fmax > 0.0) {
      const double kx = ceil(fmax * D.T) - double(D.k0) + 1.0;
      n = kx <= 0.0 ? 0 : (kx >= double(D.nb) ? D.nb : int(kx));
    }
    nend[I * B + s] = n;
  }
  if (status) status[s] = valid ? 0 : 1;
}

__device__ __forceinline__ int find_pair_g(const long long* off, int P, long long t) {
  int lo = 0, hi = P;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (off[mid] <= t) lo = mid; else hi = mid;
  }
  return lo;
}

// Cotangents of the A/E/T sums of one bin, and the bin's likelihood terms:
//   L_c = Re(dg_c B_c) - gg_c |B_c|^2 / 2  =>  Bbar_c = (dg.x - gg B.x, -dg.y - gg B.y).
// (The brackets' cotangents follow from B_A = Z' - X', B_E = X' - 2Y' + Z', B_T = X' + Y' + Z';
// link_seeds forms what the link sweeps need from them.)
__device__ __forceinline__ void aet_cotangents(const DetDev& D, int b, const double2 o[3], double v6[6],
                                               double2 bb[3]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const double2 g = D.dg[c * D.nb + b];
    const double w = D.gg[c * D.nb + b];
    v6[c] += g.x * o[c].x - g.y * o[c].y;
    v6[3 + c] += w * (o[c].x * o[c].x + o[c].y * o[c].y);
    bb[c] = make_double2(g.x - w * o[c].x, -g.y - w * o[c].y);
  }
}

// Block sum of the kGradV per-thread partials, already stored in red[i][threadIdx.x], through
// shared memory in a fixed order (block_sum6's scheme for 14 rows): thread t < 112 adds entries
// g, g + 8, ..., g + 120 of row i = t / 8 (g = t % 8) into red[i][g]; thread i < 14 then adds
// red[i][0..7] and returns the row's sum (other threads return 0). About 1,800 FP64 additions per
// tile against ~9,000 for a shuffle tree over all lanes. The caller stores the partials and holds
// the barrier before them.
__device__ __forceinline__ double grad_block_sum(double (*red)[kTileBins + kRedPad]) {
  __syncthreads();
  if (threadIdx.x < kGradV * 8) {
    const int i = threadIdx.x >> 3, g = threadIdx.x & 7;
    double s = red[i][g];
#pragma unroll
    for (int k = 1; k < kTileBins / 8; ++k) s += red[i][g + 8 * k];
    red[i][g] = s;   // only this thread touches column g of row i in this step
  }
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x < kGradV) {
    s = red[threadIdx.x][0];
#pragma unroll
    for (int g = 1; g < 8; ++g) s += red[threadIdx.x][g];
  }
  return s;
}

// Mixed-precision gradient with a double-word tape (pe_adjoint_tape_mixed.cuh): per tile the
// mixed-precision forward mode sum writes each unit's tape, the bracket cotangents are formed in
// FP64 from the mode sum, the reverse sweeps read the tape and run in double words (their theta
// components return to FP64 once per bin), and the CTA contracts the form cotangents in double
// words. The 23 partials per tile are the FP64 kernel's.
__global__ void __launch_bounds__(kTileBins, 3) k_grad_fwd_mixed(DetSet ds, int B, const SampleCoef* __restrict__ coef,
                                                              const SampleGrad* __restrict__ sgrad,
                                                              const int* __restrict__ nend,
                                                              const long long* __restrict__ off, double* part,
                                                              double* tape_all) {
  df* tape = reinterpret_cast<df*>(tape_all + (size_t)blockIdx.x * kTapeDoubles);
  __shared__ double red[kGradV][kTileBins + kRedPad];
  __shared__ unsigned tile_used;   // the slots some unit of the tile used
  __shared__ float4 stabw[kSinTab];
  __shared__ cdf lseed[6][kTileBins];   // each thread's link seeds P_l, Q_l (own column)
  __shared__ ChainW cw;                  // the tile's chain-rule coefficients as double words
  __shared__ double pc[kProj];
  __shared__ float2 pcw[kProj];
  __shared__ double sums[3][kTapeSums];
  for (int i = threadIdx.x; i < kSinTab; i += blockDim.x) stabw[i] = ds.d[0].sctw[i];
  __syncthreads();
  const int P = ds.ndet * B;
  const long long total = off[P];
  df* tcol = tape + threadIdx.x;
  const unsigned long long pol = tape_l2_policy();
  for (long long t = blockIdx.x; t < total; t += gridDim.x) {
    const int p = find_pair_g(off, P, t);
    if (!PE_CHK(p >= 0 && p < P && off[p + 1] <= total && nend[p] <= ds.d[p / B].nb, 16)) continue;
    const int I = p / B, s = p - I * B;
    const int b = int(t - off[p]) * kTileBins + threadIdx.x;
    const DetDev& D = ds.d[I];
    if (threadIdx.x == 0) tile_used = 0u;   // the previous tile's readers passed two barriers since
    proj_prologue(D, coef[s], pc);
    if (threadIdx.x < kProj) pcw[threadIdx.x] = to_dw(pc[threadIdx.x]);
    chain_fill(D, coef[s], sgrad[s], &cw);
    __syncthreads();
    double v[kGradV];
#pragma unroll
    for (int i = 0; i < kGradV; ++i) v[i] = 0.0;
    unsigned used = 0;
    if (b < nend[p]) {
      const SampleCoef& S = coef[s];
      const SampleGrad& SG = sgrad[s];
      BinIn Bn;
      load_bin(D, b, S.tc, Bn);
      BinW W;
      load_bin_w(D, b, W);
      const float4 zz = D.zw[b];
      const cdf zw = {df_make(zz.x, zz.y), df_make(zz.z, zz.w)};
      MixAcc xa;
      mix_zero(xa);
#pragma unroll 1
      for (int md = 0; md < kNModes; ++md) {
        if (md == 3 && S.pair32) continue;
        const ModeCoef& C = S.md[md];
        if (!C.active || !dlt_pos(Bn.f, C.fend)) continue;
        const int sl = tape_slot(md);
        mode_fwd_tape_mixed(D, S, C, Bn, W, xa, stabw, pcw, (md == 0 && S.pair32) ? &S.md[3] : nullptr,
                            tcol + sl * kTapeF * kTileBins, pol);
        used |= 1u << sl;
      }
      cdf x[3], od[3];
      mix_final(xa, zw, x);
      aet_from_xyz_dw(x, od);
      double2 o[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) o[c] = make_double2(df_to(od[c].re) * S.ihsc, df_to(od[c].im) * S.ihsc);
      double2 bb[3];
      aet_cotangents(D, b, o, v, bb);
      const double ih = S.ihsc;
      cdf bw[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) bw[c] = cdf{df_from_bits(bb[c].x * ih), df_from_bits(bb[c].y * ih)};
      link_seeds_dw(bw, W.sa, W.ca, &lseed[0][threadIdx.x]);
      const df lnf3 = df_from_bits(Bn.lnf3);
      GradAcc g;
      gacc_zero(g);
      GradAccDW gw;
      gaccdw_zero(gw);
#pragma unroll 1
      for (int md = 0; md < kNModes; ++md) {
        if (md == 3 && S.pair32) continue;
        const ModeCoef& C = S.md[md];
        if (!C.active || !dlt_pos(Bn.f, C.fend)) continue;
        mode_bwd_tape_mixed(D, S, SG, md, Bn, W, &lseed[0][threadIdx.x], cw, lnf3, gw, g, pcw,
                            tcol + tape_slot(md) * kTapeF * kTileBins, (md == 0 && S.pair32) ? 3 : -1, pol);
      }
      gaccdw_flush(gw, g);
      v[6] = g.M; v[7] = g.q; v[8] = g.c1; v[9] = g.c2; v[10] = g.dL; v[11] = g.io; v[12] = g.ph; v[13] = g.tc;
    }
#pragma unroll 1
    for (int sl = 0; sl < kTapeSlots; ++sl)
      if (!(used & (1u << sl))) tape_clear_dw(tcol + sl * kTapeF * kTileBins, pol);
    {
      const unsigned wu = __reduce_or_sync(0xffffffffu, used);
      if ((threadIdx.x & 31) == 0 && wu) atomicOr(&tile_used, wu);
    }
    __syncthreads();   // the tape is complete; the previous tile's readers of red are done
#pragma unroll
    for (int i = 0; i < kGradV; ++i) red[i][threadIdx.x] = v[i];
    // the contraction walks only the slots some unit of the tile used
    const unsigned tu = tile_used;
    unsigned act = 0;
    int nact = 0;
#pragma unroll
    for (int sl = 0; sl < kTapeSlots; ++sl)
      if ((tu >> sl) & 1u) act |= unsigned(sl) << (2 * nact++);
    const int ent = nact * kTileBins;
    if (threadIdx.x < 3 * kTapeSums) {
      const int j = threadIdx.x % kTapeSums, q = threadIdx.x / kTapeSums;
      const int e0 = q * ent / 3, e1 = (q + 1) * ent / 3;
      sums[q][j] = tape_sum_dw(tape, j, e0, e1, D.orbit != 0, act, pol);
    }
    const double a = grad_block_sum(red);
    if (threadIdx.x < kGradV) {
      part[t * kGradW + threadIdx.x] = a;
    } else if (threadIdx.x < kGradW) {
      const int k = threadIdx.x - kGradV;
      double pcb[kTapeSums];
      for (int j = 0; j < kTapeSums; ++j) pcb[j] = sums[0][j] + sums[1][j] + sums[2][j];
      part[t * kGradW + threadIdx.x] = tape_to_frame(D, pcb, k / 3, k % 3);
    }
  }
}

// FP64 gradient with a tape. Per tile: the forward mode sum writes each unit's tape, the bracket
// cotangents follow from the mode sum, the reverse sweeps read the tape and leave the form
// cotangents in it, and the CTA contracts them with the orbit basis (42 sums over the tile's
// 512 (bin, slot) entries, three threads per sum) and maps the sums to the sky frame. The 23
// partials per tile are those of the recomputing kernel.
__global__ void __launch_bounds__(kTileBins, 2) k_grad_fwd_tape(DetSet ds, int B, const SampleCoef* __restrict__ coef,
                                                             const SampleGrad* __restrict__ sgrad,
                                                             const int* __restrict__ nend,
                                                             const long long* __restrict__ off, double* part,
                                                             double* tape_all) {
  double* tape = tape_all + (size_t)blockIdx.x * kTapeDoubles;   // [kTapeSlots][kTapeF][kTileBins]
  __shared__ double red[kGradV][kTileBins + kRedPad];
  __shared__ unsigned tile_used;   // the slots some unit of the tile used
  __shared__ double2 stab[kSinTab];
  __shared__ double2 lseed[6][kTileBins];   // each thread's link seeds P_l, Q_l (own column)
  __shared__ double pc[kProj];
  __shared__ double sums[3][kTapeSums];
  for (int i = threadIdx.x; i < kSinTab; i += blockDim.x) stab[i] = ds.d[0].sct[i];
  __syncthreads();
  const int P = ds.ndet * B;
  const long long total = off[P];
  double* tcol = tape + threadIdx.x;
  const unsigned long long pol = tape_l2_policy();
  for (long long t = blockIdx.x; t < total; t += gridDim.x) {
    const int p = find_pair_g(off, P, t);
    if (!PE_CHK(p >= 0 && p < P && off[p + 1] <= total && nend[p] <= ds.d[p / B].nb, 16)) continue;
    const int I = p / B, s = p - I * B;
    const int b = int(t - off[p]) * kTileBins + threadIdx.x;
    const DetDev& D = ds.d[I];
    if (threadIdx.x == 0) tile_used = 0u;   // the previous tile's readers passed two barriers since
    proj_prologue(D, coef[s], pc);
    double v[kGradV];
#pragma unroll
    for (int i = 0; i < kGradV; ++i) v[i] = 0.0;
    unsigned used = 0;
    if (b < nend[p]) {
      const SampleCoef& S = coef[s];
      const SampleGrad& SG = sgrad[s];
      BinIn Bn;
      load_bin(D, b, S.tc, Bn);
      XYZAcc xa;
      xyz_zero(xa);
#pragma unroll 1
      for (int md = 0; md < kNModes; ++md) {
        if (md == 3 && S.pair32) continue;
        const ModeCoef& C = S.md[md];
        if (!C.active || !dlt_pos(Bn.f, C.fend)) continue;
        const int sl = tape_slot(md);
        mode_fwd_tape(D, S, C, Bn, xa, stab, pc, (md == 0 && S.pair32) ? &S.md[3] : nullptr,
                      tcol + sl * kTapeF * kTileBins, pol);
        used |= 1u << sl;
      }
      double2 x[3], o[3];
      xyz_final(xa, Bn.z, x);
      aet_from_xyz(x, o);
      double2 bb[3];
      aet_cotangents(D, b, o, v, bb);
      link_seeds(bb, Bn.sa, Bn.ca, &lseed[0][threadIdx.x]);
      GradAcc g;
      gacc_zero(g);
#pragma unroll 1
      for (int md = 0; md < kNModes; ++md) {
        if (md == 3 && S.pair32) continue;
        const ModeCoef& C = S.md[md];
        if (!C.active || !dlt_pos(Bn.f, C.fend)) continue;
        mode_bwd_tape(D, S, SG, md, Bn, &lseed[0][threadIdx.x], g, pc,
                      tcol + tape_slot(md) * kTapeF * kTileBins, (md == 0 && S.pair32) ? 3 : -1, pol);
      }
      v[6] = g.M; v[7] = g.q; v[8] = g.c1; v[9] = g.c2; v[10] = g.dL; v[11] = g.io; v[12] = g.ph; v[13] = g.tc;
    }
#pragma unroll 1
    for (int sl = 0; sl < kTapeSlots; ++sl)
      if (!(used & (1u << sl))) tape_clear(tcol + sl * kTapeF * kTileBins, pol);
    {
      const unsigned wu = __reduce_or_sync(0xffffffffu, used);
      if ((threadIdx.x & 31) == 0 && wu) atomicOr(&tile_used, wu);
    }
    __syncthreads();   // the tape is complete; the previous tile's readers of red are done
#pragma unroll
    for (int i = 0; i < kGradV; ++i) red[i][threadIdx.x] = v[i];
    // the contraction walks only the slots some unit of the tile used
    const unsigned tu = tile_used;
    unsigned act = 0;
    int nact = 0;
#pragma unroll
    for (int sl = 0; sl < kTapeSlots; ++sl)
      if ((tu >> sl) & 1u) act |= unsigned(sl) << (2 * nact++);
    const int ent = nact * kTileBins;
    if (threadIdx.x < 3 * kTapeSums) {
      const int j = threadIdx.x % kTapeSums, q = threadIdx.x / kTapeSums;
      const int e0 = q * ent / 3, e1 = (q + 1) * ent / 3;
      sums[q][j] = tape_sum(tape, j, e0, e1, D.orbit != 0, act, pol);
    }
    const double a = grad_block_sum(red);
    if (threadIdx.x < kGradV) {
      part[t * kGradW + threadIdx.x] = a;
    } else if (threadIdx.x < kGradW) {
      const int k = threadIdx.x - kGradV;
      double pcb[kTapeSums];
      for (int j = 0; j < kTapeSums; ++j) pcb[j] = sums[0][j] + sums[1][j] + sums[2][j];
      part[t * kGradW + threadIdx.x] = tape_to_frame(D, pcb, k / 3, k % 3);
    }
  }
}

// One warp per sample: fixed-order sums over each detector's tiles, then logL and grad[11].
__global__ void k_grad_reduce(DetSet ds, int B, const long long* off, const double* part, const SampleCoef* coef,
                              const SampleGrad* sgrad, double* logl, double* grad) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= B) return;
  const int s = warp;
  double acc[kGradW];
  for (int i = 0; i < kGradW; ++i) acc[i] = 0.0;
  double L = 0.0;
  for (int I = 0; I < ds.ndet; ++I) {
    const int p = I * B + s;
    if (!PE_CHK(off[p] >= 0 && off[p + 1] <= off[ds.ndet * B], 32)) continue;
    double v[kGradW];
    for (int i = 0; i < kGradW; ++i) v[i] = 0.0;
    for (long long t = off[p] + lane; t < off[p + 1]; t += 32)
      for (int i = 0; i < kGradW; ++i) v[i] += part[t * kGradW + i];
    for (int i = 0; i < kGradW; ++i)
      for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_down_sync(0xffffffffu, v[i], o);
    if (lane == 0) {
      for (int c = 0; c < 3; ++c) L += v[c] - 0.5 * v[3 + c] - 0.5 * ds.d[I].dd[c];
      for (int i = 6; i < kGradW; ++i) acc[i] += v[i];
    }
  }
  if (lane != 0) return;
  const bool valid = coef[s].valid != 0;
  if (logl) logl[s] = valid ? L : -INFINITY;
  GradAcc g;
  g.M = acc[6]; g.q = acc[7]; g.c1 = acc[8]; g.c2 = acc[9]; g.dL = acc[10]; g.io = acc[11]; g.ph = acc[12];
  g.tc = acc[13];
  for (int i = 0; i < 3; ++i) { g.k[i] = acc[14 + i]; g.p[i] = acc[17 + i]; g.qv[i] = acc[20 + i]; }
  double out[PE_NPARAM];
  gacc_to_theta(g, sgrad[s], out);
  for (int i = 0; i < PE_NPARAM; ++i) grad[(size_t)s * PE_NPARAM + i] = valid ? out[i] : 0.0;
}

// Fisher: one warp per 128-bin tile (four 32-bin passes). Per bin and per seed (Re/Im of X',
// Y', Z') one reverse sweep over the modes gives a Jacobian row; the rows are combined into
// A/E/T and accumulated into the thread's 66 unique entries (kept in shared memory).
__global__ void __launch_bounds__(kFisherThreads) k_fisher_fwd(DetSet ds, int B, const SampleCoef* __restrict__ coef,
                                                              const SampleGrad* __restrict__ sgrad,
                                                              const int* __restrict__ nend,
                                                              const long long* __restrict__ off, double* part) {
  __shared__ double Fs[kFisherW][kFisherThreads];
  __shared__ double Js[6][PE_NPARAM][kFisherThreads];
  const int P = ds.ndet * B;
  const long long total = off[P];
  const int tid = threadIdx.x;
  for (long long t = blockIdx.x; t < total; t += gridDim.x) {
    const int p = find_pair_g(off, P, t);
    if (!PE_CHK(p >= 0 && p < P && off[p + 1] <= total && nend[p] <= ds.d[p / B].nb, 64)) continue;
    const int I = p / B, s = p - I * B;
    const DetDev& D = ds.d[I];
    const SampleCoef& S = coef[s];
    const SampleGrad& SG = sgrad[s];
    for (int i = 0; i < kFisherW; ++i) Fs[i][tid] = 0.0;
    for (int sub = 0; sub < kTileBins / kFisherThreads; ++sub) {
      const int b = int(t - off[p]) * kTileBins + sub * kFisherThreads + tid;
      if (b >= nend[p]) continue;
      BinIn Bn;
      load_bin(D, b, S.tc, Bn);
      for (int j = 0; j < 6; ++j) {
        const double2 one = make_double2((j & 1) ? 0.0 : 1.0, (j & 1) ? 1.0 : 0.0);
        const double2 zero = make_double2(0.0, 0.0);
        const double2 sX = (j / 2 == 0) ? one : zero;
        const double2 sY = (j / 2 == 1) ? one : zero;
        const double2 sZ = (j / 2 == 2) ? one : zero;
        GradAcc g;
        gacc_zero(g);
#pragma unroll 1
        for (int md = 0; md < kNModes; ++md) {
          if (md == 3 && S.pair32) continue;
          if (S.md[md].active && Bn.f < S.md[md].fend)
            mode_bwd(D, S, SG, md, Bn, sX, sY, sZ, g, D.sct, (md == 0 && S.pair32) ? 3 : -1);
        }
        double row[PE_NPARAM];
        gacc_to_theta(g, SG, row);
        for (int i = 0; i < PE_NPARAM; ++i) Js[j][i][tid] = row[i];
      }
      // rows j: 0 Re X', 1 Im X', 2 Re Y', 3 Im Y', 4 Re Z', 5 Im Z'
      for (int c = 0; c < 3; ++c) {
        const double w = D.gg[c * D.nb + b];
        for (int ri = 0; ri < 2; ++ri) {  // real and imaginary part of B_c
          double jr[PE_NPARAM];
          for (int i = 0; i < PE_NPARAM; ++i) {
            const double X = Js[0 + ri][i][tid], Y = Js[2 + ri][i][tid], Z = Js[4 + ri][i][tid];
            jr[i] = (c == 0) ? (Z - X) : (c == 1) ? (X - 2.0 * Y + Z) : (X + Y + Z);
          }
          int e = 0;
          for (int i = 0; i < PE_NPARAM; ++i)
            for (int k = i; k < PE_NPARAM; ++k, ++e) Fs[e][tid] = fma(w * jr[i], jr[k], Fs[e][tid]);
        }
      }
    }
    __syncwarp();
    // fixed-order sum over the 32 threads of each entry
    for (int e = tid; e < kFisherW; e += kFisherThreads) {
      double a = 0.0;
      for (int k = 0; k < kFisherThreads; ++k) a += Fs[e][k];
      part[t * kFisherW + e] = a;
    }
    __syncwarp();
  }
}

__global__ void k_fisher_reduce(DetSet ds, int B, const long long* off, const double* part, const SampleCoef* coef,
                                double* F) {
  const int s = blockIdx.x;
  const int e = threadIdx.x;
  if (s >= B || e >= kFisherW) return;
  double a = 0.0;
  for (int I = 0; I < ds.ndet; ++I) {
    const int p = I * B + s;
    if (!PE_CHK(off[p] >= 0 && off[p + 1] <= off[ds.ndet * B], 128)) continue;
    for (long long t = off[p]; t < off[p + 1]; ++t) a += part[t * kFisherW + e];
  }
  if (!coef[s].valid) a = 0.0;
  int i = 0, k = 0, idx = e;
  while (idx >= PE_NPARAM - i) { idx -= PE_NPARAM - i; ++i; }
  k = i + idx;
  F[(size_t)s * 121 + i * PE_NPARAM + k] = a;
  F[(size_t)s * 121 + k * PE_NPARAM + i] = a;
}

cudaError_t launch_prep_grad(const double* theta, int B, unsigned mask, const DetSet& ds, SampleCoef* coef,
                             SampleGrad* sgrad, int* nend, int* status, cudaStream_t st) {
  k_prep_grad<<<(B + 31) / 32, 32, 0, st>>>(theta, B, mask, ds, coef, sgrad, nend, status);
  return pe::launch_status();
}
cudaError_t launch_grad_fwd(const DetSet& ds, int B, const SampleCoef* coef, const SampleGrad* sgrad, const int* nend,
                            const long long* off, double* part, int grid, bool mixed, double* tape, cudaStream_t st) {
  if (mixed)
    k_grad_fwd_mixed<<<grid, kTileBins, 0, st>>>(ds, B, coef, sgrad, nend, off, part, tape);
  else
    k_grad_fwd_tape<<<grid, kTileBins, 0, st>>>(ds, B, coef, sgrad, nend, off, part, tape);
  return pe::launch_status();
}
cudaError_t launch_grad_reduce(const DetSet& ds, int B, const long long* off, const double* part,
                               const SampleCoef* coef, const SampleGrad* sgrad, double* logl, double* grad,
                               cudaStream_t st) {
  const int threads = 128;
  const int grid = int(((long long)B * 32 + threads - 1) / threads);
  k_grad_reduce<<<grid, threads, 0, st>>>(ds, B, off, part, coef, sgrad, logl, grad);
  return pe::launch_status();
}
cudaError_t launch_fisher_fwd(const DetSet& ds, int B, const SampleCoef* coef, const SampleGrad* sgrad,
                              const int* nend, const long long* off, double* part, int grid, cudaStream_t st) {
  k_fisher_fwd<<<grid, kFisherThreads, 0, st>>>(ds, B, coef, sgrad, nend, off, part);
  return pe::launch_status();
}
cudaError_t launch_fisher_reduce(const DetSet& ds, int B, const long long* off, const double* part,
                                 const SampleCoef* coef, double* F, cudaStream_t st) {
  k_fisher_reduce<<<B, 96, 0, st>>>(ds, B, off, part, coef, F);
  return pe::launch_status();
}
int grad_partial_width() { return kGradW; }
// FP64: two CTAs per SM (230 registers, no spills; three, at 168 registers, ran 0.4 % slower);
// mixed: three (168 registers, a few hundred bytes of spills), which its latency-bound sweep
// prefers (33.6k against 30.9k grad evals/s with two, 33.0k with four)
int grad_tape_ctas_per_sm(bool mixed) { return mixed ? 3 : 2; }
size_t grad_tape_doubles_per_cta() { return (size_t)kTapeDoubles; }
int fisher_partial_width() { return kFisherW; }

// Index-check error word of this file's kernels (checked build; 0 otherwise), cleared when read.
int checked_take_grad() { return pe_checked_take_local(); }

}  // namespace pe
