// pe_kernels.cu -- CUDA kernels of the log-likelihood hot path (arXiv:2602.12011 Sec. 2):
//   k_grid_tables    row A0: per-bin grid tables of a detector
//   k_psd_model      row A0: analytic A/E/T PSD (Sec. 3.2)
//   k_data_tables    row A0: whitened data/weight tables and per-block <d|d> partials
//   k_sum_parts      fixed-order sum of per-block partials (used for <d|d>)
//   k_prep           row A1: per-sample coefficients and active bin counts per detector
//   k_scan_tiles     tile offsets of the uneven (detector, sample) work list
//   k_dw_tables      row A0: double-word copies of the per-bin and sincos tables (mixed path)
//   k_loglike_fwd    rows A2-A7: persistent fused waveform -> t_f -> orbit -> links -> TDI ->
//                    A/E/T -> PSD-weighted sums, one fixed-order partial per tile (FP64 or
//                    mixed FP64/double-word precision)
//   k_reduce         row A7: fixed-order sums of the partials -> <d|h>, <h|h>, logL
//   k_signal         noise-free A/E/T signal on the grid (per-bin output)
//   k_inject         data = signal + noise scaled by the PSD (Eq. eq_diag_Sigma_to_Sn)
#include <cuda_runtime.h>

#include "pe_device.cuh"
#include "pe_device_f32.cuh"
#include "pe_device_mixed.cuh"
#include "pe_kernels.h"
#include "pe_fault.h"

namespace pe {

// ------------------------------------------------------------------------------------------
// Row A0: grid tables f, f^(1/3), f^(-1/3), ln(f)/3, f^(-7/6), sincos(pi f L), z = e^{-2 pi i f L},
// and fpow [3][nb] = f^(-5/6), f^(-1/2), f^(-5/3) (the amplitude powers f^(-7/6 + p/3), p = 1, 2,
// and v^-5 up to the mode's constant).
// ------------------------------------------------------------------------------------------
__global__ void k_grid_tables(double T, long long k0, int nb, double L, double* f, double* f13, double* fm13,
                              double* lnf3, double* fm76, double* fpow, double2* sca, double2* z) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  const double fb = double(k0 + b) / T;
  const double c = cbrt(fb);
  f[b] = fb;
  f13[b] = c;
  fm13[b] = 1.0 / c;
  lnf3[b] = log(fb) / 3.0;
  fm76[b] = rsqrt(c) / fb;
  fpow[b] = sqrt(c) / fb;
  fpow[nb + b] = rsqrt(fb);
  fpow[2 * nb + b] = 1.0 / (fb * c * c);
  double s, co;
  sincospi(fb * L, &s, &co);
  sca[b] = make_double2(s, co);
  double s2, c2;
  sincospi(2.0 * fb * L, &s2, &c2);
  z[b] = make_double2(c2, -s2);
}

// The (cos, sin)(2 pi j / kSinTab) table of sincos_turns (exact arguments j/(kSinTab/2) half-turns).
__global__ void k_sincos_table(double2* tab) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= kSinTab) return;
  double s, c;
  sincospi(double(j) / (kSinTab / 2), &s, &c);
  tab[j] = make_double2(c, s);
}

// Double words of the mixed-precision path: per bin f, a = pi f L, a/(2 pi), sin a, cos a,
// f^(1/3), f^(-7/6) and z (from the FP64 tables), and the sincos table as (cos hi, cos lo, sin hi,
// sin lo).
__device__ __forceinline__ float2 dw_of(double a) {
  const float h = __double2float_rn(a);
  return make_float2(h, __double2float_rn(a - (double)h));
}
__global__ void k_dw_tables(const double* f, const double* f13, const double* fm76, const double2* sca, const double2* z,
                            const double2* tab, int nb, double L, float2* fw, float2* aw, float2* atw, float2* saw,
                            float2* caw, float2* f13w, float2* fm76w, float4* zw, float4* tabw) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < kSinTab) {
    const float2 c = dw_of(tab[b].x), s = dw_of(tab[b].y);
    tabw[b] = make_float4(c.x, c.y, s.x, s.y);
  }
  if (b >= nb) return;
  fw[b] = dw_of(f[b]);
  aw[b] = dw_of(kPi * f[b] * L);
  atw[b] = dw_of(0.5 * f[b] * L);
  saw[b] = dw_of(sca[b].x);
  caw[b] = dw_of(sca[b].y);
  f13w[b] = dw_of(f13[b]);
  fm76w[b] = dw_of(fm76[b]);
  const float2 zr = dw_of(z[b].x), zi = dw_of(z[b].y);
  zw[b] = make_float4(zr.x, zr.y, zi.x, zi.y);
}

// Largest |Re dg|, |Im dg| and gg of the whitened tables: per-block maxima (mx_part[block][2]),
// then one warp over the blocks (out[2]).
__global__ void k_table_max(const double2* dg, const double* gg, int n, double* mx_part) {
  __shared__ double red[2][kTileBins];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double a = 0.0, g = 0.0;
  if (i < n) {
    a = fmax(fabs(dg[i].x), fabs(dg[i].y));
    g = fabs(gg[i]);
  }
  red[0][threadIdx.x] = a;
  red[1][threadIdx.x] = g;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      red[0][threadIdx.x] = fmax(red[0][threadIdx.x], red[0][threadIdx.x + s]);
      red[1][threadIdx.x] = fmax(red[1][threadIdx.x], red[1][threadIdx.x + s]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    mx_part[blockIdx.x * 2 + 0] = red[0][0];
    mx_part[blockIdx.x * 2 + 1] = red[1][0];
  }
}
__global__ void k_max_parts(const double* part, int n, double* out) {
  for (int c = 0; c < 2; ++c) {
    double m = 0.0;
    for (int i = threadIdx.x; i < n; i += 32) m = fmax(m, part[i * 2 + c]);
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
    if (threadIdx.x == 0) out[c] = m;
  }
}

// Double-word copies of the whitened tables divided by the power-of-two scales: dgw [3][nb] as
// (re hi, re lo, im hi, im lo), ggw [3][nb].
__global__ void k_dw_data(const double2* dg, const double* gg, int n, double inv_dgs, double inv_ggs, float4* dgw,
                          float2* ggw, float2* dgf, float* ggf) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float2 r = dw_of(dg[i].x * inv_dgs), m = dw_of(dg[i].y * inv_dgs);
  dgw[i] = make_float4(r.x, r.y, m.x, m.y);
  ggw[i] = dw_of(gg[i] * inv_ggs);
  dgf[i] = make_float2(r.x, m.x);
  ggf[i] = (float)(gg[i] * inv_ggs);
}

// FP32 copies of the grid tables for the precision study (PE_PREC_FP32).
__global__ void k_f32_tables(const double* f, const double* f13, const double* fm13, const double* lnf3,
                             const double* fm76, const double2* sca, const double2* z, int nb, float* ff, float* f13f,
                             float* fm13f, float* lnf3f, float* fm76f, float2* scaf, float2* zf) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  ff[b] = (float)f[b];
  f13f[b] = (float)f13[b];
  fm13f[b] = (float)fm13[b];
  lnf3f[b] = (float)lnf3[b];
  fm76f[b] = (float)fm76[b];
  scaf[b] = make_float2((float)sca[b].x, (float)sca[b].y);
  zf[b] = make_float2((float)z[b].x, (float)z[b].y);
}

// Analytic PSD (acceleration + OMS noise only): equal-arm TDI-1.5 A/E/T spectra
//   S_A = S_E = 8 sin^2 x [(2 + cos x) S_oms + (6 + 4 cos x + 2 cos 2x) S_acc],
//   S_T = 32 sin^2 x sin^2(x/2) [S_oms + 4 sin^2(x/2) S_acc],   x = 2 pi f L,
// times |1 - z^4|^2 = 4 sin^2(2x) for TDI 2.0. out: [3][nb].
__global__ void k_psd_model(const double* f, int nb, double L, double oms, double acc, int shaping, int tdi_gen,
                            double* out) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  const double fb = f[b];
  const double x = 2.0 * kPi * fb * L;
  const double so = oms * 2.0 * kPi * fb / kC;
  const double sa = acc / (2.0 * kPi * fb * kC);
  double Soms = so * so, Sacc = sa * sa;
  if (shaping) {
    const double r1 = 2e-3 / fb, r2 = 0.4e-3 / fb, r3 = fb / 8e-3;
    Soms *= 1.0 + r1 * r1 * r1 * r1;
    Sacc *= (1.0 + r2 * r2) * (1.0 + r3 * r3 * r3 * r3);
  }
  const double sx = sin(x), cx = cos(x), sh = sin(0.5 * x);
  double SA = 8.0 * sx * sx * ((2.0 + cx) * Soms + (6.0 + 4.0 * cx + 2.0 * cos(2.0 * x)) * Sacc);
  double ST = 32.0 * sx * sx * sh * sh * (Soms + 4.0 * sh * sh * Sacc);
  if (tdi_gen == 20) {
    const double s2 = sin(2.0 * x);
    SA *= 4.0 * s2 * s2;
    ST *= 4.0 * s2 * s2;
  }
  out[b] = SA;
  out[nb + b] = SA;
  out[2 * nb + b] = ST;
}

// Per-bin TDI/transfer factor Q = TDI(z) (-i a) e^{-ia}, a = pi f L, TDI(z) = 1 - z^2 (1.5) or
// (1 - z^2)(1 - z^4) (2.0): X = Q X' for the brackets X' built per mode.
__device__ __forceinline__ double2 transfer_q(double a, double2 sca, double2 z, int tdi_gen) {
  const double2 z2 = cmul(z, z);
  double2 tdi = make_double2(1.0 - z2.x, -z2.y);
  if (tdi_gen == 20) {
    const double2 z4 = cmul(z2, z2);
    tdi = cmul(tdi, make_double2(1.0 - z4.x, -z4.y));
  }
  const double2 ma = make_double2(-a * sca.x, -a * sca.y);  // (-i a)(cos a - i sin a)
  return cmul(tdi, ma);
}

__device__ __constant__ static const double kChanNorm[3] = {0.70710678118654752440, 0.40824829046386301637,
                                                             0.57735026918962576451};

// Whitened tables (row A0): w_c = 4/(S_c T) (Eq. eq_inner_product); dg_c = conj(d_c) w_c Q n_c;
// gg_c = w_c |Q|^2 n_c^2; per-block partials of <d|d>_c = sum_k w_c |d_c|^2 in a fixed tree
// order. data: [3][nb] complex, psd: [3][nb]; dd_part: [gridDim.x][3]; bad: 1 on a bad PSD.
__global__ void k_data_tables(const double* f, const double2* sca, const double2* zt, int nb, double T, double L,
                              int tdi_gen, const double2* data, const double* psd, double2* dg, double* gg,
                              double* dd_part, int* bad) {
  __shared__ double red[3][kTileBins];
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  double ddc[3] = {0.0, 0.0, 0.0};
  if (b < nb) {
    const double2 Q = transfer_q(kPi * f[b] * L, sca[b], zt[b], tdi_gen);
    const double QQ = Q.x * Q.x + Q.y * Q.y;
    for (int c = 0; c < 3; ++c) {
      const double S = psd[c * nb + b];
      if (!(S > 0.0) || !isfinite(S)) {
        *bad = 1;
        dg[c * nb + b] = make_double2(0.0, 0.0);
        gg[c * nb + b] = 0.0;
        continue;
      }
      const double w = 4.0 / (S * T);
      const double2 d = data[c * nb + b];
      ddc[c] = w * (d.x * d.x + d.y * d.y);
      const double2 dw = make_double2(d.x * w * kChanNorm[c], -d.y * w * kChanNorm[c]);
      dg[c * nb + b] = cmul(dw, Q);
      gg[c * nb + b] = w * QQ * kChanNorm[c] * kChanNorm[c];
    }
  }
  for (int c = 0; c < 3; ++c) red[c][threadIdx.x] = ddc[c];
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s)
      for (int c = 0; c < 3; ++c) red[c][threadIdx.x] += red[c][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int c = 0; c < 3; ++c) dd_part[blockIdx.x * 3 + c] = red[c][0];
}

// Fixed-order sum of n partials of width w (single warp, lane-strided then a shuffle tree).
__global__ void k_sum_parts(const double* part, int n, int w, double* out) {
  for (int c = 0; c < w; ++c) {
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += 32) s += part[i * w + c];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) out[c] = s;
  }
}

// ------------------------------------------------------------------------------------------
// Row A1: per-sample coefficients; active bins per (detector, sample): the bins below the
// largest active mode's taper end m F_isco (one extra bin guards the rounding of the bound;
// every unit still checks f < fend of its own mode).
// ------------------------------------------------------------------------------------------
__global__ void k_prep(const double* theta, int B, unsigned mask, DetSet ds, SampleCoef* coef, int* nend,
                       int* status) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= B) return;
  SampleCoef S;
  sample_prep(theta + (size_t)s * PE_NPARAM, mask, S);
  coef[s] = S;
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
  if (status) status[s] = S.valid ? 0 : 1;
}

// Exclusive prefix sum of tiles (TILE bins each) per (detector, sample) pair; off[P] = total tiles.
// One CTA.
template <int TILE>
__global__ void k_scan_tiles(const int* nend, int P, long long* off) {
  __shared__ long long part[1024];
  const int t = threadIdx.x;
  const int chunk = (P + blockDim.x - 1) / blockDim.x;
  const int lo = t * chunk, hi = min(P, lo + chunk);
  long long s = 0;
  for (int i = lo; i < hi; ++i) s += (nend[i] + TILE - 1) / TILE;
  part[t] = s;
  __syncthreads();
  if (t == 0) {
    long long run = 0;
    for (int i = 0; i < (int)blockDim.x; ++i) { long long v = part[i]; part[i] = run; run += v; }
    off[P] = run;
  }
  __syncthreads();
  long long run = part[t];
  for (int i = lo; i < hi; ++i) { off[i] = run; run += (nend[i] + TILE - 1) / TILE; }
}

// pair index p with off[p] <= t < off[p+1]
__device__ __forceinline__ int find_pair(const long long* off, int P, long long t) {
  int lo = 0, hi = P;  // invariant off[lo] <= t < off[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (off[mid] <= t) lo = mid; else hi = mid;
  }
  return lo;
}

// ------------------------------------------------------------------------------------------
// Rows A2-A7: persistent fused kernel. The work list is every (detector, sample) pair's 128-bin
// sub-tiles (off: their offsets per pair); a work item is R consecutive sub-tiles of one pair
// (offi: the items' offsets), and CTAs stride over the items. Per item the CTA forms the pair's
// projection forms once; per sub-tile each thread owns one bin (coalesced), sums the modes' TDI
// brackets in registers, forms A/E/T and the weighted products, and the CTA reduces them in a
// fixed order into part[sub-tile][6] (<d|h>_c, <h|h>_c). The partials are per sub-tile whatever
// R, MINB (resident CTAs per SM requested from the compiler, which sets the register budget) or
// the grid, so the autotuner's choices never change a result. PREC selects the all-FP64 unit, the
// mixed FP64/double-word one (pe_device_mixed.cuh) or the all-FP32 one of the precision study
// (pe_device_f32.cuh).
// ------------------------------------------------------------------------------------------
template <int MINB, int PREC>
__global__ void __launch_bounds__(kTileBins, MINB) k_loglike_fwd(DetSet ds, int B, const SampleCoef* __restrict__ coef,
                                                                 const int* __restrict__ nend,
                                                                 const long long* __restrict__ off,
                                                                 const long long* __restrict__ offi, int R,
                                                                 double* part) {
  __shared__ double red[6][kTileBins + kRedPad];   // block_sum6 staging (as float2 or float rows)
  __shared__ double pc[kProj];    // the item's projection forms (proj_coef)
  __shared__ float2 pcw[kProj];   // the same as double words (mixed) or floats (.x, FP32)
  __shared__ SampleF sf;          // the item's sample coefficients in FP32 (FP32 path)
  __shared__ double2 stab[kSinTab];   // the sincos table (as float4 double words in the mixed path)
  if (PREC == kPrecMixed) {
    float4* t4 = reinterpret_cast<float4*>(stab);
    for (int i = threadIdx.x; i < kSinTab; i += blockDim.x) t4[i] = ds.d[0].sctw[i];
  } else if (PREC == kPrecFP64) {
    for (int i = threadIdx.x; i < kSinTab; i += blockDim.x) stab[i] = ds.d[0].sct[i];
  }
  __syncthreads();
  const int P = ds.ndet * B;
  const long long total = offi[P];
  for (long long t = blockIdx.x; t < total; t += gridDim.x) {
    const int p = find_pair(offi, P, t);
    if (!PE_CHK(p >= 0 && p < P, 1)) continue;              // checked build: uniform over the CTA
    const int I = p / B, s = p - I * B;
    const long long j0 = (t - offi[p]) * R;                 // first sub-tile of the item in the pair
    const long long q0 = off[p] + j0;                       // its index in the partials
    const long long q1 = min(q0 + R, off[p + 1]);
    if (!PE_CHK(q0 >= 0 && q1 <= off[P], 2)) continue;
    const int ne = nend[p];
    const DetDev& D = ds.d[I];
    if (!PE_CHK(ne <= D.nb, 4)) continue;
    const SampleCoef& S = coef[s];
    proj_prologue(D, S, pc);
    if constexpr (PREC == kPrecMixed) {
      if (threadIdx.x < kProj) pcw[threadIdx.x] = to_dw(pc[threadIdx.x]);
      __syncthreads();
      const double ih = S.ihsc;
      const double sd = D.dg_scale * ih, sg = D.gg_scale * ih * ih;
#pragma unroll 1
      for (long long q = q0; q < q1; ++q) {
        const int b = int(j0 + (q - q0)) * kTileBins + threadIdx.x;
        // per bin in double words, times hsc (h) and 1/dg_scale, 1/gg_scale (tables); the
        // sub-tile sums are scaled back in FP64
        df v[6];
#pragma unroll
        for (int i = 0; i < 6; ++i) v[i] = df_make(0.f, 0.f);
        if (b < ne) {
          cdf x[3], o[3];
          bin_xyz_mixed(D, S, b, x, reinterpret_cast<const float4*>(stab), pcw);
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
        if (block_sum6(v, [](df a, df b) { return dfl_add(a, b); }, reinterpret_cast<float2(*)[kTileBins + kRedPad]>(red), &r))
          part[q * 6 + threadIdx.x] = df_to(r) * (threadIdx.x < 3 ? sd : sg);
      }
    } else if constexpr (PREC == kPrecFP32) {
      float* pcf = reinterpret_cast<float*>(pcw);
      if (threadIdx.x < kProj) pcf[threadIdx.x] = (float)pc[threadIdx.x];
      if (threadIdx.x == 0) sample_to_f32(S, sf);
      __syncthreads();
      const double ih = S.ihsc;
      const double sd = D.dg_scale * ih, sg = D.gg_scale * ih * ih;
#pragma unroll 1
      for (long long q = q0; q < q1; ++q) {
        const int b = int(j0 + (q - q0)) * kTileBins + threadIdx.x;
        float v[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (b < ne) {
          float2 o[3];
          bin_aet_f32(D, sf, b, o, pcf);
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            const float2 g = D.dgf[c * D.nb + b];
            v[c] = g.x * o[c].x - g.y * o[c].y;
            v[3 + c] = D.ggf[c * D.nb + b] * (o[c].x * o[c].x + o[c].y * o[c].y);
          }
        }
        float r;
        if (block_sum6(v, [](float a, float b) { return a + b; }, reinterpret_cast<float(*)[kTileBins + kRedPad]>(red), &r))
          part[q * 6 + threadIdx.x] = (double)r * (threadIdx.x < 3 ? sd : sg);
      }
    } else {
#pragma unroll 1
      for (long long q = q0; q < q1; ++q) {
        const int b = int(j0 + (q - q0)) * kTileBins + threadIdx.x;
        double v[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
        if (b < ne) {
          double2 x[3], o[3];
          bin_xyz(D, S, b, x, stab, pc);
          aet_from_xyz(x, o);
          accum_bin(D, b, o, v);
        }
        double r;
        if (block_sum6(v, [](double a, double b) { return a + b; }, red, &r)) part[q * 6 + threadIdx.x] = r;
      }
    }
  }
}

// Row A7: one warp per sample; for each detector a lane-strided, shuffle-tree sum of that
// pair's tile partials (fixed order), then logL = sum_{I,c} (<d|h> - <h|h>/2 - <d|d>/2).
// dhhh: [B][ndet][3][2] or NULL.
__global__ void k_reduce(DetSet ds, int B, const long long* off, const double* part, const SampleCoef* coef,
                         double* logl, double* dhhh) {
  const int ndet = ds.ndet;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= B) return;
  const int s = warp;
  double L = 0.0;
  for (int I = 0; I < ndet; ++I) {
    const int p = I * B + s;
    const long long t0 = off[p], t1 = off[p + 1];
    if (!PE_CHK(t0 >= 0 && t1 <= off[ndet * B], 8)) continue;   // checked build: uniform over the warp
    double v[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (long long t = t0 + lane; t < t1; t += 32)
#pragma unroll
      for (int i = 0; i < 6; ++i) v[i] += part[t * 6 + i];
#pragma unroll
    for (int i = 0; i < 6; ++i)
      for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_down_sync(0xffffffffu, v[i], o);
    if (lane == 0) {
      for (int c = 0; c < 3; ++c) {
        L += v[c] - 0.5 * v[3 + c] - 0.5 * ds.d[I].dd[c];
        if (dhhh) {
          dhhh[(((size_t)s * ndet + I) * 3 + c) * 2 + 0] = v[c];
          dhhh[(((size_t)s * ndet + I) * 3 + c) * 2 + 1] = v[3 + c];
        }
      }
    }
  }
  if (lane == 0) logl[s] = coef[s].valid ? L : -INFINITY;
}

// Noise-free A/E/T signal of one sample on the whole grid: h_c = Q n_c B_c. out: [3][nb].
template <int PREC>
__global__ void k_signal(DetDev D, const SampleCoef* coef, double2* out) {
  __shared__ double pc[kProj];
  __shared__ float2 pcw[kProj];
  __shared__ SampleF sf;
  const SampleCoef& S = coef[0];
  proj_prologue(D, S, pc);
  if (PREC == kPrecMixed && threadIdx.x < kProj) pcw[threadIdx.x] = to_dw(pc[threadIdx.x]);
  if (PREC == kPrecFP32) {
    if (threadIdx.x < kProj) reinterpret_cast<float*>(pcw)[threadIdx.x] = (float)pc[threadIdx.x];
    if (threadIdx.x == 0) sample_to_f32(S, sf);
  }
  __syncthreads();
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= D.nb) return;
  double2 x[3], o[3];
  if (PREC == kPrecMixed) {
    cdf xw[3];
    bin_xyz_mixed(D, S, b, xw, D.sctw, pcw);
    for (int i = 0; i < 3; ++i) x[i] = make_double2(df_to(xw[i].re) * S.ihsc, df_to(xw[i].im) * S.ihsc);
    aet_from_xyz(x, o);
  } else if (PREC == kPrecFP32) {
    float2 of[3];
    bin_aet_f32(D, sf, b, of, reinterpret_cast<const float*>(pcw));
    for (int i = 0; i < 3; ++i) o[i] = make_double2((double)of[i].x * S.ihsc, (double)of[i].y * S.ihsc);
  } else {
    bin_xyz(D, S, b, x, D.sct, pc);
    aet_from_xyz(x, o);
  }
  const double2 Q = transfer_q(kPi * D.f[b] * D.L, D.sca[b], D.z[b], D.tdi_gen);
  for (int c = 0; c < 3; ++c) out[c * D.nb + b] = cscale(cmul(Q, o[c]), kChanNorm[c]);
}

// data_c = h_c + n_c sqrt(S_c T / 4) (Re, Im independent), in place on h. normals may be NULL.
__global__ void k_inject(int nb, double T, const double* psd, const double2* normals, double2* h) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 3 * nb || normals == nullptr) return;
  const double sig = sqrt(psd[i] * T / 4.0);
  const double2 n = normals[i];
  h[i] = make_double2(h[i].x + n.x * sig, h[i].y + n.y * sig);
}

// ------------------------------------------------------------------------------------------
// Host-callable launch wrappers.
// ------------------------------------------------------------------------------------------
cudaError_t launch_grid_tables(double T, long long k0, int nb, double L, double* f, double* f13, double* fm13,
                               double* lnf3, double* fm76, double* fpow, double2* sca, double2* z, cudaStream_t st) {
  k_grid_tables<<<(nb + 127) / 128, 128, 0, st>>>(T, k0, nb, L, f, f13, fm13, lnf3, fm76, fpow, sca, z);
  return pe::launch_status();
}
cudaError_t launch_sincos_table(double2* tab, cudaStream_t st) {
  k_sincos_table<<<(kSinTab + 127) / 128, 128, 0, st>>>(tab);
  return pe::launch_status();
}
cudaError_t launch_psd_model(const double* f, int nb, double L, double oms, double acc, int shaping, int tdi_gen,
                             double* out, cudaStream_t st) {
  k_psd_model<<<(nb + 127) / 128, 128, 0, st>>>(f, nb, L, oms, acc, shaping, tdi_gen, out);
  return pe::launch_status();
}
cudaError_t launch_data_tables(const double* f, const double2* sca, const double2* z, int nb, double T, double L,
                               int tdi_gen, const double2* data, const double* psd, double2* dg, double* gg,
                               double* dd_part, int* bad, int* nblocks, cudaStream_t st) {
  const int g = (nb + kTileBins - 1) / kTileBins;
  *nblocks = g;
  k_data_tables<<<g, kTileBins, 0, st>>>(f, sca, z, nb, T, L, tdi_gen, data, psd, dg, gg, dd_part, bad);
  return pe::launch_status();
}
cudaError_t launch_sum_parts(const double* part, int n, int w, double* out, cudaStream_t st) {
  k_sum_parts<<<1, 32, 0, st>>>(part, n, w, out);
  return pe::launch_status();
}
cudaError_t launch_prep(const double* theta, int B, unsigned mask, const DetSet& ds, SampleCoef* coef, int* nend,
                        int* status, cudaStream_t st) {
  k_prep<<<(B + 63) / 64, 64, 0, st>>>(theta, B, mask, ds, coef, nend, status);
  return pe::launch_status();
}
cudaError_t launch_scan_tiles(const int* nend, int P, long long* off, int tile_bins, cudaStream_t st) {
  switch (tile_bins) {
    case kTileBins: k_scan_tiles<kTileBins><<<1, 1024, 0, st>>>(nend, P, off); break;
    case 2 * kTileBins: k_scan_tiles<2 * kTileBins><<<1, 1024, 0, st>>>(nend, P, off); break;
    case 4 * kTileBins: k_scan_tiles<4 * kTileBins><<<1, 1024, 0, st>>>(nend, P, off); break;
    case 8 * kTileBins: k_scan_tiles<8 * kTileBins><<<1, 1024, 0, st>>>(nend, P, off); break;
    default: return cudaErrorInvalidValue;
  }
  return pe::launch_status();
}
cudaError_t launch_fwd_offsets(const int* nend, int P, long long* off, long long* offi, int R, cudaStream_t st) {
  cudaError_t e = launch_scan_tiles(nend, P, off, kTileBins, st);
  if (e == cudaSuccess && R > 1) e = launch_scan_tiles(nend, P, offi, R * kTileBins, st);
  return e;
}
cudaError_t launch_dw_tables(const double* f, const double* f13, const double* fm76, const double2* sca,
                             const double2* z, const double2* tab, int nb, double L, float2* fw, float2* aw,
                             float2* atw, float2* saw, float2* caw, float2* f13w, float2* fm76w, float4* zw,
                             float4* tabw, cudaStream_t st) {
  const int n = nb > kSinTab ? nb : kSinTab;
  k_dw_tables<<<(n + 127) / 128, 128, 0, st>>>(f, f13, fm76, sca, z, tab, nb, L, fw, aw, atw, saw, caw, f13w, fm76w, zw,
                                               tabw);
  return pe::launch_status();
}
cudaError_t launch_table_max(const double2* dg, const double* gg, int n, double* mx_part, double* out, cudaStream_t st) {
  const int g = (n + kTileBins - 1) / kTileBins;
  k_table_max<<<g, kTileBins, 0, st>>>(dg, gg, n, mx_part);
  k_max_parts<<<1, 32, 0, st>>>(mx_part, g, out);
  return pe::launch_status();
}
cudaError_t launch_dw_data(const double2* dg, const double* gg, int n, double inv_dgs, double inv_ggs, float4* dgw,
                           float2* ggw, float2* dgf, float* ggf, cudaStream_t st) {
  k_dw_data<<<(n + 127) / 128, 128, 0, st>>>(dg, gg, n, inv_dgs, inv_ggs, dgw, ggw, dgf, ggf);
  return pe::launch_status();
}
cudaError_t launch_f32_tables(const double* f, const double* f13, const double* fm13, const double* lnf3,
                              const double* fm76, const double2* sca, const double2* z, int nb, float* ff, float* f13f,
                              float* fm13f, float* lnf3f, float* fm76f, float2* scaf, float2* zf, cudaStream_t st) {
  k_f32_tables<<<(nb + 127) / 128, 128, 0, st>>>(f, f13, fm13, lnf3, fm76, sca, z, nb, ff, f13f, fm13f, lnf3f, fm76f,
                                                 scaf, zf);
  return pe::launch_status();
}
cudaError_t launch_loglike_fwd(const DetSet& ds, int B, const SampleCoef* coef, const int* nend, const long long* off,
                               const long long* offi, int R, double* part, int grid, int prec, cudaStream_t st) {
  return launch_loglike_fwd_variant(kFwdDefaultVariant, prec, ds, B, coef, nend, off, offi, R, part, grid, st);
}

namespace {
template <int MINB, int PREC>
cudaError_t fwd_one(const DetSet& ds, int B, const SampleCoef* coef, const int* nend, const long long* off,
                    const long long* offi, int R, double* part, int grid, cudaStream_t st) {
  k_loglike_fwd<MINB, PREC><<<grid, kTileBins, 0, st>>>(ds, B, coef, nend, off, R > 1 ? offi : off, R, part);
  return pe::launch_status();
}
template <int MINB, int PREC>
int fwd_occ() {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_loglike_fwd<MINB, PREC>, kTileBins, 0) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}
}  // namespace

cudaError_t launch_loglike_fwd_variant(int variant, int prec, const DetSet& ds, int B, const SampleCoef* coef,
                                       const int* nend, const long long* off, const long long* offi, int R,
                                       double* part, int grid, cudaStream_t st) {
  if (R != 1 && R != 2 && R != 4 && R != 8) return cudaErrorInvalidValue;
  switch (variant * 3 + prec) {
    case 0: return fwd_one<2, kPrecFP64>(ds, B, coef, nend, off, offi, R, part, grid, st);
    case 1: return fwd_one<2, kPrecMixed>(ds, B, coef, nend, off, offi, R, part, grid, st);
    case 2: return fwd_one<2, kPrecFP32>(ds, B, coef, nend, off, offi, R, part, grid, st);
    case 3: return fwd_one<3, kPrecFP64>(ds, B, coef, nend, off, offi, R, part, grid, st);
    case 4: return fwd_one<3, kPrecMixed>(ds, B, coef, nend, off, offi, R, part, grid, st);
    case 5: return fwd_one<3, kPrecFP32>(ds, B, coef, nend, off, offi, R, part, grid, st);
    case 6: return fwd_one<4, kPrecFP64>(ds, B, coef, nend, off, offi, R, part, grid, st);
    case 7: return fwd_one<4, kPrecMixed>(ds, B, coef, nend, off, offi, R, part, grid, st);
    case 8: return fwd_one<4, kPrecFP32>(ds, B, coef, nend, off, offi, R, part, grid, st);
    default: return cudaErrorInvalidValue;
  }
}
int fwd_variant_min_blocks(int variant) { return variant == 0 ? 2 : variant == 1 ? 3 : 4; }
int fwd_variant_max_blocks_per_sm(int variant, int prec) {
  switch (variant * 3 + prec) {
    case 0: return fwd_occ<2, kPrecFP64>();
    case 1: return fwd_occ<2, kPrecMixed>();
    case 2: return fwd_occ<2, kPrecFP32>();
    case 3: return fwd_occ<3, kPrecFP64>();
    case 4: return fwd_occ<3, kPrecMixed>();
    case 5: return fwd_occ<3, kPrecFP32>();
    case 6: return fwd_occ<4, kPrecFP64>();
    case 7: return fwd_occ<4, kPrecMixed>();
    case 8: return fwd_occ<4, kPrecFP32>();
    default: return 0;
  }
}
cudaError_t launch_reduce(const DetSet& ds, int B, const long long* off, const double* part, const SampleCoef* coef,
                          double* logl, double* dhhh, cudaStream_t st) {
  const int threads = 128;
  const long long warps = B;
  const int grid = int((warps * 32 + threads - 1) / threads);
  k_reduce<<<grid, threads, 0, st>>>(ds, B, off, part, coef, logl, dhhh);
  return pe::launch_status();
}
cudaError_t launch_signal(const DetDev& D, const SampleCoef* coef, double2* out, int prec, cudaStream_t st) {
  const int g = (D.nb + kTileBins - 1) / kTileBins;
  if (prec == kPrecMixed)
    k_signal<kPrecMixed><<<g, kTileBins, 0, st>>>(D, coef, out);
  else if (prec == kPrecFP32)
    k_signal<kPrecFP32><<<g, kTileBins, 0, st>>>(D, coef, out);
  else
    k_signal<kPrecFP64><<<g, kTileBins, 0, st>>>(D, coef, out);
  return pe::launch_status();
}
cudaError_t launch_inject(int nb, double T, const double* psd, const double2* normals, double2* h, cudaStream_t st) {
  k_inject<<<(3 * nb + 127) / 128, 128, 0, st>>>(nb, T, psd, normals, h);
  return pe::launch_status();
}

// Index-check error word of this file's kernels (checked build; 0 otherwise), cleared when read.
int checked_take_kernels() { return pe_checked_take_local(); }

}  // namespace pe
