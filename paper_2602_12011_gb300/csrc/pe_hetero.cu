// pe_hetero.cu -- heterodyned (relative-binning) log-likelihood (the heterodyning idea of Sec. 1,
// in the per-mode relative-binning form of Zackay, Dai & Venumadhav 2018 / Leslie, Dai & Pratten
// 2021): host edge construction, summary-data kernels and the per-sample kernel, plus the C ABI.
//
//   k_mode_brackets  reference per-mode A/E/T brackets on the fine bins [0, K) (creation)
//   k_het_summary    per coarse bin: A_o (o = 0, 1) and B_o (o = 0, 1, 2) by sequential sums
//   k_het_loglike    one CTA per sample: ratios at every edge of every detector (shared memory),
//                    then the per-bin contraction and a fixed-order block reduction
//
// The brackets B_c (A/E/T combinations of X', Y', Z' before the factor Q n_c) stand for the channel
// signals: ratios are the same, and dg = conj(d) w Q n_c, gg = w |Q|^2 n_c^2 supply the rest.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <set>
#include <vector>

#include "pe_device.cuh"
#include "pe_device_mixed.cuh"
#include "pe_internal.h"
#include "pe_kernels.h"
#include "pespace_gb300.h"
#include "pe_fault.h"

namespace pe {

constexpr int kHetMaxEdges = 640;
constexpr int kPairs = kNModes * (kNModes + 1) / 2;   // unordered mode pairs (md <= md2)

__host__ __device__ constexpr int pair_index(int a, int b) {   // a <= b
  return a * kNModes - a * (a - 1) / 2 + (b - a);
}

struct HetDev {
  DetDev det;
  const int* edge;       // [ne] fine-bin indices
  const double* fe;      // [ne] edge frequencies
  const double2* ih0e;   // [ne][5][3] inverses 1/h0 of the reference brackets at the edges (0 where h0 = 0)
  const int* src;        // [ne][5][3] edge whose ratio applies (carry-forward), -1 for none
  const double2* A;      // [ne-1][5][3][2]
  const double2* Bs;     // [ne-1][kPairs][3][3]
  const float4* Aw;      // A and Bs as double words (re hi, re lo, im hi, im lo), for the mixed kernel
  const float4* Bw;
  int ne;
  unsigned mask;
};
struct HetSet {
  HetDev h[kMaxDet];
  int n;
  int nemax;   // largest ne of the set (rows of the kernel's ratio table)
};

__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }

// Per-mode brackets of one sample at bin b (zero for inactive modes or bins past a mode's end).
__device__ __forceinline__ void mode_brackets(const DetDev& D, const SampleCoef& S, int b, unsigned mask,
                                              double2 o[kNModes][3], const double2* __restrict__ tab,
                                              const double* __restrict__ pc) {
  BinIn Bn;
  load_bin(D, b, S.tc, Bn);
#pragma unroll 1
  for (int md = 0; md < kNModes; ++md) {
    const ModeCoef& C = S.md[md];
    XYZAcc a;
    xyz_zero(a);
    if ((mask >> md) & 1u && C.active && Bn.f < C.fend) mode_bin(D, S, C, Bn, a, tab, pc);
    double2 x[3];
    xyz_final(a, Bn.z, x);
    aet_from_xyz(x, o[md]);
  }
}

// The same with the mixed-precision unit (FP64 phase, t_f and turn reductions; double-word
// geometry), each mode's brackets returned to FP64.
__device__ __forceinline__ void mode_brackets_mixed(const DetDev& D, const SampleCoef& S, int b, unsigned mask,
                                                    double2 o[kNModes][3], const float4* __restrict__ tab,
                                                    const float2* __restrict__ pcw) {
  BinIn Bn;
  load_bin(D, b, S.tc, Bn);
  BinW W;
  load_bin_w(D, b, W);
  const float4 zz = D.zw[b];
  const cdf z = {df_make(zz.x, zz.y), df_make(zz.z, zz.w)};
#pragma unroll 1
  for (int md = 0; md < kNModes; ++md) {
    const ModeCoef& C = S.md[md];
    MixAcc a;
    mix_zero(a);
    if ((mask >> md) & 1u && C.active && Bn.f < C.fend) mode_bin_mixed(D, S, C, Bn, W, a, tab, pcw);
    cdf x[3], od[3];
    mix_final(a, z, x);
    aet_from_xyz_dw(x, od);
    for (int c = 0; c < 3; ++c) o[md][c] = make_double2(df_to(od[c].re) * S.ihsc, df_to(od[c].im) * S.ihsc);
  }
}

// Reference per-mode brackets on bins [0, K): out[(md*3 + c)*K + k].
__global__ void k_mode_brackets(DetDev D, const SampleCoef* coef, int K, unsigned mask, double2* out) {
  __shared__ double pc[kProj];
  const SampleCoef& S = coef[0];
  proj_prologue(D, S, pc);
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= K) return;
  double2 o[kNModes][3];
  mode_brackets(D, S, k, mask, o, D.sct, pc);
  for (int md = 0; md < kNModes; ++md)
    for (int c = 0; c < 3; ++c) out[((size_t)md * 3 + c) * K + k] = o[md][c];
}

// h0e[(i*5 + md)*3 + c] = reference bracket (md, c) at edge i
__global__ void k_gather_edges(const double2* hb, int K, const int* edge, int ne, double2* h0e) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= ne * kNModes * 3) return;
  const int i = j / (kNModes * 3), mc = j % (kNModes * 3);
  h0e[j] = hb[(size_t)mc * K + edge[i]];
}

// h0e -> 1/h0e in place; 0 where |h0e|^2 is 0 (h0e = 0, never a ratio source, or so small that its
// square underflows, where the ratio becomes 0 instead of the overflow a division would give)
__global__ void k_invert_edges(double2* h0e, int n) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const double2 h = h0e[j];
  const double den = h.x * h.x + h.y * h.y;
  h0e[j] = den != 0.0 ? make_double2(h.x / den, -h.y / den) : make_double2(0.0, 0.0);
}

// Summary data: one thread per (coarse bin, quantity); a sequential sum over the bin's fine bins.
// Quantities per bin: A: 5 modes x 3 channels x 2 orders; B: kPairs x 3 x 3 orders.
__global__ void k_het_summary(DetDev D, const int* edge, const double* fe, int ne, const double2* h0, int K,
                              double2* A, double2* Bs) {
  constexpr int nA = kNModes * 3 * 2, nB = kPairs * 3 * 3;
  const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int nbin = ne - 1;
  if (id >= (long long)nbin * (nA + nB)) return;
  const int b = (int)(id / (nA + nB)), q = (int)(id % (nA + nB));
  const int lo = edge[b], hi = edge[b + 1] + (b == nbin - 1 ? 1 : 0);
  double2 acc = make_double2(0.0, 0.0);
  if (q < nA) {
    const int md = q / 6, c = (q / 2) % 3, o = q % 2;
    const double2* h = h0 + ((size_t)md * 3 + c) * K;
    for (int k = lo; k < hi; ++k) {
      const double df = D.f[k] - fe[b];
      const double2 t = cmul(D.dg[c * D.nb + k], h[k]);   // conj(d) w Q n_c B0
      const double s = (o == 0) ? 1.0 : df;
      acc.x = fma(t.x, s, acc.x);
      acc.y = fma(t.y, s, acc.y);
    }
    A[(((size_t)b * kNModes + md) * 3 + c) * 2 + o] = acc;
  } else {
    const int r = q - nA;
    const int p = r / 9, c = (r / 3) % 3, o = r % 3;
    int m1 = 0, m2 = 0;
    for (int a = 0; a < kNModes; ++a)
      for (int bb = a; bb < kNModes; ++bb)
        if (pair_index(a, bb) == p) { m1 = a; m2 = bb; }
    const double2* h1 = h0 + ((size_t)m1 * 3 + c) * K;
    const double2* h2 = h0 + ((size_t)m2 * 3 + c) * K;
    for (int k = lo; k < hi; ++k) {
      const double df = D.f[k] - fe[b];
      const double s = D.gg[c * D.nb + k] * (o == 0 ? 1.0 : (o == 1 ? df : df * df));
      const double2 t = cmul(h1[k], cconj(h2[k]));
      acc.x = fma(t.x, s, acc.x);
      acc.y = fma(t.y, s, acc.y);
    }
    Bs[(((size_t)b * kPairs + p) * 3 + c) * 3 + o] = acc;
  }
}

// double2 -> double-word complex (re hi, re lo, im hi, im lo)
__global__ void k_to_dw4(const double2* in, long long n, float4* out) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float2 re = to_dw(in[i].x), im = to_dw(in[i].y);
  out[i] = make_float4(re.x, re.y, im.x, im.y);
}

__device__ __forceinline__ cdf unpack4(float4 q) { return cdf{df_make(q.x, q.y), df_make(q.z, q.w)}; }

// Ratios the mixed kernel keeps as double words stay below this magnitude. Normal ratios are O(1);
// one far larger comes only from an edge where the reference signal has almost vanished (a tapered
// end that the sample outlives), and a bin that uses such an edge is contracted in FP64 instead
// (ratio squares times 1/df^2 stay far inside the FP32 exponent range below it).
constexpr double kHetDwRatioMax = 16777216.0;   // 2^24

// FP64 contraction of coarse bin b, channel c: (<d|h>, <h|h>) from the ratios ld(edge, md) and the
// summary data A, B.
template <class Ld>
__device__ __forceinline__ void het_bin_fp64(const HetDev& H, int b, int c, Ld ld, double& dh, double& hh) {
  const double idf = 1.0 / (H.fe[b + 1] - H.fe[b]);
  double2 r0[kNModes], r1[kNModes];
  for (int md = 0; md < kNModes; ++md) {
    const int s0 = H.src[(b * kNModes + md) * 3 + c], s1 = H.src[((b + 1) * kNModes + md) * 3 + c];
    const double2 ra = s0 >= 0 ? ld(s0, md) : make_double2(0.0, 0.0);
    const double2 rb = s1 >= 0 ? ld(s1, md) : make_double2(0.0, 0.0);
    r0[md] = ra;
    r1[md] = make_double2((rb.x - ra.x) * idf, (rb.y - ra.y) * idf);
  }
  dh = 0.0;
  hh = 0.0;
  for (int md = 0; md < kNModes; ++md) {
    const double2 a0 = H.A[(((size_t)b * kNModes + md) * 3 + c) * 2 + 0];
    const double2 a1 = H.A[(((size_t)b * kNModes + md) * 3 + c) * 2 + 1];
    dh += cmul(a0, r0[md]).x + cmul(a1, r1[md]).x;
    for (int m2 = md; m2 < kNModes; ++m2) {
      const double2* q = H.Bs + (((size_t)b * kPairs + pair_index(md, m2)) * 3 + c) * 3;
      const double2 t0 = cmul(r0[md], cconj(r0[m2]));
      const double2 t1 = cadd(cmul(r1[md], cconj(r0[m2])), cmul(r0[md], cconj(r1[m2])));
      const double2 t2 = cmul(r1[md], cconj(r1[m2]));
      const double x = cmul(q[0], t0).x + cmul(q[1], t1).x + cmul(q[2], t2).x;
      hh += (md == m2) ? x : 2.0 * x;
    }
  }
}
// Re(a b) and Re(a conj(b)) in double words
__device__ __forceinline__ df re_mul(const cdf& a, const cdf& b) { return dfl_sub(dfl_mul(a.re, b.re), dfl_mul(a.im, b.im)); }
__device__ __forceinline__ cdf mul_conj(const cdf& a, const cdf& b) {
  return cdf{dfl_add(dfl_mul(a.re, b.re), dfl_mul(a.im, b.im)), dfl_sub(dfl_mul(a.im, b.re), dfl_mul(a.re, b.im))};
}

// One CTA of kTileBins threads per sample. Dynamic shared memory: [max ne][5][3] double2 ratios.
// MIX: the signal at the edges by the mixed-precision unit, the ratios kept as double words and
// the contraction in double words (Aw, Bw); the sums across bins and the block reduction stay
// FP64. An edge with a ratio of kHetDwRatioMax or more keeps all its ratios in FP64 (flag byte
// per edge after the ratios), and every (bin, channel) that reads it takes the FP64 contraction.
template <bool MIX>
__global__ void __launch_bounds__(kTileBins) k_het_loglike(HetSet hs, int B, const SampleCoef* __restrict__ coef,
                                                           double* logl, double* dhhh) {
  extern __shared__ double2 rsh[];
  unsigned char* wflag = reinterpret_cast<unsigned char*>(rsh + (size_t)hs.nemax * kNModes * 3);
  __shared__ double pc[kProj];
  __shared__ float2 pcw[MIX ? kProj : 1];
  __shared__ double sh[6][kTileBins / 32];
  __shared__ double2 stab[MIX ? 1 : kSinTab];
  __shared__ float4 stabw[MIX ? kSinTab : 1];
  if constexpr (MIX) {
    for (int i = threadIdx.x; i < kSinTab; i += blockDim.x) stabw[i] = hs.h[0].det.sctw[i];
  } else {
    for (int i = threadIdx.x; i < kSinTab; i += blockDim.x) stab[i] = hs.h[0].det.sct[i];
  }
  const int s = blockIdx.x;
  const SampleCoef& S = coef[s];
  double L = 0.0;
  for (int I = 0; I < hs.n; ++I) {
    const HetDev& H = hs.h[I];
    const DetDev& D = H.det;
    proj_prologue(D, S, pc);   // its barriers also order the table staging and the previous detector
    if constexpr (MIX) {
      if (threadIdx.x < kProj) pcw[threadIdx.x] = to_dw(pc[threadIdx.x]);
      __syncthreads();
    }
    for (int e = threadIdx.x; e < H.ne; e += blockDim.x) {
      bool need = false;
      for (int j = 0; j < kNModes * 3; ++j) need |= (H.src[e * kNModes * 3 + j] == e);
      if (!need) continue;
      double2 o[kNModes][3];
      if constexpr (MIX)
        mode_brackets_mixed(D, S, H.edge[e], H.mask, o, stabw, pcw);
      else
        mode_brackets(D, S, H.edge[e], H.mask, o, stab, pc);
      // ratios in place of the brackets; in the mixed kernel, flag the edge if one of them is out
      // of the double words' range (also for inf and NaN)
      bool wide = false;
#pragma unroll
      for (int md = 0; md < kNModes; ++md)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const int j = (e * kNModes + md) * 3 + c;
          if (H.src[j] != e) continue;
          o[md][c] = cmul(o[md][c], H.ih0e[j]);
          if constexpr (MIX) wide |= !(fmax(fabs(o[md][c].x), fabs(o[md][c].y)) < kHetDwRatioMax);
        }
      if constexpr (MIX) wflag[e] = wide ? 1 : 0;
#pragma unroll
      for (int md = 0; md < kNModes; ++md)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const int j = (e * kNModes + md) * 3 + c;
          if (H.src[j] != e) continue;
          if (MIX && !wide) {
            const float2 re = to_dw(o[md][c].x), im = to_dw(o[md][c].y);
            reinterpret_cast<float4*>(rsh)[j] = make_float4(re.x, re.y, im.x, im.y);
          } else {
            rsh[j] = o[md][c];
          }
        }
    }
    __syncthreads();
    double v[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    if constexpr (MIX) {
      const float4* rw = reinterpret_cast<const float4*>(rsh);
      const cdf zc = {df_make(0.f, 0.f), df_make(0.f, 0.f)};
      for (int b = threadIdx.x; b < H.ne - 1; b += blockDim.x) {
        const df idf = to_dw(1.0 / (H.fe[b + 1] - H.fe[b]));
#pragma unroll 1
        for (int c = 0; c < 3; ++c) {
          cdf r0[kNModes], r1[kNModes];
          bool wide = false;
#pragma unroll
          for (int md = 0; md < kNModes; ++md) {
            const int s0 = H.src[(b * kNModes + md) * 3 + c], s1 = H.src[((b + 1) * kNModes + md) * 3 + c];
            wide |= (s0 >= 0 && wflag[s0]) || (s1 >= 0 && wflag[s1]);
            const cdf ra = s0 >= 0 ? unpack4(rw[(s0 * kNModes + md) * 3 + c]) : zc;
            const cdf rb = s1 >= 0 ? unpack4(rw[(s1 * kNModes + md) * 3 + c]) : zc;
            r0[md] = ra;
            r1[md] = cdf{dfl_mul(dfl_sub(rb.re, ra.re), idf), dfl_mul(dfl_sub(rb.im, ra.im), idf)};
          }
          if (wide) {   // an edge of this bin keeps FP64 ratios (the double words above are unused)
            auto ld = [&](int e, int md) -> double2 {
              const int j = (e * kNModes + md) * 3 + c;
              if (wflag[e]) return rsh[j];
              const cdf r = unpack4(rw[j]);
              return make_double2(df_to(r.re), df_to(r.im));
            };
            double dh, hh;
            het_bin_fp64(H, b, c, ld, dh, hh);
            v[c] += dh;
            v[3 + c] += hh;
            continue;
          }
          df dh = df_make(0.f, 0.f), hh = df_make(0.f, 0.f);
#pragma unroll
          for (int md = 0; md < kNModes; ++md) {
            const float4* a = H.Aw + (((size_t)b * kNModes + md) * 3 + c) * 2;
            dh = dfl_add(dh, dfl_add(re_mul(unpack4(a[0]), r0[md]), re_mul(unpack4(a[1]), r1[md])));
#pragma unroll
            for (int m2 = md; m2 < kNModes; ++m2) {
              const float4* q = H.Bw + (((size_t)b * kPairs + pair_index(md, m2)) * 3 + c) * 3;
              const cdf t0 = mul_conj(r0[md], r0[m2]);
              const cdf ta = mul_conj(r1[md], r0[m2]), tb = mul_conj(r0[md], r1[m2]);
              const cdf t1 = {dfl_add(ta.re, tb.re), dfl_add(ta.im, tb.im)};
              const cdf t2 = mul_conj(r1[md], r1[m2]);
              df x = dfl_add(dfl_add(re_mul(unpack4(q[0]), t0), re_mul(unpack4(q[1]), t1)), re_mul(unpack4(q[2]), t2));
              if (md != m2) x = df_scale2(x, 2.0f);
              hh = dfl_add(hh, x);
            }
          }
          v[c] += df_to(dh);
          v[3 + c] += df_to(hh);
        }
      }
    } else
    for (int b = threadIdx.x; b < H.ne - 1; b += blockDim.x) {
#pragma unroll 1
      for (int c = 0; c < 3; ++c) {
        double dh, hh;
        het_bin_fp64(H, b, c, [&](int e, int md) { return rsh[(e * kNModes + md) * 3 + c]; }, dh, hh);
        v[c] += dh;
        v[3 + c] += hh;
      }
    }
    block_sum<6>(v, sh);
    if (threadIdx.x == 0) {
      for (int c = 0; c < 3; ++c) {
        L += v[c] - 0.5 * v[3 + c] - 0.5 * D.dd[c];
        if (dhhh) {
          dhhh[(((size_t)s * hs.n + I) * 3 + c) * 2 + 0] = v[c];
          dhhh[(((size_t)s * hs.n + I) * 3 + c) * 2 + 1] = v[3 + c];
        }
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) logl[s] = S.valid ? L : -INFINITY;
}

}  // namespace pe

// ------------------------------------------------------------------------------------------
// Host side
// ------------------------------------------------------------------------------------------
struct pe_hetero_s {
  pe::HetDev dev;
  void* mem;
  int device;
};

namespace {

constexpr double kMsunSh = 4.925490947641267e-6;
const double kGam[5] = {-5.0 / 3.0, -2.0 / 3.0, 1.0, 5.0 / 3.0, 7.0 / 3.0};
const int kModeMh[pe::kNModes] = {2, 1, 3, 2, 4};

double phase_metric(double f, double flo, double fhi) {
  double s = 0.0;
  for (double g : kGam) s += (g < 0 ? -1.0 : 1.0) * std::pow(f / (g < 0 ? flo : fhi), g);
  return s;
}
double fisco_of(const double* th) { return std::pow(6.0, -1.5) / (2.0 * pe::kPi * th[0] * kMsunSh); }

// Taper marks 1 - 0.1 * 0.7^j (j = 0..10) of m F_isco, as grid indices; kend: last bin below it.
void taper_marks(double T, long long k0, double fisco, int m, long long ks[11], long long* kend) {
  const double fe = m * fisco;
  for (int j = 0; j < 11; ++j) ks[j] = (long long)std::ceil((1.0 - 0.1 * std::pow(0.7, j)) * fe * T) - k0;
  *kend = (long long)std::ceil(fe * T) - k0 - 1;
}

bool mask_ok(unsigned m) { return (m & PE_MODE_ALL) != 0u && (m & ~(PE_MODE_ALL | PE_PREC_MIXED)) == 0u; }

pe_status herr(pe_status st, const char* msg) { return pe::set_error(st, msg); }

}  // namespace

extern "C" {

pe_status pe_hetero_default_edges(double T_obs, int64_t k0, int64_t nbins, const double* theta0, unsigned mode_mask,
                                  int nbins_coarse, int64_t* out_edges, int* inout_n) {
  if (theta0 == nullptr || out_edges == nullptr || inout_n == nullptr)
    return herr(PE_EINVAL, "pe_hetero_default_edges: NULL argument");
  if (!(T_obs > 0.0) || k0 < 1 || nbins < 2 || nbins_coarse < 1 || !mask_ok(mode_mask) || !(theta0[0] > 0.0))
    return herr(PE_EINVAL, "pe_hetero_default_edges: bad grid, mask, theta0 or bin count");
  const double fisco = fisco_of(theta0);
  double fend = 0.0;
  for (int md = 0; md < pe::kNModes; ++md)
    if ((mode_mask >> md) & 1u) fend = std::max(fend, kModeMh[md] * fisco);
  const long long kmax = std::min<long long>(nbins - 1, (long long)std::ceil(fend * T_obs) - k0 - 1);
  if (kmax < 1) return herr(PE_EINVAL, "pe_hetero_default_edges: the reference's band ends below the grid");
  const double flo = k0 / T_obs, fhi = (k0 + kmax) / T_obs;
  const double p0 = phase_metric(flo, flo, fhi), p1 = phase_metric(fhi, flo, fhi);
  std::set<long long> cand = {0, kmax};
  for (int j = 1; j < nbins_coarse; ++j) {
    const double target = p0 + (p1 - p0) * j / nbins_coarse;
    double a = flo, b = fhi;
    for (int it = 0; it < 200; ++it) {
      const double mid = 0.5 * (a + b);
      if (phase_metric(mid, flo, fhi) < target) a = mid; else b = mid;
    }
    cand.insert((long long)std::llround(0.5 * (a + b) * T_obs) - k0);
  }
  std::vector<std::pair<long long, long long>> forbid;   // (last mark, kend) per mode
  for (int md = 0; md < pe::kNModes; ++md) {
    if (!((mode_mask >> md) & 1u)) continue;
    long long ks[11], kend;
    taper_marks(T_obs, k0, fisco, kModeMh[md], ks, &kend);
    for (long long k : ks) cand.insert(k);
    forbid.push_back({ks[10], kend});
  }
  std::vector<int64_t> keep;
  for (long long k : cand) {
    if (k < 0 || k > kmax) continue;
    bool bad = false;
    if (k != kmax)
      for (auto& fb : forbid) bad |= (k > fb.first && k <= fb.second);
    if (!bad) keep.push_back(k);
  }
  if ((int)keep.size() > *inout_n) {
    char msg[160];
    snprintf(msg, sizeof(msg), "pe_hetero_default_edges: %zu edges do not fit in %d", keep.size(), *inout_n);
    return herr(PE_EINVAL, msg);
  }
  std::copy(keep.begin(), keep.end(), out_edges);
  *inout_n = (int)keep.size();
  return PE_OK;
}

pe_status pe_hetero_create(pe_detector det, const double* theta0, unsigned mode_mask, const int64_t* edges,
                           int nedges, pe_hetero* out) {
  if (out == nullptr || theta0 == nullptr || edges == nullptr) return herr(PE_EINVAL, "pe_hetero_create: NULL argument");
  *out = nullptr;
  if (!mask_ok(mode_mask)) return herr(PE_EINVAL, "pe_hetero_create: bad mode mask (PE_PREC_FP32 is not taken)");
  pe::DetSet ds;
  pe_status s0 = pe::detset_from_handles(&det, 1, &ds);
  if (s0 != PE_OK) return s0;
  const pe::DetDev& D = ds.d[0];
  const int ne = nedges;
  if (ne < 2 || ne > pe::kHetMaxEdges) return herr(PE_EINVAL, "pe_hetero_create: nedges outside [2, 640]");
  for (int i = 0; i < ne; ++i) {
    if (edges[i] < 0 || edges[i] >= D.nb || (i > 0 && edges[i] <= edges[i - 1]))
      return herr(PE_EINVAL, "pe_hetero_create: edges must increase strictly inside the grid");
  }
  for (int i = 0; i < PE_NPARAM; ++i)
    if (!std::isfinite(theta0[i])) return herr(PE_EINVAL, "pe_hetero_create: theta0 is not finite");
  const int K = (int)edges[ne - 1] + 1;
  const int nb = ne - 1;
  // one allocation: edge [ne] int, src [ne][5][3] int, fe [ne] double, h0e [ne][15], A [nb][30], Bs [nb][kPairs*9]
  auto a256 = [](size_t x) { return (x + 255) & ~size_t(255); };
  const size_t o_edge = 0;
  const size_t o_src = a256(o_edge + ne * sizeof(int));
  const size_t o_fe = a256(o_src + (size_t)ne * 15 * sizeof(int));
  const size_t o_h0e = a256(o_fe + ne * sizeof(double));
  const size_t o_A = a256(o_h0e + (size_t)ne * 15 * sizeof(double2));
  const size_t o_B = a256(o_A + (size_t)nb * 30 * sizeof(double2));
  const size_t o_Aw = a256(o_B + (size_t)nb * pe::kPairs * 9 * sizeof(double2));
  const size_t o_Bw = a256(o_Aw + (size_t)nb * 30 * sizeof(float4));
  const size_t bytes = o_Bw + (size_t)nb * pe::kPairs * 9 * sizeof(float4);
  pe_hetero_s* h = new (std::nothrow) pe_hetero_s();
  if (!h) return herr(PE_ENOMEM, "pe_hetero_create: host allocation failed");
  cudaGetDevice(&h->device);
  if (pe::dmalloc(&h->mem, bytes) != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return herr(PE_ENOMEM, "pe_hetero_create: device allocation failed");
  }
  unsigned char* base = static_cast<unsigned char*>(h->mem);
  int* d_edge = reinterpret_cast<int*>(base + o_edge);
  int* d_src = reinterpret_cast<int*>(base + o_src);
  double* d_fe = reinterpret_cast<double*>(base + o_fe);
  double2* d_h0e = reinterpret_cast<double2*>(base + o_h0e);
  double2* d_A = reinterpret_cast<double2*>(base + o_A);
  double2* d_B = reinterpret_cast<double2*>(base + o_B);
  float4* d_Aw = reinterpret_cast<float4*>(base + o_Aw);
  float4* d_Bw = reinterpret_cast<float4*>(base + o_Bw);
  std::vector<int> he(ne);
  std::vector<double> hfe(ne);
  for (int i = 0; i < ne; ++i) {
    he[i] = (int)edges[i];
    hfe[i] = double(D.k0 + edges[i]) / D.T;
  }
  double* th0 = nullptr;
  pe::SampleCoef* coef = nullptr;
  int* nend = nullptr;
  double2* hb = nullptr;
  cudaError_t e = pe::dmalloc(&th0, PE_NPARAM * sizeof(double));
  if (e == cudaSuccess) e = pe::dmalloc(&coef, sizeof(pe::SampleCoef));
  if (e == cudaSuccess) e = pe::dmalloc(&nend, sizeof(int));
  if (e == cudaSuccess) e = pe::dmalloc(&hb, (size_t)pe::kNModes * 3 * K * sizeof(double2));
  if (e == cudaSuccess) e = pe::upload(th0, theta0, PE_NPARAM * sizeof(double));
  if (e == cudaSuccess) e = pe::upload(d_edge, he.data(), ne * sizeof(int));
  if (e == cudaSuccess) e = pe::upload(d_fe, hfe.data(), ne * sizeof(double));
  if (e == cudaSuccess) e = pe::launch_prep(th0, 1, mode_mask, ds, coef, nend, nullptr, 0);
  if (e == cudaSuccess) {
    pe::k_mode_brackets<<<(K + pe::kTileBins - 1) / pe::kTileBins, pe::kTileBins>>>(D, coef, K, mode_mask, hb);
    e = pe::launch_status();
  }
  // reference brackets at the edges, and the carry-forward sources
  std::vector<double2> h0e((size_t)ne * 15);
  if (e == cudaSuccess) {
    pe::k_gather_edges<<<(ne * 15 + 127) / 128, 128>>>(hb, K, d_edge, ne, d_h0e);
    e = pe::launch_status();
  }
  if (e == cudaSuccess) e = cudaMemcpy(h0e.data(), d_h0e, h0e.size() * sizeof(double2), cudaMemcpyDeviceToHost);
  std::vector<int> src((size_t)ne * 15, -1);
  if (e == cudaSuccess) {
    const double fisco = fisco_of(theta0);
    for (int md = 0; md < pe::kNModes; ++md) {
      long long klast = -1;
      if ((mode_mask >> md) & 1u) {
        long long ks[11], kend;
        taper_marks(D.T, D.k0, fisco, kModeMh[md], ks, &kend);
        klast = ks[10];
      }
      for (int c = 0; c < 3; ++c)
        for (int i = 0; i < ne; ++i) {
          const size_t j = ((size_t)i * pe::kNModes + md) * 3 + c;
          const bool ok = he[i] <= klast && (h0e[j].x != 0.0 || h0e[j].y != 0.0);
          src[j] = ok ? i : (i > 0 ? src[j - 15] : -1);
        }
    }
    e = pe::upload(d_src, src.data(), src.size() * sizeof(int));
  }
  if (e == cudaSuccess) {   // the per-sample kernel multiplies by the inverses (no division per ratio)
    pe::k_invert_edges<<<(ne * 15 + 127) / 128, 128>>>(d_h0e, ne * 15);
    e = pe::launch_status();
  }
  if (e == cudaSuccess) {
    const long long n = (long long)nb * (30 + pe::kPairs * 9);
    pe::k_het_summary<<<(unsigned)((n + 127) / 128), 128>>>(D, d_edge, d_fe, ne, hb, K, d_A, d_B);
    e = pe::launch_status();
  }
  if (e == cudaSuccess) {   // double-word copies of the summary data for the mixed-precision kernel
    const long long na = (long long)nb * 30, nbq = (long long)nb * pe::kPairs * 9;
    pe::k_to_dw4<<<(unsigned)((na + 255) / 256), 256>>>(d_A, na, d_Aw);
    pe::k_to_dw4<<<(unsigned)((nbq + 255) / 256), 256>>>(d_B, nbq, d_Bw);
    e = pe::launch_status();
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  pe::dfree(th0);
  pe::dfree(coef);
  pe::dfree(nend);
  pe::dfree(hb);
  if (e != cudaSuccess) {
    cudaGetLastError();
    pe::dfree(h->mem);
    delete h;
    char msg[200];
    snprintf(msg, sizeof(msg), "pe_hetero_create: %s", cudaGetErrorString(e));
    return herr(PE_ECUDA, msg);
  }
  h->dev.det = D;
  h->dev.edge = d_edge;
  h->dev.fe = d_fe;
  h->dev.ih0e = d_h0e;
  h->dev.src = d_src;
  h->dev.A = d_A;
  h->dev.Bs = d_B;
  h->dev.Aw = d_Aw;
  h->dev.Bw = d_Bw;
  h->dev.ne = ne;
  h->dev.mask = mode_mask;
  *out = h;
  return PE_OK;
}

pe_status pe_hetero_destroy(pe_hetero h) {
  if (h == nullptr) return PE_OK;
  cudaDeviceSynchronize();
  pe::dfree(h->mem);
  cudaGetLastError();
  delete h;
  return PE_OK;
}

pe_status pe_hetero_loglike_batch(const pe_hetero* hets, int ndet, const double* theta, int B, double* out_logl,
                                  double* out_dhhh, int32_t* out_status, void* stream) {
  if (hets == nullptr || theta == nullptr || out_logl == nullptr) return herr(PE_EINVAL, "pe_hetero_loglike_batch: NULL");
  if (ndet < 1 || ndet > pe::kMaxDet) return herr(PE_EINVAL, "pe_hetero_loglike_batch: ndet outside [1, 8]");
  if (B < 1 || B > (1 << 20)) return herr(PE_EINVAL, "pe_hetero_loglike_batch: B outside [1, 2^20]");
  pe::HetSet hs;
  memset(&hs, 0, sizeof(hs));
  pe::DetSet ds;
  memset(&ds, 0, sizeof(ds));
  hs.n = ndet;
  ds.ndet = ndet;
  int dev = 0, nemax = 0;
  cudaGetDevice(&dev);
  for (int i = 0; i < ndet; ++i) {
    if (hets[i] == nullptr) return herr(PE_EINVAL, "pe_hetero_loglike_batch: NULL handle");
    if (hets[i]->device != dev) return herr(PE_EINVAL, "pe_hetero_loglike_batch: handle on another device");
    if (hets[i]->dev.mask != hets[0]->dev.mask) return herr(PE_EINVAL, "pe_hetero_loglike_batch: mode masks differ");
    hs.h[i] = hets[i]->dev;
    ds.d[i] = hets[i]->dev.det;
    nemax = std::max(nemax, hets[i]->dev.ne);
  }
  hs.nemax = nemax;
  auto is_dev = [](const void* p) {
    if (p == nullptr) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) { cudaGetLastError(); return false; }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
  };
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  std::vector<void*> bufs;
  cudaError_t e = cudaSuccess;
  auto alloc = [&](void** p, size_t n) {
    if (e != cudaSuccess) return;
    e = pe::dmalloc_async(p, n + 16, st);
    if (e == cudaSuccess) bufs.push_back(*p);
  };
  const double* th = theta;
  if (!is_dev(theta)) {
    void* t = nullptr;
    alloc(&t, (size_t)B * PE_NPARAM * sizeof(double));
    if (e == cudaSuccess) e = pe::upload_async(t, theta, (size_t)B * PE_NPARAM * sizeof(double), st);
    th = static_cast<const double*>(t);
  }
  void *coef = nullptr, *nend = nullptr, *ll = out_logl, *dh = out_dhhh, *stt = out_status;
  alloc(&coef, (size_t)B * sizeof(pe::SampleCoef));
  alloc(&nend, (size_t)B * ndet * sizeof(int));
  const bool hl = !is_dev(out_logl), hd = out_dhhh && !is_dev(out_dhhh), hsx = out_status && !is_dev(out_status);
  if (hl) alloc(&ll, (size_t)B * sizeof(double));
  if (hd) alloc(&dh, (size_t)B * ndet * 6 * sizeof(double));
  if (hsx) alloc(&stt, (size_t)B * sizeof(int32_t));
  if (e == cudaSuccess)
    e = pe::launch_prep(th, B, hets[0]->dev.mask, ds, static_cast<pe::SampleCoef*>(coef), static_cast<int*>(nend),
                        static_cast<int*>(stt), st);
  const bool mix = (hets[0]->dev.mask & PE_PREC_MIXED) != 0u;
  const size_t smem = (size_t)nemax * pe::kNModes * 3 * sizeof(double2) + (mix ? (size_t)nemax : 0);
  auto kern = mix ? pe::k_het_loglike<true> : pe::k_het_loglike<false>;
  if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) {
    kern<<<B, pe::kTileBins, smem, st>>>(hs, B, static_cast<const pe::SampleCoef*>(coef), static_cast<double*>(ll),
                                         static_cast<double*>(dh));
    e = pe::launch_status();
  }
  if (e == cudaSuccess && hl) e = cudaMemcpyAsync(out_logl, ll, (size_t)B * sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && hd)
    e = cudaMemcpyAsync(out_dhhh, dh, (size_t)B * ndet * 6 * sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && hsx) e = cudaMemcpyAsync(out_status, stt, (size_t)B * sizeof(int32_t), cudaMemcpyDeviceToHost, st);
  for (void* p : bufs) pe::dfree_async(p, st);
  if (e == cudaSuccess && (hl || hd || hsx)) e = pe::wait_stream(st);
  if (e == cudaErrorNotReady) return herr(PE_ETIMEOUT, "pe_hetero_loglike_batch: stream did not finish within the wait limit");
  if (e != cudaSuccess) {
    cudaGetLastError();
    char msg[200];
    snprintf(msg, sizeof(msg), "pe_hetero_loglike_batch: %s", cudaGetErrorString(e));
    return herr(PE_ECUDA, msg);
  }
  return PE_OK;
}

}  // extern "C"
