// pe_oracle.cpp -- plain, slow, FP64 CPU oracle for the MBHB Whittle log-likelihood of
// arXiv:2602.12011 (pespace), restated from the paper's Sec. 2.1-2.2 and the project readings
// of what the paper leaves to its references.
//
// TEST INFRASTRUCTURE ONLY. Nothing in the library's product path may include, link or call
// this file. Only the test suite, the smoke check and the benchmark's CPU-baseline leg load it.
// It shares no code, header, table or constant with the CUDA library: every constant below is
// this file's own copy.
//
// Structure (each function cites the passage it follows):
//   * Dual<T,N> forward-mode dual numbers: the scalar type every formula is templated on.
//     T = double gives values; Dual<double,11> gives the exact gradient and the Jacobian for
//     the Fisher matrix; Dual<.,1> in the frequency gives t_f = (1/2pi) dPsi/df (Eq. eq_tf).
//   * TaylorF2 waveform per (l,m) mode (fallback waveform: 3.5PN phase of Buonanno, Iyer,
//     Ochsner, Pan & Sathyaprakash 2009, leading-order spherical-mode amplitudes of
//     Blanchet's Living Review, SPA; a C-infinity Planck taper ends every mode at the ISCO).
//   * -2Y_lm from the general Wigner-d sum (Goldberg et al. 1967; Ajith et al. 2007).
//   * Analytic orbits: heliocentric Keplerian constellation to first order in eccentricity
//     (Rubbo, Cornish & Poujade 2004) for LISA/Taiji; geocentric circular constellation
//     around a circular-orbit Earth for TianQin (Sec. 2.1, Sec. 3.2).
//   * Single-link FD response, Eq. eq_fd_resp; FD TDI 1.5/2.0 (Sec. 2.1, after Eq. eq_tf);
//     A/E/T (Sec. 2.1, the orthogonal-channel equations).
//   * PSD (acceleration + OMS noise only, Sec. 3.2), Whittle likelihood Eq. eq_ll_fd with the
//     inner product Eq. eq_inner_product, joint product over channels/detectors (Sec. 2.2).
//   * Fisher matrix F_ij = <ds/dtheta_i | ds/dtheta_j> (Sec. 2.2, Eq. eq_ll_fisher and below).
// Sums over bins use Neumaier-compensated accumulation.
//
// Parity unpinned (no check here beyond the transcription itself; the tests pin everything
// else against closed forms, brute force, energy balance, multipole flux, the 1PN polarisations
// or the paper's identities):
//   * the TianQin normal direction and every noise level (configuration readings); the A/E/T
//     algebra of psd_aet is pinned.
//
// Build: g++ -O2 -std=c++17 -fPIC -shared -fopenmp (no fast-math).

#include <cmath>
#include <cstdint>
#include <cstring>
#include <type_traits>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace oracle {

// ----------------------------------------------------------------------------------------
// Constants (this file's own copy).
// ----------------------------------------------------------------------------------------
static const double PI = 3.14159265358979323846;
static const double C_SI = 299792458.0;                  // speed of light [m/s]
static const double MSUN_S = 4.925490947641267e-6;       // G Msun / c^3 [s] (IAU 2015 nominal)
static const double GPC_S = 1.02927125054339e17;         // 1 Gpc / c [s]
static const double AU_S = 499.00478383615643;           // 1 au / c [s]
static const double YEAR_S = 31557600.0;                 // Julian year [s]
static const double EULER_GAMMA = 0.57721566490153286061;

// ----------------------------------------------------------------------------------------
// Forward-mode dual numbers over any scalar type T.
// ----------------------------------------------------------------------------------------
template <class T, int N>
struct Dual {
  T v;
  T d[N];
  Dual() : v(0.0) { for (int i = 0; i < N; ++i) d[i] = T(0.0); }
  Dual(const T& x) : v(x) { for (int i = 0; i < N; ++i) d[i] = T(0.0); }
  template <class U = T, typename std::enable_if<!std::is_same<U, double>::value, int>::type = 0>
  Dual(double x) : v(x) { for (int i = 0; i < N; ++i) d[i] = T(0.0); }
  Dual(const T& x, int) : v(x) { for (int i = 0; i < N; ++i) d[i] = T(0.0); }
};

template <class T> struct is_dual { static const bool value = false; };
template <class T, int N> struct is_dual<Dual<T, N>> { static const bool value = true; };

inline double val(double x) { return x; }
inline double val(long double x) { return (double)x; }
template <class T, int N> inline double val(const Dual<T, N>& x) { return val(x.v); }

#define DUAL_T template <class T, int N>
DUAL_T inline Dual<T, N> operator+(const Dual<T, N>& a, const Dual<T, N>& b) {
  Dual<T, N> r; r.v = a.v + b.v; for (int i = 0; i < N; ++i) r.d[i] = a.d[i] + b.d[i]; return r; }
DUAL_T inline Dual<T, N> operator-(const Dual<T, N>& a, const Dual<T, N>& b) {
  Dual<T, N> r; r.v = a.v - b.v; for (int i = 0; i < N; ++i) r.d[i] = a.d[i] - b.d[i]; return r; }
DUAL_T inline Dual<T, N> operator-(const Dual<T, N>& a) {
  Dual<T, N> r; r.v = -a.v; for (int i = 0; i < N; ++i) r.d[i] = -a.d[i]; return r; }
DUAL_T inline Dual<T, N> operator*(const Dual<T, N>& a, const Dual<T, N>& b) {
  Dual<T, N> r; r.v = a.v * b.v; for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i]; return r; }
DUAL_T inline Dual<T, N> operator/(const Dual<T, N>& a, const Dual<T, N>& b) {
  Dual<T, N> r; r.v = a.v / b.v; T ib = T(1.0) / (b.v * b.v);
  for (int i = 0; i < N; ++i) r.d[i] = (a.d[i] * b.v - a.v * b.d[i]) * ib; return r; }
DUAL_T inline Dual<T, N> operator+(const Dual<T, N>& a, double b) { Dual<T, N> r = a; r.v = r.v + b; return r; }
DUAL_T inline Dual<T, N> operator+(double b, const Dual<T, N>& a) { return a + b; }
DUAL_T inline Dual<T, N> operator-(const Dual<T, N>& a, double b) { Dual<T, N> r = a; r.v = r.v - b; return r; }
DUAL_T inline Dual<T, N> operator-(double b, const Dual<T, N>& a) { return (-a) + b; }
DUAL_T inline Dual<T, N> operator*(const Dual<T, N>& a, double b) {
  Dual<T, N> r; r.v = a.v * b; for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * b; return r; }
DUAL_T inline Dual<T, N> operator*(double b, const Dual<T, N>& a) { return a * b; }
DUAL_T inline Dual<T, N> operator/(const Dual<T, N>& a, double b) { return a * (1.0 / b); }
DUAL_T inline Dual<T, N> operator/(double a, const Dual<T, N>& b) { return Dual<T, N>(a) / b; }
DUAL_T inline Dual<T, N>& operator+=(Dual<T, N>& a, const Dual<T, N>& b) { a = a + b; return a; }
DUAL_T inline Dual<T, N>& operator-=(Dual<T, N>& a, const Dual<T, N>& b) { a = a - b; return a; }
DUAL_T inline Dual<T, N>& operator*=(Dual<T, N>& a, const Dual<T, N>& b) { a = a * b; return a; }

// chain rule helper: f(a) with f'(a.v) = df
DUAL_T inline Dual<T, N> chain(const Dual<T, N>& a, const T& f, const T& df) {
  Dual<T, N> r; r.v = f; for (int i = 0; i < N; ++i) r.d[i] = df * a.d[i]; return r; }

using std::sin; using std::cos; using std::exp; using std::log; using std::sqrt; using std::cbrt;
using std::pow; using std::fabs;
DUAL_T inline Dual<T, N> sin(const Dual<T, N>& a) { return chain(a, sin(a.v), cos(a.v)); }
DUAL_T inline Dual<T, N> cos(const Dual<T, N>& a) { return chain(a, cos(a.v), -sin(a.v)); }
DUAL_T inline Dual<T, N> exp(const Dual<T, N>& a) { T e = exp(a.v); return chain(a, e, e); }
DUAL_T inline Dual<T, N> log(const Dual<T, N>& a) { return chain(a, log(a.v), T(1.0) / a.v); }
DUAL_T inline Dual<T, N> sqrt(const Dual<T, N>& a) { T s = sqrt(a.v); return chain(a, s, T(0.5) / s); }
DUAL_T inline Dual<T, N> cbrt(const Dual<T, N>& a) { T c = cbrt(a.v); return chain(a, c, c / (T(3.0) * a.v)); }
DUAL_T inline Dual<T, N> pow(const Dual<T, N>& a, double p) {
  T f = pow(a.v, p); return chain(a, f, T(p) * pow(a.v, p - 1.0)); }

// ----------------------------------------------------------------------------------------
// Operation-counting scalar: a double that counts every arithmetic operation and math-library
// call made on it (the algorithmic-work model of the method, or_op_count). Single-threaded use.
// ----------------------------------------------------------------------------------------
enum { OP_ADD, OP_MUL, OP_DIV, OP_SQRT, OP_SINCOS, OP_EXP, OP_LOG, OP_CBRT, OP_POW, OP_CMP, OP_N };
static unsigned long long g_ops[OP_N];
struct Flop {
  double v;
  Flop() : v(0.0) {}
  Flop(double x) : v(x) {}
};
inline double val(const Flop& x) { return x.v; }
inline Flop fop(int k, double r) { ++g_ops[k]; return Flop(r); }
inline Flop operator+(const Flop& a, const Flop& b) { return fop(OP_ADD, a.v + b.v); }
inline Flop operator-(const Flop& a, const Flop& b) { return fop(OP_ADD, a.v - b.v); }
inline Flop operator*(const Flop& a, const Flop& b) { return fop(OP_MUL, a.v * b.v); }
inline Flop operator/(const Flop& a, const Flop& b) { return fop(OP_DIV, a.v / b.v); }
inline Flop operator+(const Flop& a, double b) { return fop(OP_ADD, a.v + b); }
inline Flop operator+(double a, const Flop& b) { return fop(OP_ADD, a + b.v); }
inline Flop operator-(const Flop& a, double b) { return fop(OP_ADD, a.v - b); }
inline Flop operator-(double a, const Flop& b) { return fop(OP_ADD, a - b.v); }
inline Flop operator*(const Flop& a, double b) { return fop(OP_MUL, a.v * b); }
inline Flop operator*(double a, const Flop& b) { return fop(OP_MUL, a * b.v); }
inline Flop operator/(const Flop& a, double b) { return fop(OP_DIV, a.v / b); }
inline Flop operator/(double a, const Flop& b) { return fop(OP_DIV, a / b.v); }
inline Flop operator-(const Flop& a) { return Flop(-a.v); }
inline Flop& operator+=(Flop& a, const Flop& b) { a = a + b; return a; }
inline Flop& operator-=(Flop& a, const Flop& b) { a = a - b; return a; }
inline Flop& operator*=(Flop& a, const Flop& b) { a = a * b; return a; }
inline Flop sin(const Flop& a) { return fop(OP_SINCOS, std::sin(a.v)); }
inline Flop cos(const Flop& a) { return fop(OP_SINCOS, std::cos(a.v)); }
inline Flop exp(const Flop& a) { return fop(OP_EXP, std::exp(a.v)); }
inline Flop log(const Flop& a) { return fop(OP_LOG, std::log(a.v)); }
inline Flop sqrt(const Flop& a) { return fop(OP_SQRT, std::sqrt(a.v)); }
inline Flop cbrt(const Flop& a) { return fop(OP_CBRT, std::cbrt(a.v)); }
inline Flop pow(const Flop& a, double p) { return fop(OP_POW, std::pow(a.v, p)); }
inline Flop fabs(const Flop& a) { return Flop(std::fabs(a.v)); }

// ----------------------------------------------------------------------------------------
// Complex numbers over T (std::complex is only specified for built-in floating types).
// ----------------------------------------------------------------------------------------
template <class T>
struct Cx {
  T re, im;
  Cx() : re(0.0), im(0.0) {}
  Cx(const T& r) : re(r), im(0.0) {}
  Cx(const T& r, const T& i) : re(r), im(i) {}
};
template <class T> inline Cx<T> operator+(const Cx<T>& a, const Cx<T>& b) { return Cx<T>(a.re + b.re, a.im + b.im); }
template <class T> inline Cx<T> operator-(const Cx<T>& a, const Cx<T>& b) { return Cx<T>(a.re - b.re, a.im - b.im); }
template <class T> inline Cx<T> operator*(const Cx<T>& a, const Cx<T>& b) {
  return Cx<T>(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re); }
template <class T> inline Cx<T> operator*(const Cx<T>& a, const T& s) { return Cx<T>(a.re * s, a.im * s); }
template <class T> inline Cx<T> operator*(const T& s, const Cx<T>& a) { return Cx<T>(a.re * s, a.im * s); }
template <class T> inline Cx<T> conj(const Cx<T>& a) { return Cx<T>(a.re, -a.im); }
template <class T> inline T norm2(const Cx<T>& a) { return a.re * a.re + a.im * a.im; }
// e^{i x}
template <class T> inline Cx<T> expi(const T& x) { return Cx<T>(cos(x), sin(x)); }

// ----------------------------------------------------------------------------------------
// Neumaier-compensated accumulator, applied component by component for dual numbers.
// ----------------------------------------------------------------------------------------
template <class T> struct Acc;
template <> struct Acc<double> {
  double s = 0.0, c = 0.0;
  void add(double x) {
    double t = s + x;
    if (fabs(s) >= fabs(x)) c += (s - t) + x; else c += (x - t) + s;
    s = t;
  }
  double get() const { return s + c; }
};
template <> struct Acc<Flop> {
  Flop s;
  void add(const Flop& x) { s = s + x; }
  Flop get() const { return s; }
};
template <class T, int N> struct Acc<Dual<T, N>> {
  Acc<T> v; Acc<T> d[N];
  void add(const Dual<T, N>& x) { v.add(x.v); for (int i = 0; i < N; ++i) d[i].add(x.d[i]); }
  Dual<T, N> get() const { Dual<T, N> r; r.v = v.get(); for (int i = 0; i < N; ++i) r.d[i] = d[i].get(); return r; }
};

// ----------------------------------------------------------------------------------------
// Detector configuration (this file's own layout; the tests fill it from a Python dict).
// ----------------------------------------------------------------------------------------
struct OrConfig {
  int orbit;            // 0 = heliocentric Keplerian (LISA/Taiji), 1 = geocentric (TianQin)
  int tdi_gen;          // 15 or 20
  int psd_shaping;      // 1: LISA-type shaping factors on the OMS and acceleration noise
  int pad_;
  double arm_m;         // nominal arm length L [m]
  double alpha0;        // initial revolution angle around the Sun [rad]
  double cartwheel0;    // initial orientation of the heliocentric constellation [rad]
  double geo_period_s;  // TianQin constellation period [s]
  double geo_lon;       // TianQin constellation normal, ecliptic longitude [rad]
  double geo_lat;       // TianQin constellation normal, ecliptic latitude [rad]
  double oms_m_rtHz;    // optical-metrology displacement noise [m/sqrt(Hz)]
  double acc_ms2_rtHz;  // test-mass acceleration noise [m/s^2/sqrt(Hz)]
};

// ----------------------------------------------------------------------------------------
// Source parameters. theta[11] = Mtot[Msun], q=m1/m2>=1, chi1, chi2, dL[Gpc], iota, phi_c,
// lambda, beta, psi, t_c[s] (Table tab_pe_res lists the same eleven; q is inverted here).
// ----------------------------------------------------------------------------------------
template <class T>
struct Source {
  T Mtot, q, chi1, chi2, dL, iota, phic, lam, bet, psi, tc;
};
template <class T>
Source<T> source_from(const T* th) {
  Source<T> s;
  s.Mtot = th[0]; s.q = th[1]; s.chi1 = th[2]; s.chi2 = th[3]; s.dL = th[4]; s.iota = th[5];
  s.phic = th[6]; s.lam = th[7]; s.bet = th[8]; s.psi = th[9]; s.tc = th[10];
  return s;
}

// modes, in mode-mask bit order
static const int MODE_L[5] = {2, 2, 3, 3, 4};
static const int MODE_M[5] = {2, 1, 3, 2, 4};

// ----------------------------------------------------------------------------------------
// TaylorF2 phase (Buonanno et al. 2009, Eq. 3.18 there; spin-orbit at 1.5PN and aligned
// spin-spin at 2PN as the project's stated truncation). Returns Psi_PN(v) in radians:
//   Psi_PN(v) = 3/(128 eta v^5) * sum_k alpha_k(v) v^k.
// ----------------------------------------------------------------------------------------
template <class T, class V>
V psi_pn(const Source<T>& s, const V& v) {
  const T eta = s.q / ((1.0 + s.q) * (1.0 + s.q));
  const T m1 = s.q / (1.0 + s.q), m2 = 1.0 / (1.0 + s.q);  // masses in units of Mtot
  const T beta_so = s.chi1 * (113.0 / 12.0 * m1 * m1 + 25.0 / 4.0 * eta) +
                    s.chi2 * (113.0 / 12.0 * m2 * m2 + 25.0 / 4.0 * eta);
  const T sigma_ss = 79.0 / 8.0 * eta * s.chi1 * s.chi2;
  const double vlso = 1.0 / std::sqrt(6.0);
  const V lnv = log(v);
  V a[8];
  a[0] = V(1.0);
  a[1] = V(0.0);
  a[2] = V(3715.0 / 756.0 + 55.0 / 9.0 * eta);
  a[3] = V(-16.0 * PI + 4.0 * beta_so);
  a[4] = V(15293365.0 / 508032.0 + 27145.0 / 504.0 * eta + 3085.0 / 72.0 * eta * eta - 10.0 * sigma_ss);
  a[5] = V(PI * (38645.0 / 756.0 - 65.0 / 9.0 * eta)) * (1.0 + 3.0 * (lnv - std::log(vlso)));
  a[6] = V(11583231236531.0 / 4694215680.0 - 640.0 / 3.0 * PI * PI - 6848.0 / 21.0 * EULER_GAMMA +
           (-15737765635.0 / 3048192.0 + 2255.0 / 12.0 * PI * PI) * eta + 76055.0 / 1728.0 * eta * eta -
           127825.0 / 1296.0 * eta * eta * eta) -
         6848.0 / 21.0 * (std::log(4.0) + lnv);
  a[7] = V(PI * (77096675.0 / 254016.0 + 378515.0 / 1512.0 * eta - 74045.0 / 756.0 * eta * eta));
  V sum(0.0);
  V vk(1.0);
  for (int k = 0; k < 8; ++k) { sum = sum + a[k] * vk; vk = vk * v; }
  V v5 = v * v * v * v * v;
  return V(3.0 / 128.0) * sum / (V(eta) * v5);
}

// lift a T into a Dual<T,1> constant
template <class T> inline Dual<T, 1> lift1(const T& x) { return Dual<T, 1>(x, 0); }

// SPA phase of the positive-frequency (l,m) mode, Psi_lm(f) = 2 pi f t_c - m phi_c - pi/4
// + (m/2) Psi_PN(v_m), v_m = (2 pi M f / m)^(1/3); evaluated on any scalar F (F = T or a
// dual number in f).
template <class T, class F>
F psi_lm(const Source<T>& s, int m, const F& f) {
  const T M = s.Mtot * MSUN_S;
  F vm = cbrt(F(2.0 * PI) * F(M) * f / F(double(m)));
  return F(2.0 * PI) * f * F(s.tc) - F(double(m) * s.phic) - F(PI / 4.0) + F(0.5 * m) * psi_pn(s, vm);
}

// Planck taper on the orbital frequency Fo = f/m: 1 below 0.9 F_isco, 0 at and above F_isco
// (McKechan, Robinson & Sathyaprakash 2010 window, here used as a falling edge).
template <class T>
T planck_taper(const Source<T>& s, double f, int m) {
  const T M = s.Mtot * MSUN_S;
  const T Fisco = 1.0 / (std::pow(6.0, 1.5) * 2.0 * PI * M);
  const T F2 = Fisco, F1 = 0.9 * Fisco;
  const double Fo = f / m;
  if (Fo <= val(F1)) return T(1.0);
  if (Fo >= val(F2)) return T(0.0);
  T a = F2 - F1;
  T z = a / (F2 - Fo) - a / (Fo - F1);
  if (val(z) > 700.0) return T(0.0);
  return 1.0 / (1.0 + exp(z));
}

// Leading-order mode factor H_lm(x) of h_lm = 2 M eta x / D sqrt(16 pi/5) H_lm e^{-i m psi}
// (Blanchet, Living Rev. Relativ. 17, 2 (2014), spherical modes at Newtonian order).
// Magnitudes pinned by the multipole flux; the phases (+-i, signs) by the 1PN polarisations.
template <class T>
Cx<T> Hhat(const Source<T>& s, int l, int m, const T& x) {
  const T eta = s.q / ((1.0 + s.q) * (1.0 + s.q));
  const T delta = (s.q - 1.0) / (s.q + 1.0);
  if (l == 2 && m == 2) return Cx<T>(T(1.0), T(0.0));
  if (l == 2 && m == 1) return Cx<T>(T(0.0), delta * sqrt(x) / 3.0);
  if (l == 3 && m == 3) return Cx<T>(T(0.0), -0.75 * std::sqrt(15.0 / 14.0) * delta * sqrt(x));
  if (l == 3 && m == 2) return Cx<T>(std::sqrt(5.0 / 7.0) / 3.0 * (1.0 - 3.0 * eta) * x, T(0.0));
  if (l == 4 && m == 4) return Cx<T>(-8.0 / 9.0 * std::sqrt(5.0 / 7.0) * (1.0 - 3.0 * eta) * x, T(0.0));
  return Cx<T>();
}

// Positive-frequency SPA mode H~_lm(f) = FT[h*_lm](f) and its time-frequency map t_f(f),
// Eq. eq_tf with Phi = -Psi: t_f = (1/2pi) dPsi_lm/df, taken by a dual number in f.
//   H~_lm(f) = (2 pi M^2/D) sqrt(eta/(3m)) x^{-7/4} conj(H_lm(x)) w(f/m) e^{-i Psi_lm(f)},
// x = v_m^2 (stationary-phase amplitude sqrt(2 pi/(m phi'')) with the leading-order
// radiation reaction dOmega/dt = (96/5) eta x^{11/2}/M^2).
template <class T>
void mode_h(const Source<T>& s, int l, int m, double f, Cx<T>* h, T* tf) {
  const T M = s.Mtot * MSUN_S;
  const T D = s.dL * GPC_S;
  const T eta = s.q / ((1.0 + s.q) * (1.0 + s.q));
  typedef Dual<T, 1> F1;
  F1 fd = lift1(T(f)); fd.d[0] = T(1.0);
  F1 ps = psi_lm(s, m, fd);
  *tf = ps.d[0] / (2.0 * PI);
  T w = planck_taper(s, f, m);
  if (val(w) == 0.0) { *h = Cx<T>(); return; }
  T vm = cbrt(2.0 * PI * M * f / double(m));
  T x = vm * vm;
  T amp = 2.0 * PI * M * M / D * sqrt(eta / (3.0 * m)) * pow(x, -1.75) * w;
  Cx<T> H = conj(Hhat(s, l, m, x));
  Cx<T> ph = expi(-ps.v);
  *h = (H * amp) * ph;
}

// ----------------------------------------------------------------------------------------
// Spin-weighted spherical harmonic -2Y_lm(theta, phi=0) from the Wigner-d sum
// (Goldberg et al. 1967; as written in Ajith et al. 2007, arXiv:0709.0093, Eq. II.7-II.8):
//   -sY_lm = (-1)^s sqrt((2l+1)/4pi) d^l_{m,s}(theta),
//   d^l_{m,s} = sum_k (-1)^k sqrt((l+m)!(l-m)!(l+s)!(l-s)!) / ((l+m-k)!(l-s-k)!(k+s-m)! k!)
//               cos(theta/2)^{2l+m-s-2k} sin(theta/2)^{2k+s-m}, with s = 2.
// ----------------------------------------------------------------------------------------
static double fact(int n) { double r = 1.0; for (int i = 2; i <= n; ++i) r *= i; return r; }

template <class T>
T sYlm_m2(int l, int m, const T& theta) {
  const int s = 2;
  T c = cos(theta / 2.0), sn = sin(theta / 2.0);
  T d(0.0);
  const double pre = std::sqrt(fact(l + m) * fact(l - m) * fact(l + s) * fact(l - s));
  for (int k = 0; k <= 2 * l; ++k) {
    if (l + m - k < 0 || l - s - k < 0 || k + s - m < 0) continue;
    double coef = ((k % 2) ? -1.0 : 1.0) * pre / (fact(l + m - k) * fact(l - s - k) * fact(k + s - m) * fact(k));
    int pc = 2 * l + m - s - 2 * k, ps = 2 * k + s - m;
    T term(coef);
    for (int i = 0; i < pc; ++i) term = term * c;
    for (int i = 0; i < ps; ++i) term = term * sn;
    d = d + term;
  }
  return std::sqrt((2.0 * l + 1.0) / (4.0 * PI)) * d;
}

// Polarization weights of one positive-frequency mode (h_{l,-m} = (-1)^l h*_{lm}):
//   h~_+ = 1/2 sum H~_lm [Y*_lm + (-1)^l Y_{l,-m}],  h~_x = i/2 sum H~_lm [(-1)^l Y_{l,-m} - Y*_lm]
// with Y evaluated at (iota, 0), where every Y is real.
template <class T>
void pol_weights(const Source<T>& s, int l, int m, Cx<T>* Pp, Cx<T>* Pc) {
  T Ylm = sYlm_m2(l, m, s.iota);
  T Ylmm = sYlm_m2(l, -m, s.iota);
  double sgn = (l % 2) ? -1.0 : 1.0;
  *Pp = Cx<T>(0.5 * (Ylm + sgn * Ylmm), T(0.0));
  *Pc = Cx<T>(T(0.0), 0.5 * (sgn * Ylmm - Ylm));
}

// ----------------------------------------------------------------------------------------
// Sky and polarization basis: propagation direction k = -(source direction), polarization
// tensors e+ = pp - qq, ex = pq + qp with (p, q) the (u, v) frame rotated by psi.
// ----------------------------------------------------------------------------------------
template <class T>
void sky_basis(const Source<T>& s, T k[3], T ep[3][3], T ec[3][3]) {
  T cl = cos(s.lam), sl = sin(s.lam), cb = cos(s.bet), sb = sin(s.bet);
  T cp = cos(s.psi), sp = sin(s.psi);
  k[0] = -(cb * cl); k[1] = -(cb * sl); k[2] = -sb;
  T u[3] = {sl, -cl, T(0.0)};
  T v[3] = {-(sb * cl), -(sb * sl), cb};
  T p[3], q[3];
  for (int i = 0; i < 3; ++i) { p[i] = cp * u[i] + sp * v[i]; q[i] = -(sp * u[i]) + cp * v[i]; }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) { ep[i][j] = p[i] * p[j] - q[i] * q[j]; ec[i][j] = p[i] * q[j] + q[i] * p[j]; }
}

// ----------------------------------------------------------------------------------------
// Orbits: spacecraft position x_i(t), i = 1..3 (index 0..2), in light-seconds, as the guiding
// centre c(t) plus each spacecraft's offset d_i(t), x_i = c + d_i. The link vectors x_r - x_s are
// formed from the offsets (d_r - d_s): equal in exact arithmetic, and free of the cancellation of
// the 1 au centre that would otherwise cost ~AU/L ulps in every link vector.
// ----------------------------------------------------------------------------------------
template <class T>
void orbit_parts(const OrConfig& cfg, const T& t, T c[3], T d[3][3]) {
  const double L = cfg.arm_m / C_SI;
  if (cfg.orbit == 0) {
    // Rubbo, Cornish & Poujade 2004, Eq. (1)-(3) there: first order in the eccentricity.
    const double R = AU_S;
    const double e = L / (2.0 * std::sqrt(3.0) * R);
    T alpha = cfg.alpha0 + 2.0 * PI * t / YEAR_S;
    c[0] = R * cos(alpha); c[1] = R * sin(alpha); c[2] = T(0.0);
    for (int i = 0; i < 3; ++i) {
      double b = 2.0 * PI * i / 3.0 + cfg.cartwheel0;
      d[i][0] = 0.5 * e * R * (cos(2.0 * alpha - b) - 3.0 * std::cos(b));
      d[i][1] = 0.5 * e * R * (sin(2.0 * alpha - b) - 3.0 * std::sin(b));
      d[i][2] = -std::sqrt(3.0) * e * R * cos(alpha - b);
    }
  } else {
    // Earth on a circular 1 au orbit in the ecliptic plus an equilateral triangle of radius
    // L/sqrt(3) rotating with period P about the fixed normal n(geo_lon, geo_lat).
    const double R = AU_S, r = L / std::sqrt(3.0);
    T alpha = cfg.alpha0 + 2.0 * PI * t / YEAR_S;
    double nl = cfg.geo_lon, nb = cfg.geo_lat;
    double n[3] = {std::cos(nb) * std::cos(nl), std::cos(nb) * std::sin(nl), std::sin(nb)};
    double e1[3] = {-std::sin(nl), std::cos(nl), 0.0};
    double e2[3] = {n[1] * e1[2] - n[2] * e1[1], n[2] * e1[0] - n[0] * e1[2], n[0] * e1[1] - n[1] * e1[0]};
    c[0] = R * cos(alpha); c[1] = R * sin(alpha); c[2] = T(0.0);
    for (int i = 0; i < 3; ++i) {
      T ph = 2.0 * PI * t / cfg.geo_period_s + 2.0 * PI * i / 3.0;
      T ci = cos(ph), si = sin(ph);
      for (int j = 0; j < 3; ++j) d[i][j] = r * (ci * e1[j] + si * e2[j]);
    }
  }
}

template <class T>
void orbit_pos(const OrConfig& cfg, const T& t, T x[3][3]) {
  T c[3], d[3][3];
  orbit_parts(cfg, t, c, d);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) x[i][j] = c[j] + d[i][j];
}

template <class T>
T sinc(const T& x) {
  if (fabs(val(x)) < 1e-3) {
    T x2 = x * x;
    return 1.0 - x2 / 6.0 + x2 * x2 / 120.0 - x2 * x2 * x2 / 5040.0;
  }
  return sin(x) / x;
}

// Single-link FD response of one mode, Eq. eq_fd_resp, link s -> r (1-based r, s):
//   y~_rs = -i pi f L sinc[pi f L (1 - k.n_rs)] exp{-i pi f [L + k.(x_r + x_s)]} n_rs.h~.n_rs
// with n_rs = (x_r - x_s)/|x_r - x_s| and positions taken at t_f of the mode. With x = c + d
// (orbit_parts): x_r - x_s = d_r - d_s, and the phase factor is exp{-i pi f (L + 2 k.c)} times
// exp{-i pi f k.(d_r + d_s)}; the first factor is the same for every link of the bin.
template <class T>
Cx<T> link_response(const OrConfig& cfg, const T k[3], const Cx<T> h[3][3], const T c[3], const T d[3][3],
                    double f, int r, int s) {
  const double L = cfg.arm_m / C_SI;
  T n[3];
  T nn(0.0);
  for (int i = 0; i < 3; ++i) { n[i] = d[r - 1][i] - d[s - 1][i]; nn = nn + n[i] * n[i]; }
  T inv = 1.0 / sqrt(nn);
  for (int i = 0; i < 3; ++i) n[i] = n[i] * inv;
  Cx<T> nhn;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) nhn = nhn + h[i][j] * (n[i] * n[j]);
  T kn = k[0] * n[0] + k[1] * n[1] + k[2] * n[2];
  T kc = k[0] * c[0] + k[1] * c[1] + k[2] * c[2];
  T kd = T(0.0);
  for (int i = 0; i < 3; ++i) kd = kd + k[i] * (d[r - 1][i] + d[s - 1][i]);
  T sc = sinc(PI * f * L * (1.0 - kn));
  Cx<T> pre(T(0.0), T(-PI * f * L) * sc);
  Cx<T> ph = expi(T(-PI * f) * (L + 2.0 * kc)) * expi(T(-PI * f) * kd);
  return (pre * ph) * nhn;
}

// FD TDI (Sec. 2.1): X = (TDI factor)[y13 - y12 + z(y31 - y21)], z = e^{-2 pi i f L}, factor
// (1 - z^2) for generation 1.5 and (1 - z^2 - z^4 + z^6) for 2.0; Y, Z by the cyclic
// permutation 1 -> 2 -> 3 -> 1. Returns X, Y, Z of one mode.
template <class T>
void tdi_xyz_mode(const OrConfig& cfg, const Source<T>& s, int l, int m, double f, const T k[3],
                  const T ep[3][3], const T ec[3][3], Cx<T> xyz[3]) {
  Cx<T> H; T tf;
  mode_h(s, l, m, f, &H, &tf);
  if (val(H.re) == 0.0 && val(H.im) == 0.0) { xyz[0] = xyz[1] = xyz[2] = Cx<T>(); return; }
  Cx<T> Pp, Pc;
  pol_weights(s, l, m, &Pp, &Pc);
  Cx<T> h[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) h[i][j] = H * (Pp * ep[i][j] + Pc * ec[i][j]);
  T c[3], d[3][3];
  orbit_parts(cfg, tf, c, d);
  const double L = cfg.arm_m / C_SI;
  Cx<double> zd(std::cos(-2.0 * PI * f * L), std::sin(-2.0 * PI * f * L));
  Cx<T> z(T(zd.re), T(zd.im));
  Cx<T> z2 = z * z, z4 = z2 * z2, z6 = z4 * z2;
  Cx<T> one(T(1.0));
  Cx<T> fac = (cfg.tdi_gen == 15) ? (one - z2) : (one - z2 - z4 + z6);
  auto y = [&](int r, int ss) { return link_response(cfg, k, h, c, d, f, r, ss); };
  xyz[0] = fac * (y(1, 3) - y(1, 2) + z * (y(3, 1) - y(2, 1)));
  xyz[1] = fac * (y(2, 1) - y(2, 3) + z * (y(1, 2) - y(3, 2)));
  xyz[2] = fac * (y(3, 2) - y(3, 1) + z * (y(2, 3) - y(1, 3)));
}

// A = (Z - X)/sqrt2, E = (X - 2Y + Z)/sqrt6, T = (X + Y + Z)/sqrt3, summed over modes.
template <class T>
void response_aet(const OrConfig& cfg, const Source<T>& s, unsigned mode_mask, double f, Cx<T> aet[3]) {
  T k[3], ep[3][3], ec[3][3];
  sky_basis(s, k, ep, ec);
  Cx<T> X, Y, Z;
  for (int md = 0; md < 5; ++md) {
    if (!(mode_mask & (1u << md))) continue;
    Cx<T> xyz[3];
    tdi_xyz_mode(cfg, s, MODE_L[md], MODE_M[md], f, k, ep, ec, xyz);
    X = X + xyz[0]; Y = Y + xyz[1]; Z = Z + xyz[2];
  }
  const T r2(1.0 / std::sqrt(2.0)), r6(1.0 / std::sqrt(6.0)), r3(1.0 / std::sqrt(3.0));
  aet[0] = (Z - X) * r2;
  aet[1] = (X - Y * T(2.0) + Z) * r6;
  aet[2] = (X + Y + Z) * r3;
}

// ----------------------------------------------------------------------------------------
// Noise PSD of A/E/T in fractional-frequency units (acceleration + OMS noise only, Sec. 3.2;
// equal-arm TDI-1.5 X PSD and XY cross-spectrum, then A/E/T; TDI 2.0 multiplies by
// |1 - z^4|^2 = 4 sin^2(2x), x = 2 pi f L).
// ----------------------------------------------------------------------------------------
void psd_aet(const OrConfig& cfg, double f, double out[3]) {
  const double L = cfg.arm_m / C_SI;
  const double x = 2.0 * PI * f * L;
  double Soms = std::pow(cfg.oms_m_rtHz * 2.0 * PI * f / C_SI, 2);
  double Sacc = std::pow(cfg.acc_ms2_rtHz / (2.0 * PI * f * C_SI), 2);
  if (cfg.psd_shaping) {
    Soms *= 1.0 + std::pow(2e-3 / f, 4);
    Sacc *= (1.0 + std::pow(0.4e-3 / f, 2)) * (1.0 + std::pow(f / 8e-3, 4));
  }
  double sx = std::sin(x), sx2 = std::sin(0.5 * x);
  double SA = 8.0 * sx * sx * ((2.0 + std::cos(x)) * Soms + (6.0 + 4.0 * std::cos(x) + 2.0 * std::cos(2.0 * x)) * Sacc);
  double ST = 32.0 * sx * sx * sx2 * sx2 * (Soms + 4.0 * sx2 * sx2 * Sacc);
  if (cfg.tdi_gen == 20) {
    double s2 = std::sin(2.0 * x);
    SA *= 4.0 * s2 * s2;
    ST *= 4.0 * s2 * s2;
  }
  out[0] = SA; out[1] = SA; out[2] = ST;
}

// ----------------------------------------------------------------------------------------
// Whittle log-likelihood of one detector (Eq. eq_ll_fd, Eq. eq_inner_product):
//   <a|b> = 4 Re sum_k a*(f_k) b(f_k) / (S_c(f_k) T),  f_k = k/T,
//   log L = sum_c ( <d|h>_c - 1/2 <h|h>_c - 1/2 <d|d>_c ) = -1/2 sum_c <d-h|d-h>_c.
// data: [3][nb][2] (re, im), psd: [3][nb].
// ----------------------------------------------------------------------------------------
struct DetData {
  OrConfig cfg;
  double T;
  int64_t k0, nb;
  const double* data;
  const double* psd;
};

template <class T>
void detector_sums(const DetData& D, const Source<T>& s, unsigned mode_mask, T dh[3], T hh[3], T rr[3],
                   double dd[3]) {
  Acc<T> adh[3], ahh[3], arr[3];
  Acc<double> add[3];
  for (int64_t b = 0; b < D.nb; ++b) {
    double f = double(D.k0 + b) / D.T;
    Cx<T> aet[3];
    response_aet(D.cfg, s, mode_mask, f, aet);
    for (int c = 0; c < 3; ++c) {
      double w = 4.0 / (D.psd[c * D.nb + b] * D.T);
      Cx<T> d(T(D.data[(c * D.nb + b) * 2 + 0]), T(D.data[(c * D.nb + b) * 2 + 1]));
      adh[c].add(w * (conj(d) * aet[c]).re);
      ahh[c].add(w * norm2(aet[c]));
      Cx<T> r = d - aet[c];
      arr[c].add(w * norm2(r));
      add[c].add(w * (val(d.re) * val(d.re) + val(d.im) * val(d.im)));
    }
  }
  for (int c = 0; c < 3; ++c) { dh[c] = adh[c].get(); hh[c] = ahh[c].get(); rr[c] = arr[c].get(); dd[c] = add[c].get(); }
}

}  // namespace oracle

using namespace oracle;

// ========================================================================================
// C ABI (ctypes). Arrays are host pointers; complex values are interleaved (re, im).
// ========================================================================================
extern "C" {

int or_abi_version(void) { return 1; }

double or_sylm(int l, int m, double iota) { return sYlm_m2<double>(l, m, iota); }

// Hhat(l, m, x) for mass ratio q: out = (re, im).
void or_hhat(double q, int l, int m, double x, double* out) {
  Source<double> s{};
  s.q = q;
  const Cx<double> h = Hhat(s, l, m, x);
  out[0] = h.re;
  out[1] = h.im;
}

void or_psd(const OrConfig* cfg, const double* f, int64_t n, double* out /*[3][n]*/) {
  for (int64_t i = 0; i < n; ++i) {
    double p[3];
    psd_aet(*cfg, f[i], p);
    for (int c = 0; c < 3; ++c) out[c * n + i] = p[c];
  }
}

void or_orbit(const OrConfig* cfg, double t, double* x /*[3][3]*/) {
  double xx[3][3];
  orbit_pos(*cfg, t, xx);
  for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) x[3 * i + j] = xx[i][j];
}

// one mode: H~_lm(f) (complex) and t_f(f); also Psi_lm(f) for phase checks.
void or_mode(const double* theta, int l, int m, const double* f, int64_t n, double* h, double* tf, double* psi) {
  Source<double> s = source_from(theta);
  for (int64_t i = 0; i < n; ++i) {
    Cx<double> H; double t;
    mode_h(s, l, m, f[i], &H, &t);
    h[2 * i] = H.re; h[2 * i + 1] = H.im; tf[i] = t;
    if (psi) psi[i] = psi_lm(s, m, f[i]);
  }
}

// Psi_PN(v) with the spin and eta of theta (for the closed-form pins).
double or_psi_pn(const double* theta, double v) { Source<double> s = source_from(theta); return psi_pn(s, v); }

double or_taper(const double* theta, double f, int m) { Source<double> s = source_from(theta); return planck_taper(s, f, m); }

void or_polarizations(const double* theta, unsigned mode_mask, const double* f, int64_t n, double* hp, double* hc) {
  Source<double> s = source_from(theta);
  for (int64_t i = 0; i < n; ++i) {
    Cx<double> P, C;
    for (int md = 0; md < 5; ++md) {
      if (!(mode_mask & (1u << md))) continue;
      Cx<double> H, Pp, Pc; double tf;
      mode_h(s, MODE_L[md], MODE_M[md], f[i], &H, &tf);
      pol_weights(s, MODE_L[md], MODE_M[md], &Pp, &Pc);
      P = P + H * Pp; C = C + H * Pc;
    }
    hp[2 * i] = P.re; hp[2 * i + 1] = P.im; hc[2 * i] = C.re; hc[2 * i + 1] = C.im;
  }
}

void or_sky_basis(const double* theta, double* k, double* ep, double* ec) {
  Source<double> s = source_from(theta);
  double kk[3], p[3][3], c[3][3];
  sky_basis(s, kk, p, c);
  for (int i = 0; i < 3; ++i) { k[i] = kk[i]; for (int j = 0; j < 3; ++j) { ep[3 * i + j] = p[i][j]; ec[3 * i + j] = c[i][j]; } }
}

// Single link (r <- s) response of one mode at frequencies f; positions at that mode's t_f,
// unless t_fixed is non-NaN (then positions are frozen at t_fixed, for limit checks).
void or_link(const OrConfig* cfg, const double* theta, int l, int m, const double* f, int64_t n, int r, int sidx,
             double t_fixed, double* out) {
  Source<double> s = source_from(theta);
  double k[3], ep[3][3], ec[3][3];
  sky_basis(s, k, ep, ec);
  Cx<double> Pp, Pc;
  pol_weights(s, l, m, &Pp, &Pc);
  for (int64_t i = 0; i < n; ++i) {
    Cx<double> H; double tf;
    mode_h(s, l, m, f[i], &H, &tf);
    Cx<double> h[3][3];
    for (int a = 0; a < 3; ++a) for (int b = 0; b < 3; ++b) h[a][b] = H * (Pp * ep[a][b] + Pc * ec[a][b]);
    double c[3], d[3][3];
    orbit_parts(*cfg, std::isnan(t_fixed) ? tf : t_fixed, c, d);
    Cx<double> y = link_response(*cfg, k, h, c, d, f[i], r, sidx);
    out[2 * i] = y.re; out[2 * i + 1] = y.im;
  }
}

// A/E/T response: out [3][n][2]
void or_response(const OrConfig* cfg, const double* theta, unsigned mode_mask, const double* f, int64_t n, double* out) {
  Source<double> s = source_from(theta);
  for (int64_t i = 0; i < n; ++i) {
    Cx<double> aet[3];
    response_aet(*cfg, s, mode_mask, f[i], aet);
    for (int c = 0; c < 3; ++c) { out[(c * n + i) * 2] = aet[c].re; out[(c * n + i) * 2 + 1] = aet[c].im; }
  }
}

// The same A/E/T response evaluated in long double (every step of the template above with the
// scalar type long double): an extended-precision twin that bounds the double oracle's own
// rounding, used only by the oracle's pins. out [3][n][2] (rounded back to double).
void or_response_ld(const OrConfig* cfg, const double* theta, unsigned mode_mask, const double* f, int64_t n, double* out) {
  long double th[11];
  for (int i = 0; i < 11; ++i) th[i] = theta[i];
  Source<long double> s = source_from(th);
  for (int64_t i = 0; i < n; ++i) {
    Cx<long double> aet[3];
    response_aet(*cfg, s, mode_mask, f[i], aet);
    for (int c = 0; c < 3; ++c) { out[(c * n + i) * 2] = (double)aet[c].re; out[(c * n + i) * 2 + 1] = (double)aet[c].im; }
  }
}

// Algorithmic work of the method, counted on the oracle's own steps with the operation-counting
// scalar: per active (mode, bin) unit the mode's waveform, t_f, orbit, six links and TDI brackets
// (tdi_xyz_mode), and per bin with at least one active mode the A/E/T combination and the three
// channels' likelihood terms (detector_sums' per-bin body); the sample's sky frame once. Inactive
// (mode, bin) pairs (taper exactly 0) are not counted. data [3][n][2] and psd [3][n] may be NULL
// (zeros and ones). out: [0] active units, [1] active bins, then OP_N counts per unit, OP_N per
// bin, OP_N per sample (add/sub, mul, div, sqrt, sin or cos, exp, log, cbrt, pow, comparisons).
void or_op_count(const OrConfig* cfg, const double* theta, unsigned mode_mask, const double* f, int64_t n,
                 const double* data, const double* psd, double T_obs, double* out) {
  Flop th[11];
  for (int i = 0; i < 11; ++i) th[i] = Flop(theta[i]);
  Source<Flop> s = source_from(th);
  unsigned long long unit[OP_N] = {0}, bin[OP_N] = {0}, samp[OP_N] = {0};
  double n_units = 0.0, n_bins = 0.0;
  for (int k = 0; k < OP_N; ++k) g_ops[k] = 0;
  Flop kv[3], ep[3][3], ec[3][3];
  sky_basis(s, kv, ep, ec);
  for (int k = 0; k < OP_N; ++k) samp[k] = g_ops[k];
  for (int64_t i = 0; i < n; ++i) {
    Cx<Flop> X, Y, Z;
    bool any = false;
    for (int md = 0; md < 5; ++md) {
      if (!(mode_mask & (1u << md))) continue;
      for (int k = 0; k < OP_N; ++k) g_ops[k] = 0;
      Cx<Flop> xyz[3];
      tdi_xyz_mode(*cfg, s, MODE_L[md], MODE_M[md], f[i], kv, ep, ec, xyz);
      const bool active = val(xyz[0].re) != 0.0 || val(xyz[0].im) != 0.0 || val(xyz[1].re) != 0.0 ||
                          val(xyz[1].im) != 0.0 || val(xyz[2].re) != 0.0 || val(xyz[2].im) != 0.0;
      if (!active) continue;
      any = true;
      n_units += 1.0;
      for (int k = 0; k < OP_N; ++k) unit[k] += g_ops[k];
      X = X + xyz[0]; Y = Y + xyz[1]; Z = Z + xyz[2];
    }
    if (!any) continue;
    for (int k = 0; k < OP_N; ++k) g_ops[k] = 0;
    const Flop r2(1.0 / std::sqrt(2.0)), r6(1.0 / std::sqrt(6.0)), r3(1.0 / std::sqrt(3.0));
    Cx<Flop> aet[3] = {(Z - X) * r2, (X - Y * Flop(2.0) + Z) * r6, (X + Y + Z) * r3};
    Acc<Flop> adh, ahh;
    for (int c = 0; c < 3; ++c) {
      const Flop w = Flop(4.0) / (Flop(psd ? psd[c * n + i] : 1.0) * T_obs);
      Cx<Flop> d(Flop(data ? data[(c * n + i) * 2] : 0.0), Flop(data ? data[(c * n + i) * 2 + 1] : 0.0));
      adh.add(w * (conj(d) * aet[c]).re);
      ahh.add(w * norm2(aet[c]));
    }
    n_bins += 1.0;
    for (int k = 0; k < OP_N; ++k) bin[k] += g_ops[k];
  }
  out[0] = n_units;
  out[1] = n_bins;
  for (int k = 0; k < OP_N; ++k) {
    out[2 + k] = n_units > 0 ? (double)unit[k] / n_units : 0.0;
    out[2 + OP_N + k] = n_bins > 0 ? (double)bin[k] / n_bins : 0.0;
    out[2 + 2 * OP_N + k] = (double)samp[k];
  }
}

// X/Y/Z response (mode sum): out [3][n][2]
void or_response_xyz(const OrConfig* cfg, const double* theta, unsigned mode_mask, const double* f, int64_t n, double* out) {
  Source<double> s = source_from(theta);
  double k[3], ep[3][3], ec[3][3];
  sky_basis(s, k, ep, ec);
  for (int64_t i = 0; i < n; ++i) {
    Cx<double> acc[3];
    for (int md = 0; md < 5; ++md) {
      if (!(mode_mask & (1u << md))) continue;
      Cx<double> xyz[3];
      tdi_xyz_mode(*cfg, s, MODE_L[md], MODE_M[md], f[i], k, ep, ec, xyz);
      for (int c = 0; c < 3; ++c) acc[c] = acc[c] + xyz[c];
    }
    for (int c = 0; c < 3; ++c) { out[(c * n + i) * 2] = acc[c].re; out[(c * n + i) * 2 + 1] = acc[c].im; }
  }
}

// Data = injection + noise, noise Re/Im ~ N(0, S T/4) (Eq. eq_diag_Sigma_to_Sn: E|n~|^2 = S T/2).
// normals: [3][nb][2] standard-normal draws supplied by the caller (may be NULL: no noise).
void or_make_data(const OrConfig* cfg, const double* theta, unsigned mode_mask, double T, int64_t k0, int64_t nb,
                  const double* normals, double* data /*[3][nb][2]*/) {
  Source<double> s = source_from(theta);
  for (int64_t b = 0; b < nb; ++b) {
    double f = double(k0 + b) / T;
    Cx<double> aet[3];
    response_aet(*cfg, s, mode_mask, f, aet);
    double p[3];
    psd_aet(*cfg, f, p);
    for (int c = 0; c < 3; ++c) {
      double sig = std::sqrt(p[c] * T / 4.0);
      double nr = normals ? normals[(c * nb + b) * 2] * sig : 0.0;
      double ni = normals ? normals[(c * nb + b) * 2 + 1] * sig : 0.0;
      data[(c * nb + b) * 2] = aet[c].re + nr;
      data[(c * nb + b) * 2 + 1] = aet[c].im + ni;
    }
  }
}

struct OrDetector {  // ABI view of one detector's grid and data
  OrConfig cfg;
  double T;
  int64_t k0, nb;
  const double* data;
  const double* psd;
};

static DetData to_dd(const OrDetector& d) { DetData D{d.cfg, d.T, d.k0, d.nb, d.data, d.psd}; return D; }

// Joint log-likelihood over detectors and channels (Sec. 2.2, product of likelihoods).
// out: [0] logL (component form), [1] logL (residual form -1/2 sum <d-h|d-h>),
//      then per detector: dh[3], hh[3], dd[3].
void or_loglike(const OrDetector* dets, int ndet, const double* theta, unsigned mode_mask, double* out) {
  Source<double> s = source_from(theta);
  Acc<double> L1, L2;
  for (int I = 0; I < ndet; ++I) {
    double dh[3], hh[3], rr[3], dd[3];
    detector_sums(to_dd(dets[I]), s, mode_mask, dh, hh, rr, dd);
    for (int c = 0; c < 3; ++c) {
      L1.add(dh[c]); L1.add(-0.5 * hh[c]); L1.add(-0.5 * dd[c]);
      L2.add(-0.5 * rr[c]);
      out[2 + I * 9 + c] = dh[c]; out[2 + I * 9 + 3 + c] = hh[c]; out[2 + I * 9 + 6 + c] = dd[c];
    }
  }
  out[0] = L1.get(); out[1] = L2.get();
}

// Batched log-likelihood, OpenMP over samples. out_logl[B]; out_dhhh [B][ndet][3][2] or NULL.
void or_loglike_batch(const OrDetector* dets, int ndet, const double* theta, int B, unsigned mode_mask, int nthreads,
                      double* out_logl, double* out_dhhh) {
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
  for (int b = 0; b < B; ++b) {
    std::vector<double> o(2 + 9 * ndet);
    or_loglike(dets, ndet, theta + 11 * b, mode_mask, o.data());
    out_logl[b] = o[0];
    if (out_dhhh)
      for (int I = 0; I < ndet; ++I)
        for (int c = 0; c < 3; ++c) {
          out_dhhh[((b * ndet + I) * 3 + c) * 2 + 0] = o[2 + I * 9 + c];
          out_dhhh[((b * ndet + I) * 3 + c) * 2 + 1] = o[2 + I * 9 + 3 + c];
        }
  }
}

int or_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

// Exact gradient d logL / d theta[11] by forward-mode dual numbers over all 11 parameters.
void or_grad(const OrDetector* dets, int ndet, const double* theta, unsigned mode_mask, double* out_logl, double* grad) {
  typedef Dual<double, 11> D11;
  D11 th[11];
  for (int i = 0; i < 11; ++i) { th[i] = D11(theta[i]); th[i].d[i] = 1.0; }
  Source<D11> s = source_from(th);
  Acc<D11> L;
  for (int I = 0; I < ndet; ++I) {
    D11 dh[3], hh[3], rr[3]; double dd[3];
    detector_sums(to_dd(dets[I]), s, mode_mask, dh, hh, rr, dd);
    for (int c = 0; c < 3; ++c) { L.add(dh[c]); L.add(-0.5 * hh[c]); L.add(D11(-0.5 * dd[c])); }
  }
  D11 r = L.get();
  *out_logl = r.v;
  for (int i = 0; i < 11; ++i) grad[i] = r.d[i];
}

void or_grad_batch(const OrDetector* dets, int ndet, const double* theta, int B, unsigned mode_mask, int nthreads,
                   double* out_logl, double* grad) {
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
  for (int b = 0; b < B; ++b) or_grad(dets, ndet, theta + 11 * b, mode_mask, out_logl + b, grad + 11 * b);
}

// Fisher matrix F_ij = sum_{I,c,k} w Re( conj(dh/dtheta_i) dh/dtheta_j ), Sec. 2.2, with the
// Jacobian of every A/E/T bin taken by dual numbers. out_F: [11][11] row-major.
void or_fisher(const OrDetector* dets, int ndet, const double* theta, unsigned mode_mask, double* out_F) {
  typedef Dual<double, 11> D11;
  D11 th[11];
  for (int i = 0; i < 11; ++i) { th[i] = D11(theta[i]); th[i].d[i] = 1.0; }
  Source<D11> s = source_from(th);
  Acc<double> F[11][11];
  for (int I = 0; I < ndet; ++I) {
    const OrDetector& d = dets[I];
    for (int64_t b = 0; b < d.nb; ++b) {
      double f = double(d.k0 + b) / d.T;
      Cx<D11> aet[3];
      response_aet(d.cfg, s, mode_mask, f, aet);
      for (int c = 0; c < 3; ++c) {
        double w = 4.0 / (d.psd[c * d.nb + b] * d.T);
        for (int i = 0; i < 11; ++i)
          for (int j = 0; j < 11; ++j)
            F[i][j].add(w * (aet[c].re.d[i] * aet[c].re.d[j] + aet[c].im.d[i] * aet[c].im.d[j]));
      }
    }
  }
  for (int i = 0; i < 11; ++i) for (int j = 0; j < 11; ++j) out_F[i * 11 + j] = F[i][j].get();
}

// Jacobian of the A/E/T response at frequencies f: out [n][3][2][11] (d Re/Im of channel c).
void or_response_jac(const OrConfig* cfg, const double* theta, unsigned mode_mask, const double* f, int64_t n, double* out) {
  typedef Dual<double, 11> D11;
  D11 th[11];
  for (int i = 0; i < 11; ++i) { th[i] = D11(theta[i]); th[i].d[i] = 1.0; }
  Source<D11> s = source_from(th);
  for (int64_t k = 0; k < n; ++k) {
    Cx<D11> aet[3];
    response_aet(*cfg, s, mode_mask, f[k], aet);
    for (int c = 0; c < 3; ++c)
      for (int i = 0; i < 11; ++i) {
        out[((k * 3 + c) * 2 + 0) * 11 + i] = aet[c].re.d[i];
        out[((k * 3 + c) * 2 + 1) * 11 + i] = aet[c].im.d[i];
      }
  }
}

}  // extern "C"
