// FP64 CPU oracle for the galaxy-model log-likelihood of Rigamonti et al. (2022),
// "Maximally informed Bayesian modelling of disc galaxies".
//
// TEST INFRASTRUCTURE ONLY.  This file is the slow, plain, obviously-correct restatement
// of the method that the CUDA library is checked against.  Only the test suite, the
// smoke check and the CPU-baseline leg of the benchmark may load it.  It shares no code,
// header, table or constant generator with the CUDA path.
//
// Everything is written once as a template over the scalar type T, instantiated with
// `double` (values) and with `Dual` (forward-mode derivatives with respect to every
// parameter), so the oracle gradient is the exact derivative of the same arithmetic.
//
// Step order follows Algorithm 1 of the paper (model evaluation on CPU): evaluate every
// sub-point of the (padded) oversampled grid, then for each spaxel average the PSF-weighted
// values of its sub-points, then compare with the data through the Gaussian likelihood.
//
// Readings of the paper taken here (each is also listed in the design notes):
//  * Freeman disc velocity (Eq. 9) is garbled as printed; the Binney & Tremaine form
//    v^2 = (2 G M_d / R_d) y^2 [I0 K0 - I1 K1](y), y = r / (2 R_d) is used.
//  * The bulge is the Dehnen (1993) gamma family named in Sec. 2.2; gamma = 1 is Eq. 1
//    (Hernquist) and gamma = 2 is Eq. B1 (Jaffe).  Its projected density (Eq. 4 definition)
//    and isotropic projected dispersion (Eq. 6 definition, bulge potential only) are radial
//    integrals done with r = R cosh t on [0, 16] by an n-node Gauss-Legendre rule; the
//    dispersion uses the single-integral form Sigma sigma^2 = 2G int rho M sqrt(r^2-R^2)/r^2 dr,
//    equivalent to Eq. 6's double integral.
//  * The halo is NFW with M200 and concentration c (rho_crit for H0 = 70 km/s/Mpc).
//  * The PSF of Eq. 21 is a normalised Gaussian over a square window of half-width
//    h = floor(3 sigma / p) fine pixels (p the fine pitch); B, v, sigma and <L/M> are each
//    convolved on their own; the model M/L is 1/<L/M> (footnote to Eq. 19).
//  * Oversampling: an os x os fine grid per spaxel, padded by h fine pixels on every side,
//    convolved then averaged per spaxel.
//  * PSF modes (bits of psf_mode): 1 - the window is the circle of radius 3 sigma that
//    Eq. 21 names instead of the square; 2 - App. A's centre sampling: each spaxel's value
//    is the PSF-weighted mean of the fine points around its centre (no average over its
//    sub-points); 4 - flux-weighted moments: B, B v, B (sigma^2 + v^2) and the surface
//    mass are convolved, and v, sigma and M/L are formed from them per spaxel.
//  * Likelihood (Eq. 18): each term is Gaussian, logL = -chi^2/2 - sum ln(sqrt(2 pi) delta).
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

constexpr int PMAX = 19;                       // largest parameter vector (two discs)
constexpr double kPi = 3.14159265358979323846;
constexpr double kG = 4.30091727e-6;           // kpc (km/s)^2 / Msun
constexpr double kRhoCrit = 3.0 * 0.07 * 0.07 / (8.0 * kPi * kG);  // Msun/kpc^3, H0 = 70 km/s/Mpc
constexpr double kTmax = 16.0;                 // upper limit of t in r = R cosh t
constexpr double kRfloor2 = 1e-12;             // radii are floored at 1e-6 kpc

// ------------------------------------------------------------------ forward-mode duals
struct Dual {
  double v;
  double d[PMAX];
  Dual() : v(0.0) { for (int i = 0; i < PMAX; ++i) d[i] = 0.0; }
  Dual(double x) : v(x) { for (int i = 0; i < PMAX; ++i) d[i] = 0.0; }
};

inline double val(double x) { return x; }
inline double val(const Dual& x) { return x.v; }

// chain rule helper: result value fv, derivative factor df/dx
inline Dual chain(const Dual& x, double fv, double dfdx) {
  Dual r; r.v = fv;
  for (int i = 0; i < PMAX; ++i) r.d[i] = dfdx * x.d[i];
  return r;
}

inline Dual operator+(const Dual& a, const Dual& b) { Dual r; r.v = a.v + b.v; for (int i = 0; i < PMAX; ++i) r.d[i] = a.d[i] + b.d[i]; return r; }
inline Dual operator-(const Dual& a, const Dual& b) { Dual r; r.v = a.v - b.v; for (int i = 0; i < PMAX; ++i) r.d[i] = a.d[i] - b.d[i]; return r; }
inline Dual operator-(const Dual& a) { Dual r; r.v = -a.v; for (int i = 0; i < PMAX; ++i) r.d[i] = -a.d[i]; return r; }
inline Dual operator*(const Dual& a, const Dual& b) { Dual r; r.v = a.v * b.v; for (int i = 0; i < PMAX; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i]; return r; }
inline Dual operator/(const Dual& a, const Dual& b) {
  Dual r; r.v = a.v / b.v; const double ib = 1.0 / b.v;
  for (int i = 0; i < PMAX; ++i) r.d[i] = (a.d[i] - r.v * b.d[i]) * ib;
  return r;
}
inline Dual operator+(const Dual& a, double b) { Dual r = a; r.v += b; return r; }
inline Dual operator+(double a, const Dual& b) { return b + a; }
inline Dual operator-(const Dual& a, double b) { Dual r = a; r.v -= b; return r; }
inline Dual operator-(double a, const Dual& b) { Dual r = -b; r.v += a; return r; }
inline Dual operator*(const Dual& a, double b) { Dual r; r.v = a.v * b; for (int i = 0; i < PMAX; ++i) r.d[i] = a.d[i] * b; return r; }
inline Dual operator*(double a, const Dual& b) { return b * a; }
inline Dual operator/(const Dual& a, double b) { return a * (1.0 / b); }
inline Dual operator/(double a, const Dual& b) { return Dual(a) / b; }
inline Dual& operator+=(Dual& a, const Dual& b) { a = a + b; return a; }

inline Dual exp(const Dual& x) { const double e = std::exp(x.v); return chain(x, e, e); }
inline Dual log(const Dual& x) { return chain(x, std::log(x.v), 1.0 / x.v); }
inline Dual log1p(const Dual& x) { return chain(x, std::log1p(x.v), 1.0 / (1.0 + x.v)); }
inline Dual sqrt(const Dual& x) { const double s = std::sqrt(x.v); return chain(x, s, 0.5 / s); }
inline Dual sin(const Dual& x) { return chain(x, std::sin(x.v), std::cos(x.v)); }
inline Dual cos(const Dual& x) { return chain(x, std::cos(x.v), -std::sin(x.v)); }
inline Dual pow(const Dual& x, double p) { return chain(x, std::pow(x.v, p), p * std::pow(x.v, p - 1.0)); }
inline Dual pow(const Dual& x, const Dual& p) { return exp(p * log(x)); }
inline Dual pow(double x, const Dual& p) { return exp(p * std::log(x)); }

using std::exp; using std::log; using std::log1p; using std::sqrt; using std::sin; using std::cos; using std::pow;

// I0(y)K0(y) - I1(y)K1(y) and its derivative, from the libstdc++ C++17 special functions.
// d/dy uses I0' = I1, K0' = -K1, I1' = I0 - I1/y, K1' = -K0 - K1/y.
inline void bessel_diff_raw(double y, double* f, double* df) {
  const double i0 = std::cyl_bessel_i(0.0, y), i1 = std::cyl_bessel_i(1.0, y);
  const double k0 = std::cyl_bessel_k(0.0, y), k1 = std::cyl_bessel_k(1.0, y);
  *f = i0 * k0 - i1 * k1;
  *df = 2.0 * (i1 * k0 - i0 * k1) + 2.0 * i1 * k1 / y;
}
inline double bessel_diff(double y) { double f, df; bessel_diff_raw(y, &f, &df); return f; }
inline Dual bessel_diff(const Dual& y) { double f, df; bessel_diff_raw(y.v, &f, &df); return chain(y, f, df); }

// radius with the 1e-6 kpc floor, from its square
template <class T> T floored_sqrt(const T& x2) { return val(x2) < kRfloor2 ? T(std::sqrt(kRfloor2)) : sqrt(x2); }

// ------------------------------------------------------------------ quadrature rule
// Gauss-Legendre nodes and weights on [-1, 1] by Newton iteration on P_n, with P_n and
// P_n' from the three-term Legendre recurrence (a textbook method).
void gauss_legendre(int n, double* x, double* w) {
  for (int k = 0; k < n; ++k) {
    double z = std::cos(kPi * (k + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int j = 2; j <= n; ++j) { const double p2 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p0) / j; p0 = p1; p1 = p2; }
      const double dp = n * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    double p0 = 1.0, p1 = z;
    for (int j = 2; j <= n; ++j) { const double p2 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p0) / j; p0 = p1; p1 = p2; }
    const double dp = n * (z * p1 - p0) / (z * z - 1.0);
    x[n - 1 - k] = z;                                     // ascending order
    w[n - 1 - k] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

// The fixed radial rule: t_k in [0, T], weights w_k, with cosh t_k and tanh^2 t_k.
struct RadialRule {
  int n = 0;
  std::vector<double> t, w, ch, th2;
  explicit RadialRule(int nq) : n(nq), t(nq), w(nq), ch(nq), th2(nq) {
    std::vector<double> x(nq), wg(nq);
    gauss_legendre(nq, x.data(), wg.data());
    for (int k = 0; k < nq; ++k) {
      t[k] = 0.5 * kTmax * (x[k] + 1.0);
      w[k] = 0.5 * kTmax * wg[k];
      ch[k] = std::cosh(t[k]);
      const double th = std::tanh(t[k]);
      th2[k] = th * th;
    }
  }
};

// ------------------------------------------------------------------ components
// Dehnen (1993) density, gamma family: gamma = 1 reproduces Eq. 1, gamma = 2 Eq. B1.
template <class T> T dehnen_rho(const T& r, const T& a, const T& g, const T& M) {
  return (3.0 - g) * M * a / (4.0 * kPi) * pow(r, -g) * pow(r + a, g - 4.0);
}
// Dehnen enclosed mass M(<r) = M (r / (r + a))^(3 - gamma).
template <class T> T dehnen_mass(const T& r, const T& a, const T& g, const T& M) {
  return M * pow(r / (r + a), 3.0 - g);
}

// Projected surface density (Eq. 4 definition) and isotropic projected dispersion
// (Eq. 6 definition, the bulge's own potential only as Sec. 2.2 states) at sky radius R.
// With r = R cosh t:  Sigma = 2 int_0^T rho(r) r dt,
//                     Sigma sigma^2 = 2 G int_0^T rho(r) M(r) tanh^2 t dt.
template <class T>
void bulge_projected(const T& R, const T& a, const T& g, const T& M, const RadialRule& q, T* Sigma, T* sigma2) {
  T s(0.0), p(0.0);
  for (int k = 0; k < q.n; ++k) {
    const T r = R * q.ch[k];
    const T rho = dehnen_rho(r, a, g, M);
    s += q.w[k] * rho * r;
    p += q.w[k] * q.th2[k] * rho * dehnen_mass(r, a, g, M);
  }
  *Sigma = 2.0 * s;
  *sigma2 = 2.0 * kG * p / *Sigma;
}

// The closed forms of the paper for the projected density and dispersion of the Hernquist
// bulge (Eqs. 4-6, X(s) of Eq. 5 for s = R / a < 1) and of the Jaffe bulge (Eqs. B4-B5), for
// the closed-form bulge option at s < 1e-3.  There the fixed radial rule, which reaches only
// r = R cosh 16 ~ 4.4e6 R, no longer covers a Hernquist bulge, while the closed forms have no
// cancellation (they do near s = 1 and, for the dispersion, at large s, where the rule is
// used instead).
template <class T>
void bulge_closed_small(const T& R, const T& a, int kind, const T& M, T* Sigma, T* sigma2) {
  const T s = R / a;
  const T q = 1.0 - s * s;
  const T X = log((1.0 + sqrt(q)) / s) / sqrt(q);
  if (kind == 1) {
    *Sigma = M / (2.0 * kPi * a * a * q * q) * ((2.0 + s * s) * X - 3.0);
    const T brace = (-3.0 * s * s * X * (8.0 * pow(s, 6.0) - 28.0 * pow(s, 4.0) + 35.0 * s * s - 20.0)
                     - 24.0 * pow(s, 6.0) + 68.0 * pow(s, 4.0) - 65.0 * s * s + 6.0) / (2.0 * q * q * q)
                    - 6.0 * kPi * s;
    *sigma2 = kG * M * M / (12.0 * kPi * a * a * a * *Sigma) * brace;
    return;
  }
  *Sigma = M / (a * a) * (1.0 / (4.0 * s) + (1.0 - (2.0 - s * s) * X) / (2.0 * kPi * q));
  const T br = kPi / (2.0 * s) + 11.0 - 6.5 * kPi * s - 12.0 * s * s + 6.0 * kPi * s * s * s
               - X * (6.0 - 19.0 * s * s + 12.0 * pow(s, 4.0));
  *sigma2 = kG * M * M / (4.0 * kPi * a * a * a * *Sigma) / q * br;
}

// The bulge's projected density and dispersion as the model uses them: the radial rule,
// or for the closed-form bulges (kind 1, 2) their closed forms below s = 1e-3.
template <class T>
void bulge_model(const T& R, const T& a, const T& g, const T& M, int kind, const RadialRule& q, T* Sigma,
                 T* sigma2) {
  if (kind != 0 && val(R / a) < 1e-3) bulge_closed_small(R, a, kind, M, Sigma, sigma2);
  else bulge_projected(R, a, g, M, q, Sigma, sigma2);
}

// Circular velocity squared of the bulge at 3-D radius r: G M(<r) / r (Eq. 2 at gamma = 1).
template <class T> T bulge_vc2(const T& r, const T& a, const T& g, const T& M) {
  return kG * dehnen_mass(r, a, g, M) / r;
}

// NFW halo from M200 and concentration: G M(<r) / r with M(<r) = M200 m(r/rs) / m(c).
template <class T> T nfw_m(const T& x) { return log1p(x) - x / (1.0 + x); }
template <class T> T nfw_vc2(const T& r, const T& M200, const T& c) {
  const T r200 = pow(3.0 * M200 / (4.0 * kPi * 200.0 * kRhoCrit), 1.0 / 3.0);
  const T rs = r200 / c;
  return kG * M200 * nfw_m(r / rs) / (nfw_m(c) * r);
}

// Hernquist halo (the paper's, Sec. 2.2): v^2 = G M r / (r + R)^2, Eq. 2 with the halo's
// mass and scale radius.
template <class T> T hernquist_vc2(const T& r, const T& M, const T& Rh) {
  return kG * M * r / ((r + Rh) * (r + Rh));
}
template <class T> T halo_vc2(const T& r, const T& M, const T& p, int halo) {
  return halo == 0 ? nfw_vc2(r, M, p) : hernquist_vc2(r, M, p);
}

// Razor-thin exponential disc: circular velocity squared (Eq. 9, Binney & Tremaine form).
template <class T> T freeman_vc2(const T& r, const T& Md, const T& Rd) {
  const T y = r / (2.0 * Rd);
  return 2.0 * kG * Md / Rd * y * y * bessel_diff(y);
}

// ------------------------------------------------------------------ parameters
// Parameter vector layout (angles in radians, masses and radii as log10 of Msun and kpc):
//  0 x0, 1 y0 [kpc], 2 PA, 3 i, 4 log Mb, 5 log Rb, 6 gamma, 7 log Md1, 8 log Rd1, 9 k1,
//  10 (M/L)b, 11 (M/L)d1, 12 log M200, 13 c, 14 v_sys [km/s],
//  15 log Md2, 16 log Rd2, 17 k2, 18 (M/L)d2 (two-disc models only).
template <class T> struct Model {
  int nd;
  T x0, y0, cpa, spa, ci, si;
  T a, g, Mb, MLb;
  T Md[2], Rd[2], k[2], MLd[2];
  int halo;             // 0: NFW (M200, c); 1: Hernquist (M_h, R_h), the paper's halo
  int bulge_kind;       // 0: Dehnen gamma; 1: Hernquist, 2: Jaffe (closed forms at small R/a)
  T M200, c, vsys;      // for the Hernquist halo M200 holds M_h and c holds R_h
};

// bulge_kind 1 (Hernquist, Eqs. 1-6) and 2 (Jaffe, Eqs. B1-B5) fix gamma at 1 and 2: the
// theta slot of gamma is then not used (zero gradient) and the bulge is the same radial
// quadrature at that gamma (the closed forms equal it, see the bulge pins).
template <class T> Model<T> decode(const T* th, int nd, int halo, int bulge_kind = 0) {
  Model<T> m;
  m.nd = nd;
  m.x0 = th[0]; m.y0 = th[1];
  m.cpa = cos(th[2]); m.spa = sin(th[2]);
  m.ci = cos(th[3]); m.si = sin(th[3]);
  m.Mb = pow(10.0, th[4]); m.a = pow(10.0, th[5]);
  m.g = bulge_kind == 0 ? th[6] : T((double)bulge_kind);
  m.bulge_kind = bulge_kind;
  m.Md[0] = pow(10.0, th[7]); m.Rd[0] = pow(10.0, th[8]); m.k[0] = th[9];
  m.MLb = th[10]; m.MLd[0] = th[11];
  m.halo = halo;
  m.M200 = pow(10.0, th[12]); m.vsys = th[14];
  m.c = halo == 0 ? th[13] : pow(10.0, th[13]);
  if (nd == 2) { m.Md[1] = pow(10.0, th[15]); m.Rd[1] = pow(10.0, th[16]); m.k[1] = th[17]; m.MLd[1] = th[18]; }
  return m;
}

bool in_domain(const double* th, int np, int halo, int bulge_kind = 0) {
  for (int i = 0; i < np; ++i) if (!std::isfinite(th[i])) return false;
  if (!(th[3] >= 0.0 && th[3] < 0.5 * kPi)) return false;   // inclination
  if (bulge_kind == 0 && !(th[6] >= 0.0 && th[6] < 3.0)) return false;   // Dehnen inner slope
  if (!(std::fabs(th[9]) <= 1.0)) return false;             // Satoh k
  if (!(th[10] > 0.0 && th[11] > 0.0)) return false;        // M/L
  if (halo == 0 && !(th[13] > 0.0)) return false;           // NFW concentration
  if (np == 19 && !(std::fabs(th[17]) <= 1.0 && th[18] > 0.0)) return false;
  return true;
}

// ------------------------------------------------------------------ one sky point
// The four light-weighted observables at one sky point (arcsec): B_tot (Eq. 13, Lsun/pc^2),
// v_los (Eq. 14), sigma_los (Eq. 15) and <L/M> (Eq. 19).
// With flux = true the four outputs are instead the quantities a flux-weighted PSF
// convolves: B, B v_los, B (sigma_los^2 + v_los^2) and the surface mass (1e-6 Sigma, so
// that M/L = its convolution over B's).
template <class T>
void eval_point(const Model<T>& m, double xs, double ys, double kpa, const RadialRule& q, T out[4],
                bool flux = false) {
  // Sec. 2.1: move the centre to the origin, rotate the major axis onto x (footnote on P.A.).
  const T X = xs * kpa - m.x0, Y = ys * kpa - m.y0;
  const T xr = X * m.cpa + Y * m.spa;
  const T yr = -X * m.spa + Y * m.cpa;
  const T R = floored_sqrt(xr * xr + yr * yr);              // projected radius
  // disc plane (razor-thin discs): stretch the minor axis by 1/cos i
  const T yd = yr / m.ci;
  const T r = floored_sqrt(xr * xr + yd * yd);              // in-plane radius
  const T cphi = xr / r;                                    // azimuth from the major axis

  T Sb, s2b;
  bulge_model(R, m.a, m.g, m.Mb, m.bulge_kind, q, &Sb, &s2b);

  // Eq. 10: every component's circular velocity adds in quadrature
  T vint2 = bulge_vc2(r, m.a, m.g, m.Mb) + halo_vc2(r, m.M200, m.c, m.halo);
  T Sd[2], vd[2], s2d[2];
  for (int j = 0; j < m.nd; ++j) vint2 += freeman_vc2(r, m.Md[j], m.Rd[j]);
  const T vint = sqrt(vint2);
  for (int j = 0; j < m.nd; ++j) {
    Sd[j] = m.Md[j] / (2.0 * kPi * m.Rd[j] * m.Rd[j]) * exp(-r / m.Rd[j]) / m.ci;  // Eqs. 7-8
    vd[j] = -m.k[j] * m.si * cphi * vint;                                           // Eq. 11
    s2d[j] = (1.0 - m.k[j] * m.k[j]) * vint2 / 3.0;                                 // Eq. 12
  }
  // Eq. 13: B = Sigma / (M/L); Sigma in Msun/kpc^2 -> Lsun/pc^2 with the factor 1e-6
  const T Bb = Sb * 1e-6 / m.MLb;
  T B = Bb, Bv(0.0), Bs2 = Bb * s2b, Stot = Sb;
  for (int j = 0; j < m.nd; ++j) {
    const T Bd = Sd[j] * 1e-6 / m.MLd[j];
    B += Bd; Bv += Bd * vd[j]; Bs2 += Bd * s2d[j]; Stot += Sd[j];
  }
  if (flux) {
    out[0] = B;
    out[1] = Bv;
    out[2] = Bs2 + Bv * Bv / B;       // B (sigma^2 + v^2)
    out[3] = 1e-6 * Stot;
    return;
  }
  out[0] = B;
  out[1] = Bv / B;                    // Eq. 14
  out[2] = sqrt(Bs2 / B);             // Eq. 15
  out[3] = B / (1e-6 * Stot);         // Eq. 19, L/M in Lsun/Msun
}

// ------------------------------------------------------------------ grid and PSF
enum { kPsfCircle = 1, kPsfCentre = 2, kPsfFlux = 4 };

struct Galaxy {
  int nx, ny, os, h;
  double dpix, kpa, pitch;
  int psf_kind; double fwhm, beta;
  int psf_mode;   // bits kPsfCircle, kPsfCentre, kPsfFlux
  double rho;     // window radius 3 sigma in fine pixels (0 without a PSF)
  const double* data; const double* err; const uint8_t* mask;
  int W() const { return os * nx + 2 * h; }
  int H() const { return os * ny + 2 * h; }
  // sky coordinate (arcsec) of padded fine column / row index q
  double xq(int q) const { return dpix * ((q - h + 0.5) / os - 0.5 * nx); }
  double yq(int q) const { return dpix * ((q - h + 0.5) / os - 0.5 * ny); }
};

// Gaussian sigma from the FWHM; the window half-width is floor(3 sigma / pitch) (Eq. 21,
// "within 3 sigma").  The Moffat PSF uses the same window with sigma = FWHM / 2.35482.
int psf_halfwidth(double fwhm, double pitch) {
  const double sig = fwhm / (2.0 * std::sqrt(2.0 * std::log(2.0)));
  return (int)std::floor(3.0 * sig / pitch);
}

// Unnormalised PSF value at a fine-pixel offset (dx, dy) (Eq. 21's Gaussian, or Moffat).
double psf_value(const Galaxy& g, double dx, double dy) {
  const double d2 = (dx * dx + dy * dy) * g.pitch * g.pitch;
  if (g.psf_kind == 0) {
    const double sig = g.fwhm / (2.0 * std::sqrt(2.0 * std::log(2.0)));
    return std::exp(-d2 / (2.0 * sig * sig));
  }
  const double alpha = g.fwhm / (2.0 * std::sqrt(std::pow(2.0, 1.0 / g.beta) - 1.0));
  return std::pow(1.0 + d2 / (alpha * alpha), -g.beta);
}

// Is the offset (dx, dy) (fine pixels) inside the PSF window: the square |dx|, |dy| <=
// 3 sigma, or with kPsfCircle the circle of radius 3 sigma.
bool in_window(const Galaxy& g, double dx, double dy) {
  if (g.psf_mode & kPsfCircle) return dx * dx + dy * dy <= g.rho * g.rho;
  return std::fabs(dx) <= g.rho && std::fabs(dy) <= g.rho;
}

// Normalised 2-D PSF weights W[(dy + h) * (2h+1) + (dx + h)] (Eq. 21).
std::vector<double> psf_weights(const Galaxy& g) {
  const int n = 2 * g.h + 1;
  std::vector<double> w(n * n, 0.0);
  if (g.h == 0) { w[0] = 1.0; return w; }                  // no PSF: the identity
  double tot = 0.0;
  for (int dy = -g.h; dy <= g.h; ++dy)
    for (int dx = -g.h; dx <= g.h; ++dx) {
      if (!in_window(g, dx, dy)) continue;
      const double v = psf_value(g, dx, dy);
      w[(dy + g.h) * n + (dx + g.h)] = v;
      tot += v;
    }
  for (double& v : w) v /= tot;
  return w;
}

// Evaluate the four observables on every point of the padded fine grid: field[c][qy][qx].
template <class T>
void fine_field(const Galaxy& g, const Model<T>& m, const RadialRule& q, std::vector<T>& f) {
  const int W = g.W(), H = g.H();
  const bool flux = (g.psf_mode & kPsfFlux) != 0;
  f.assign((size_t)4 * W * H, T(0.0));
#pragma omp parallel for schedule(static)
  for (int qy = 0; qy < H; ++qy)
    for (int qx = 0; qx < W; ++qx) {
      T o[4];
      eval_point(m, g.xq(qx), g.yq(qy), g.kpa, q, o, flux);
      for (int c = 0; c < 4; ++c) f[((size_t)c * H + qy) * W + qx] = o[c];
    }
}

// App. A's centre sampling (kPsfCentre): each spaxel's value is the PSF-weighted mean
// (Eq. 21) of the fine points around its centre, fine coordinate (h + i os + (os-1)/2,
// h + j os + (os-1)/2): the points inside the window, and always the one to four points
// nearest the centre (|dx|, |dy| <= 1/2), which alone are used without a PSF (equal
// weights).
template <class T>
void convolve_centre(const Galaxy& g, const std::vector<T>& f, std::vector<T>& maps) {
  const int W = g.W(), H = g.H();
  maps.assign((size_t)4 * g.nx * g.ny, T(0.0));
#pragma omp parallel for schedule(static)
  for (int j = 0; j < g.ny; ++j)
    for (int i = 0; i < g.nx; ++i) {
      const double cx = g.h + i * g.os + 0.5 * (g.os - 1), cy = g.h + j * g.os + 0.5 * (g.os - 1);
      T acc[4] = {T(0.0), T(0.0), T(0.0), T(0.0)};
      double tot = 0.0;
      for (int qy = 0; qy < H; ++qy)
        for (int qx = 0; qx < W; ++qx) {
          const double dx = qx - cx, dy = qy - cy;
          const bool nearest = std::fabs(dx) <= 0.5 && std::fabs(dy) <= 0.5;
          if (!nearest && !(g.fwhm > 0.0 && in_window(g, dx, dy))) continue;
          const double w = g.fwhm > 0.0 ? psf_value(g, dx, dy) : 1.0;
          tot += w;
          for (int c = 0; c < 4; ++c) acc[c] += w * f[((size_t)c * H + qy) * W + qx];
        }
      for (int c = 0; c < 4; ++c) maps[((size_t)c * g.ny + j) * g.nx + i] = acc[c] / tot;
    }
}

// Algorithm 1, second step: for each spaxel, average over its os x os sub-points the
// PSF-weighted mean of the field around each sub-point (Eq. 21).  maps[c][j][i].
template <class T>
void convolve_bin(const Galaxy& g, const std::vector<double>& wts, const std::vector<T>& f, std::vector<T>& maps) {
  if (g.psf_mode & kPsfCentre) {
    convolve_centre(g, f, maps);
    return;
  }
  const int W = g.W(), H = g.H(), n = 2 * g.h + 1;
  maps.assign((size_t)4 * g.nx * g.ny, T(0.0));
#pragma omp parallel for schedule(static)
  for (int j = 0; j < g.ny; ++j)
    for (int i = 0; i < g.nx; ++i)
      for (int c = 0; c < 4; ++c) {
        const T* fc = &f[(size_t)c * H * W];
        T acc(0.0);
        for (int sn = 0; sn < g.os; ++sn)
          for (int sm = 0; sm < g.os; ++sm) {
            const int qx = g.h + i * g.os + sm, qy = g.h + j * g.os + sn;   // the sub-point
            T conv(0.0);
            for (int dy = -g.h; dy <= g.h; ++dy)
              for (int dx = -g.h; dx <= g.h; ++dx)
                conv += wts[(dy + g.h) * n + (dx + g.h)] * fc[(size_t)(qy + dy) * W + (qx + dx)];
            acc += conv;
          }
        maps[((size_t)c * g.ny + j) * g.nx + i] = acc / (double)(g.os * g.os);
      }
}

// Observable maps compared with the data: B, v_los + v_sys, sigma_los, M/L = 1 / <L/M>.
// Flux-weighted moments: v = C1 / C0, sigma^2 = C2 / C0 - v^2, M/L = C3 / C0.
template <class T>
void observables(const Galaxy& g, const Model<T>& m, std::vector<T>& maps) {
  const size_t n = (size_t)g.nx * g.ny;
  for (size_t s = 0; s < n; ++s) {
    if (g.psf_mode & kPsfFlux) {
      const T B = maps[s], v = maps[n + s] / B;
      const T s2 = maps[2 * n + s] / B - v * v;
      maps[n + s] = v + m.vsys;
      maps[2 * n + s] = sqrt(s2);
      maps[3 * n + s] = maps[3 * n + s] / B;
      continue;
    }
    maps[n + s] = maps[n + s] + m.vsys;
    maps[3 * n + s] = 1.0 / maps[3 * n + s];
  }
}

template <class T>
void model_maps(const Galaxy& g, const Model<T>& m, const RadialRule& q, std::vector<T>& maps) {
  std::vector<T> f;
  fine_field(g, m, q, f);
  convolve_bin(g, psf_weights(g), f, maps);
  observables(g, m, maps);
}

// Eq. 18 with Gaussian terms: chi^2 over the four maps and the normalisation constant.
template <class T>
T chi2_of(const Galaxy& g, const std::vector<T>& maps) {
  const size_t n = (size_t)4 * g.nx * g.ny;
  T chi(0.0);
  for (size_t s = 0; s < n; ++s) {
    if (g.mask && !g.mask[s]) continue;
    const T r = (maps[s] - g.data[s]) / g.err[s];
    chi += r * r;
  }
  return chi;
}
double norm_const(const Galaxy& g) {
  const size_t n = (size_t)4 * g.nx * g.ny;
  double c = 0.0;
  for (size_t s = 0; s < n; ++s) {
    if (g.mask && !g.mask[s]) continue;
    c += std::log(std::sqrt(2.0 * kPi) * g.err[s]);
  }
  return c;
}

}  // namespace

// ================================================================== C ABI
extern "C" {

typedef struct {
  int nx, ny, oversample;
  double spaxel_arcsec, kpc_per_arcsec;
  int psf_kind;            // 0 Gaussian, 1 Moffat
  double psf_fwhm_arcsec, moffat_beta;
  const double* data;      // [4][ny][nx]: B, v, sigma, M/L
  const double* err;       // [4][ny][nx]: delta > 0
  const uint8_t* mask;     // [4][ny][nx] or NULL
  int psf_mode;            // bits: 1 circular window, 2 centre sampling, 4 flux-weighted
} bang_oracle_galaxy;

typedef struct { int n_discs; int n_quad; int halo_kind; int bulge_kind; } bang_oracle_opts;

static Galaxy make_galaxy(const bang_oracle_galaxy* d) {
  Galaxy g;
  g.nx = d->nx; g.ny = d->ny; g.os = d->oversample;
  g.dpix = d->spaxel_arcsec; g.kpa = d->kpc_per_arcsec; g.pitch = d->spaxel_arcsec / d->oversample;
  g.psf_kind = d->psf_kind; g.fwhm = d->psf_fwhm_arcsec; g.beta = d->moffat_beta;
  g.h = d->psf_fwhm_arcsec > 0.0 ? psf_halfwidth(d->psf_fwhm_arcsec, g.pitch) : 0;
  g.psf_mode = d->psf_mode;
  g.rho = d->psf_fwhm_arcsec > 0.0 ? 3.0 * d->psf_fwhm_arcsec / (2.0 * std::sqrt(2.0 * std::log(2.0))) / g.pitch : 0.0;
  g.data = d->data; g.err = d->err; g.mask = d->mask;
  return g;
}

static void set_threads(int nthreads) {
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
}

int bang_oracle_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

int bang_oracle_nparams(int n_discs) { return n_discs == 2 ? 19 : 15; }

int bang_oracle_psf_halfwidth(const bang_oracle_galaxy* d) { return make_galaxy(d).h; }

void bang_oracle_gauss_legendre(int n, double* x, double* w) { gauss_legendre(n, x, w); }

int bang_oracle_psf_weights(const bang_oracle_galaxy* d, double* w) {
  const Galaxy g = make_galaxy(d);
  const std::vector<double> v = psf_weights(g);
  std::memcpy(w, v.data(), v.size() * sizeof(double));
  return (int)v.size();
}

void bang_oracle_bulge_projected(double R, double a, double gamma, double M, int nq, double* Sigma, double* sigma2) {
  const RadialRule q(nq);
  bulge_projected(R, a, gamma, M, q, Sigma, sigma2);
}
void bang_oracle_bulge_model(double R, double a, double gamma, double M, int nq, int bulge_kind, double* Sigma,
                             double* sigma2) {
  const RadialRule q(nq);
  bulge_model(R, a, bulge_kind == 0 ? gamma : (double)bulge_kind, M, bulge_kind, q, Sigma, sigma2);
}
double bang_oracle_bulge_vc2(double r, double a, double gamma, double M) { return bulge_vc2(r, a, gamma, M); }
double bang_oracle_dehnen_rho(double r, double a, double gamma, double M) { return dehnen_rho(r, a, gamma, M); }
double bang_oracle_dehnen_mass(double r, double a, double gamma, double M) { return dehnen_mass(r, a, gamma, M); }
double bang_oracle_nfw_vc2(double r, double M200, double c) { return nfw_vc2(r, M200, c); }
double bang_oracle_hernquist_halo_vc2(double r, double Mh, double Rh) { return hernquist_vc2(r, Mh, Rh); }
double bang_oracle_nfw_r200(double M200) { return std::pow(3.0 * M200 / (4.0 * kPi * 200.0 * kRhoCrit), 1.0 / 3.0); }
double bang_oracle_freeman_vc2(double r, double Md, double Rd) { return freeman_vc2(r, Md, Rd); }
double bang_oracle_bessel_diff(double y) { return bessel_diff(y); }
double bang_oracle_G(void) { return kG; }
double bang_oracle_rho_crit(void) { return kRhoCrit; }

// Observables at arbitrary sky points (arcsec), before PSF and binning: out[4][n].
int bang_oracle_points(const bang_oracle_opts* o, const double* theta, const double* xs, const double* ys, int n,
                       double kpa, double* out) {
  const int np = bang_oracle_nparams(o->n_discs);
  if (!in_domain(theta, np, o->halo_kind, o->bulge_kind)) return 1;
  const RadialRule q(o->n_quad);
  const Model<double> m = decode(theta, o->n_discs, o->halo_kind, o->bulge_kind);
  for (int p = 0; p < n; ++p) {
    double v[4];
    eval_point(m, xs[p], ys[p], kpa, q, v);
    for (int c = 0; c < 4; ++c) out[(size_t)c * n + p] = v[c];
  }
  return 0;
}

// Padded fine field field[4][H][W], H = os*ny + 2h, W = os*nx + 2h.
int bang_oracle_fine_field(const bang_oracle_galaxy* d, const bang_oracle_opts* o, const double* theta,
                           double* field, int nthreads) {
  set_threads(nthreads);
  const Galaxy g = make_galaxy(d);
  const int np = bang_oracle_nparams(o->n_discs);
  if (!in_domain(theta, np, o->halo_kind, o->bulge_kind)) return 1;
  const RadialRule q(o->n_quad);
  std::vector<double> f;
  fine_field(g, decode(theta, o->n_discs, o->halo_kind, o->bulge_kind), q, f);
  std::memcpy(field, f.data(), f.size() * sizeof(double));
  return 0;
}

// PSF + binning of a caller-given padded field[4][H][W] -> maps[4][ny][nx] (no offsets).
int bang_oracle_convolve_bin(const bang_oracle_galaxy* d, const double* field, double* maps, int nthreads) {
  set_threads(nthreads);
  const Galaxy g = make_galaxy(d);
  std::vector<double> f(field, field + (size_t)4 * g.W() * g.H()), out;
  convolve_bin(g, psf_weights(g), f, out);
  std::memcpy(maps, out.data(), out.size() * sizeof(double));
  return 0;
}

// Model observable maps maps[4][ny][nx]: B, v_los + v_sys, sigma_los, M/L.
int bang_oracle_maps(const bang_oracle_galaxy* d, const bang_oracle_opts* o, const double* theta, double* maps,
                     int nthreads) {
  set_threads(nthreads);
  const Galaxy g = make_galaxy(d);
  const int np = bang_oracle_nparams(o->n_discs);
  if (!in_domain(theta, np, o->halo_kind, o->bulge_kind)) return 1;
  const RadialRule q(o->n_quad);
  std::vector<double> out;
  model_maps(g, decode(theta, o->n_discs, o->halo_kind, o->bulge_kind), q, out);
  std::memcpy(maps, out.data(), out.size() * sizeof(double));
  return 0;
}

double bang_oracle_norm_const(const bang_oracle_galaxy* d) { return norm_const(make_galaxy(d)); }

// logL[b] = -chi2/2 - sum ln(sqrt(2 pi) delta); chi2[b] also returned when non-null.
// Rows outside the parameter domain give logL = -inf and chi2 = +inf.
int bang_oracle_loglike(const bang_oracle_galaxy* d, const bang_oracle_opts* o, const double* theta, int B,
                        double* logL, double* chi2, int nthreads) {
  set_threads(nthreads);
  const Galaxy g = make_galaxy(d);
  const int np = bang_oracle_nparams(o->n_discs);
  const RadialRule q(o->n_quad);
  const double cst = norm_const(g);
  for (int b = 0; b < B; ++b) {
    const double* th = theta + (size_t)b * np;
    if (!in_domain(th, np, o->halo_kind, o->bulge_kind)) {
      logL[b] = -INFINITY;
      if (chi2) chi2[b] = INFINITY;
      continue;
    }
    std::vector<double> maps;
    model_maps(g, decode(th, o->n_discs, o->halo_kind, o->bulge_kind), q, maps);
    const double c2 = chi2_of(g, maps);
    logL[b] = -0.5 * c2 - cst;
    if (chi2) chi2[b] = c2;
  }
  return 0;
}

// logL and its gradient grad[b][p] = d logL / d theta_p, by forward-mode duals through the
// same arithmetic.  Out-of-domain rows give logL = -inf and a zero gradient.
int bang_oracle_loglike_grad(const bang_oracle_galaxy* d, const bang_oracle_opts* o, const double* theta, int B,
                             double* logL, double* grad, int nthreads) {
  set_threads(nthreads);
  const Galaxy g = make_galaxy(d);
  const int np = bang_oracle_nparams(o->n_discs);
  const RadialRule q(o->n_quad);
  const double cst = norm_const(g);
  for (int b = 0; b < B; ++b) {
    const double* th = theta + (size_t)b * np;
    if (!in_domain(th, np, o->halo_kind, o->bulge_kind)) {
      logL[b] = -INFINITY;
      for (int p = 0; p < np; ++p) grad[(size_t)b * np + p] = 0.0;
      continue;
    }
    Dual td[PMAX];
    for (int p = 0; p < np; ++p) { td[p] = Dual(th[p]); td[p].d[p] = 1.0; }
    std::vector<Dual> maps;
    model_maps(g, decode(td, o->n_discs, o->halo_kind, o->bulge_kind), q, maps);
    const Dual c2 = chi2_of(g, maps);
    logL[b] = -0.5 * c2.v - cst;
    for (int p = 0; p < np; ++p) grad[(size_t)b * np + p] = -0.5 * c2.d[p];
  }
  return 0;
}

}  // extern "C"
