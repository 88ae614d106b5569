// Device-side model arithmetic for the GB300 likelihood kernels (sm_103a).
//
// Per sky point: reference frame (Sec. 2.1), Dehnen-family bulge projected density and
// isotropic dispersion by a fixed radial quadrature (Sec. 2.2, Eqs. 4 and 6 definitions),
// circular velocities of bulge (Eq. 2 generalised), NFW halo and exponential discs (Eq. 9,
// Binney & Tremaine form), Satoh decomposition (Eqs. 10-12) and the light-weighted
// observables (Eqs. 13-15, 19).  Arithmetic is float32, per-model constants decoded once
// per row.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "bulge_fit.h"
#include "disc_fit.h"

namespace bang {

constexpr int kMaxQuad = 128;
constexpr int kMaxParams = 19;
constexpr double kPi = 3.14159265358979323846;
constexpr double kG = 4.30091727e-6;                                  // kpc (km/s)^2 / Msun
constexpr double kRhoCrit = 3.0 * 0.07 * 0.07 / (8.0 * kPi * kG);     // H0 = 70 km/s/Mpc
constexpr float kR2Floor = 1e-12f;                                    // radii floored at 1e-6 kpc

// Radial rule r = R cosh t, t in [0, 16], Gauss-Legendre nodes (filled at model creation).
// For node k: cm1 = cosh t_k - 1, lc = log2 cosh t_k, ws = w_k cosh t_k, wq = w_k tanh^2 t_k.
// Rows [0, 64) hold the 64-node rule, rows [64, 192) the 128-node rule.  Every translation
// unit has its own copy; each exports an upload function that fills it.
static __constant__ float kNodeCm1[192];
static __constant__ float kNodeLc[192];
static __constant__ float kNodeWs[192];
static __constant__ float kNodeWq[192];

template <int NQ> struct NodeBase { static constexpr int value = NQ == 64 ? 0 : 64; };

// For the series coefficients (rows as above): log2 m_k and log2(cosh t_k / m_k), with m_k
// the float32 cosh t_k - 1 of kNodeCm1 (computed in float64 on the host, then rounded).
static __constant__ float kNodeLm[192];
static __constant__ float kNodeLcm[192];

// Splits of the radial rule for the upper-node series (see fill_tail_coeffs), two levels:
// nodes k >= KF of points with w (cosh t_KF - 1) >= kFarZ are summed by a kFarTerms-term
// series (t_KF ~ 3: the far level, most of the grid); otherwise nodes k >= K of points with
// w (cosh t_K - 1) >= kTailZ by a kTailTerms-term series (t_K ~ 5: the mid level); the
// points nearest the bulge centre take every node one by one.
template <int NQ> struct TailRule;
template <> struct TailRule<64> { static constexpr int K = 24, KF = 18; };
template <> struct TailRule<128> { static constexpr int K = 48, KF = 36; };
constexpr int kTailTerms = 8;     // mid level: j = 0 .. 7
constexpr float kTailZ = 16.0f;   // mid level serves points with w (cosh t_K - 1) >= 16
constexpr int kFarTerms = 14;     // far level: j = 0 .. 13
constexpr float kFarZ = 7.0f;     // far level serves points with w (cosh t_KF - 1) >= 7
// shared coefficient pairs of one set: the far level's kFarTerms, then the mid level's
// kTailTerms padded with zeros to kFarTerms (one Horner length serves both)
constexpr int kTailSet = 2 * kFarTerms;

// One galaxy on the device.
struct GalDev {
  int nx, ny, os, h;
  int L;                 // os + 2h: taps of the combined PSF (x) box filter per axis
  int W, H;              // padded fine grid: os*nx + 2h by os*ny + 2h
  int psf_kind;          // taps: 0 separable (Gaussian, square window), 1 two-dimensional
  int flux;              // 1: flux-weighted moments are convolved (psf_mode bit 4)
  int bulge_kind;        // 0 Dehnen gamma (radial rule); 1 Hernquist, 2 Jaffe (closed-form fits)
  float pitch_kpa;       // fine pitch in kpc
  double xoff_kpa;       // x (kpc) of padded fine column 0 is xoff_kpa + 0 * pitch_kpa
  double yoff_kpa;
  const float* taps;     // [L] (separable) or [L][L]
  const float* data;     // [4][ny][nx]
  const float* iv;       // [4][ny][nx]: mask / delta^2
  double norm_const;     // sum over used spaxels of ln(sqrt(2 pi) delta)
};

// One block-sized unit of work: spaxel rows [j0, j1) of row b against galaxy g.
struct WorkItem {
  int b, g, j0, j1;
};

// Per-model constants (float32), decoded once per row and held in shared memory.
struct ModelConst {
  float X0, Y0;            // kpc offset of fine column/row 0 relative to the model centre
  float cpa, spa;          // cos, sin of the position angle
  float inv_ci, si;        // 1 / cos i, sin i
  // bulge (Dehnen): a, gamma
  float inv_a, ngam, g4, g3, three_mg;
  float cS, cQ, vb_c;      // Sigma = cS x pS S; Sigma sigma^2 = cQ pQ Q; vb^2 = vb_c u^(3-g) / (r/a)
  float vb_r;              // G M_b: vb^2 = vb_r u^(3-g) / r (the forward's form, with 1/r at hand)
  float Lb;                // 1e-6 / (M/L)_b
  // halo (NFW)
  float inv_rs, vh_c;      // x = r / rs; NFW vh^2 = vh_c m(x) / r; Hernquist vh^2 = vh_c x / (1 + x)^2
  int hern;                // halo kind: 0 NFW, 1 Hernquist
  // discs
  float inv_Rd[2], half_inv_Rd[2], vd_c[2], Sd_c[2], Ld[2], ks[2], omk[2];
  float two_Rd[2];         // 2 R_d: 1 / y = 2 R_d / r for the disc's velocity fit
  float vsys;
  int flux;                // the galaxy's flux-weighted PSF mode (GalDev::flux)
  int bulge_fit;           // GalDev::bulge_kind: 0 radial rule, 1 / 2 closed-form fits
  int valid;
};

// floor(n / d) for 0 <= n < 2^21 from inv_d = 1.0f / d (d >= 1): n + 1/2 is never a
// multiple of d and (n + 1/2) / d lies at least 1 / (2d) from an integer, more than the
// float32 rounding of the reciprocal and the product can move it; one multiply and one
// conversion instead of the integer division sequence (the stencils' index ranges).
__device__ __forceinline__ int floor_div(int n, float inv_d) { return __float2int_rz(((float)n + 0.5f) * inv_d); }

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float lg2_approx(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
// SFU reciprocal and square root (about 1 ulp, flush-to-zero).  The forward model's
// per-point reciprocals, divisions, square roots, exp and log use these single MUFU
// operations instead of the correctly rounded sequences: the node loop leaves the SFU room
// while instruction issue is the limit, and the change moves logL by < 2e-7 relative.
__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rsqrt_approx(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float sqrt_approx(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Decode row theta (float32) into per-model constants.  Returns 0 when the row is outside
// the parameter domain (non-finite, i not in [0, pi/2), gamma not in [0, 3), |k| > 1,
// M/L <= 0, and for the NFW halo c <= 0).  halo_kind 0: NFW (slot 13 = c); 1: Hernquist
// (slot 13 = log10 R_h, the paper's halo).
// bulge_kind 1 and 2 fix gamma at 1 and 2: the gamma slot is then not used.
__device__ inline bool theta_in_domain(const float* __restrict__ th, int nd, int halo_kind, int bulge_kind) {
  const int np = nd == 2 ? 19 : 15;
  for (int i = 0; i < np; ++i)
    if (!isfinite((double)th[i])) return false;
  const double inc = th[3], gam = th[6];
  if (!(inc >= 0.0 && inc < 0.5 * kPi)) return false;
  if (bulge_kind == 0 && !(gam >= 0.0 && gam < 3.0)) return false;
  if (!(fabs((double)th[9]) <= 1.0)) return false;
  if (!(th[10] > 0.f && th[11] > 0.f)) return false;
  if (halo_kind == 0 && !(th[13] > 0.f)) return false;
  if (nd == 2 && !(fabs((double)th[17]) <= 1.0 && th[18] > 0.f)) return false;
  return true;
}

// The transcendental parts of the decode, independent of one another, so that a warp can
// take one per lane (decode_kernel) or one thread all of them in turn (decode_model):
//   0 cos i, 1 sin i, 2 cos PA, 3 sin PA, 4 M_b, 5 a, 6 M_200 (or M_h),
//   7 r_200 = (3 M_200 / (4 pi 200 rho_c))^(1/3) (or R_h), 8 m(c) = ln(1 + c) - c / (1 + c)
//   (NFW only), 9 M_d1, 10 R_d1, 11 M_d2, 12 R_d2.
// r_200 is 10^((log10 M_200 + l10k) / 3) with l10k = log10(3 / (4 pi 200 rho_c)).
// The decode runs in float32 (CUDA's sinf, cosf, exp10f and log1pf, within 2 ulp): the
// constants are float32 in the model anyway, a float64 operation issues at 1/64 of the
// float32 rate here, and the float64 form (each constant rounded once) made the decode of
// one row a 16 us chain of dependent float64 operations (7 us in float32) at no gain in
// logL against the float64 oracle.
constexpr int kDecodeTerms = 13;

__device__ inline double decode_l10k() { return log10(3.0 / (4.0 * kPi * 200.0 * kRhoCrit)); }

__device__ inline float decode_term(int i, const float* __restrict__ th, int nd, int halo_kind, double l10k) {
  int kind = 1;   // 0 sin, 1 10^x, 2 ln(1 + x) - x / (1 + x), 3 unused, 4 cos
  float x = 0.f;
  switch (i) {
    case 0: kind = 4; x = th[3]; break;
    case 1: kind = 0; x = th[3]; break;
    case 2: kind = 4; x = th[2]; break;
    case 3: kind = 0; x = th[2]; break;
    case 4: x = th[4]; break;
    case 5: x = th[5]; break;
    case 6: x = th[12]; break;
    case 7: x = halo_kind == 0 ? (float)(((double)th[12] + l10k) / 3.0) : th[13]; break;
    case 8: kind = halo_kind == 0 ? 2 : 3; x = th[13]; break;
    case 9: x = th[7]; break;
    case 10: x = th[8]; break;
    case 11: kind = nd == 2 ? 1 : 3; x = th[15]; break;
    case 12: kind = nd == 2 ? 1 : 3; x = th[16]; break;
    default: kind = 3;
  }
  if (kind == 0) return sinf(x);
  if (kind == 4) return cosf(x);
  if (kind == 1) return exp10f(x);
  if (kind == 2) return log1pf(x) - x / (1.0f + x);
  return 0.f;
}

// The per-model constants from theta and its decode terms T[kDecodeTerms] (float32; the
// centre offsets X0, Y0 are one float64 subtraction, rounded once).
__device__ inline void decode_finish(const float* __restrict__ th, const float* T, int nd, int halo_kind,
                                     const GalDev& g, ModelConst& m) {
  const float two_pi = (float)(2.0 * kPi), G = (float)kG;
  const float ci = T[0], si = T[1];
  m.X0 = (float)(g.xoff_kpa - (double)th[0]);
  m.Y0 = (float)(g.yoff_kpa - (double)th[1]);
  m.cpa = T[2];
  m.spa = T[3];
  m.inv_ci = 1.0f / ci;
  m.si = si;
  // bulge
  const float Mb = T[4], a = T[5], gam = g.bulge_kind == 0 ? th[6] : (float)g.bulge_kind;
  const float ia = 1.0f / a;
  m.inv_a = ia;
  m.ngam = -gam;
  m.g4 = gam - 4.0f;
  m.g3 = 3.0f - 2.0f * gam;
  m.three_mg = 3.0f - gam;
  m.cS = (3.0f - gam) * Mb * (ia * ia) / two_pi;
  m.cQ = G * (3.0f - gam) * (Mb * Mb) * (ia * ia * ia) / two_pi;
  m.vb_c = G * Mb * ia;
  m.vb_r = G * Mb;
  m.bulge_fit = g.bulge_kind;
  if (g.bulge_kind != 0) {   // closed-form fits: Sigma = (M / a^2) F_S, Sigma sigma^2 = (G M^2 / a^3) F_Q
    m.cS = Mb * (ia * ia);
    m.cQ = G * (Mb * Mb) * (ia * ia * ia);
  }
  m.Lb = 1e-6f / th[10];
  // halo
  m.hern = halo_kind;
  if (halo_kind == 0) {   // NFW: vh^2 = vh_c m(r/rs) / r
    const float M200 = T[6], c = th[13], r200 = T[7], mc = T[8];
    m.inv_rs = c / r200;
    m.vh_c = G * M200 / mc;
  } else {                // Hernquist (Eq. 2 with M_h, R_h): vh^2 = vh_c x / (1 + x)^2, x = r / R_h
    const float Mh = T[6], Rh = T[7];
    m.inv_rs = 1.0f / Rh;
    m.vh_c = G * Mh / Rh;
  }
  // discs
  for (int j = 0; j < 2; ++j) {
    if (j >= nd) {
      m.inv_Rd[j] = m.half_inv_Rd[j] = m.vd_c[j] = m.Sd_c[j] = m.Ld[j] = m.ks[j] = m.omk[j] = m.two_Rd[j] = 0.f;
      continue;
    }
    const int o = j == 0 ? 7 : 15;
    const float Md = T[9 + 2 * j], Rd = T[10 + 2 * j], k = th[o + 2];
    const float ml = j == 0 ? th[11] : th[18];
    const float iR = 1.0f / Rd;
    m.inv_Rd[j] = iR;
    m.half_inv_Rd[j] = 0.5f * iR;
    m.two_Rd[j] = 2.0f * Rd;
    m.vd_c[j] = 2.0f * G * Md * iR;
    m.Sd_c[j] = Md * (iR * iR) / (two_pi * ci);
    m.Ld[j] = 1e-6f / ml;
    m.ks[j] = -k * si;
    m.omk[j] = (1.0f - k * k) / 3.0f;
  }
  m.vsys = th[14];
  m.flux = g.flux;
}

// theta -> per-model constants by one warp (all 32 lanes call it): lane i < kDecodeTerms
// evaluates decode term i (the terms are independent, so a row costs the latency of one
// transcendental, not thirteen in a chain), lane 0 gathers them and writes m.  A row outside
// the parameter domain, or with ok_gal false, gets m.valid = 0 and no other field.
__device__ inline void decode_row_warp(const float* __restrict__ th, int nd, int halo_kind, const GalDev& g,
                                       bool ok_gal, double l10k, int lane, ModelConst& m) {
  const bool ok = ok_gal && theta_in_domain(th, nd, halo_kind, g.bulge_kind);
  const float v = (ok && lane < kDecodeTerms) ? decode_term(lane, th, nd, halo_kind, l10k) : 0.f;
  float T[kDecodeTerms];
#pragma unroll
  for (int i = 0; i < kDecodeTerms; ++i) T[i] = __shfl_sync(0xffffffffu, v, i);
  if (lane != 0) return;
  m.valid = 0;
  if (ok) {
    decode_finish(th, T, nd, halo_kind, g, m);
    m.valid = 1;
  }
}

// theta -> per-model constants by one thread; 0 for a row outside the domain.
__device__ inline int decode_model(const float* __restrict__ th, int nd, int halo_kind, const GalDev& g,
                                   ModelConst& m) {
  if (!theta_in_domain(th, nd, halo_kind, g.bulge_kind)) return 0;
  float T[kDecodeTerms];
  const double l10k = decode_l10k();
  for (int i = 0; i < kDecodeTerms; ++i) T[i] = decode_term(i, th, nd, halo_kind, l10k);
  decode_finish(th, T, nd, halo_kind, g, m);
  return 1;
}

// F(y) = y^2 [I0 K0 - I1 K1](y) from the generated float32 fits (see disc_fit.h).
// u = 1 / y, used for y > 1 (the caller may have it from a reciprocal it already holds).
__device__ __forceinline__ float disc_F(float y, float u) {
  if (y <= 1.0f) {
    const float s = y * y;
    float P = kDiscP[BANG_DISC_DEG_A], Q = kDiscQ[BANG_DISC_DEG_A];
#pragma unroll
    for (int k = BANG_DISC_DEG_A - 1; k >= 0; --k) {
      P = fmaf(P, s, kDiscP[k]);
      Q = fmaf(Q, s, kDiscQ[k]);
    }
    return s * (P - lg2_approx(y) * 0.693147181f * Q);
  }
  const int e = (int)((__float_as_uint(u) >> 23) & 0xff) - 127;   // u in [2^e, 2^(e+1))
  int k = -e - 1;
  k = k < 0 ? 0 : (k > BANG_DISC_NPIECE_B - 1 ? BANG_DISC_NPIECE_B - 1 : k);
  const float t = (u - kDiscMid[k]) * kDiscInvHalf[k];
  float gv = kDiscG[k][BANG_DISC_DEG_B];
#pragma unroll
  for (int i = BANG_DISC_DEG_B - 1; i >= 0; --i) gv = fmaf(gv, t, kDiscG[k][i]);
  return gv * (0.25f * u);
}

__device__ __forceinline__ float disc_F(float y) { return disc_F(y, y > 1.0f ? rcp_approx(y) : 0.f); }

// F(y) and dF/dy from the same fits (Horner carries the derivative along).
//   y <= 1: F = s (P - ln y Q)  ->  F' = 2y [P + s P' - ln y (Q + s Q') - Q/2]
//   y >  1: F = g(t) u / 4      ->  F' = -(u^2 / 4) [g + u g'(t) invhalf]
// u = 1 / y, used for y > 1 (as in disc_F).
__device__ __forceinline__ void disc_F_d(float y, float u, float& F, float& dF) {
  if (y <= 1.0f) {
    const float s = y * y;
    float P = kDiscP[BANG_DISC_DEG_A], Q = kDiscQ[BANG_DISC_DEG_A], dP = 0.f, dQ = 0.f;
#pragma unroll
    for (int k = BANG_DISC_DEG_A - 1; k >= 0; --k) {
      dP = fmaf(dP, s, P);
      dQ = fmaf(dQ, s, Q);
      P = fmaf(P, s, kDiscP[k]);
      Q = fmaf(Q, s, kDiscQ[k]);
    }
    const float ly = lg2_approx(y) * 0.693147181f;
    F = s * (P - ly * Q);
    dF = 2.0f * y * (P + s * dP - ly * (Q + s * dQ) - 0.5f * Q);
    return;
  }
  const int e = (int)((__float_as_uint(u) >> 23) & 0xff) - 127;
  int k = -e - 1;
  k = k < 0 ? 0 : (k > BANG_DISC_NPIECE_B - 1 ? BANG_DISC_NPIECE_B - 1 : k);
  const float ih = kDiscInvHalf[k];
  const float t = (u - kDiscMid[k]) * ih;
  float gv = kDiscG[k][BANG_DISC_DEG_B], dg = 0.f;
#pragma unroll
  for (int i = BANG_DISC_DEG_B - 1; i >= 0; --i) {
    dg = fmaf(dg, t, gv);
    gv = fmaf(gv, t, kDiscG[k][i]);
  }
  F = gv * (0.25f * u);
  dF = -0.25f * u * u * fmaf(u * ih, dg, gv);
}

// m(x) = ln(1 + x) - x / (1 + x) of the NFW enclosed mass.  For x <= 1, with z = x / (2 + x):
// m = 2 z^2 / (1 + z) + 2 z^3 (1/3 + z^2/5 + z^4/7 + ...), free of the cancellation at small x;
// z and 2 z^2 / (1 + z) = x^2 / ((1 + x)(2 + x)) share one reciprocal.
__device__ __forceinline__ float nfw_m(float x) {
  if (x <= 1.0f) {
    const float x1 = 1.0f + x, rr = rcp_approx(x1 * (2.0f + x));   // 1 / ((1 + x)(2 + x))
    const float z = x * x1 * rr;                                     // x / (2 + x)
    const float z2 = z * z;
    float s = 1.0f / 19.0f;
    s = fmaf(s, z2, 1.0f / 17.0f);
    s = fmaf(s, z2, 1.0f / 15.0f);
    s = fmaf(s, z2, 1.0f / 13.0f);
    s = fmaf(s, z2, 1.0f / 11.0f);
    s = fmaf(s, z2, 1.0f / 9.0f);
    s = fmaf(s, z2, 1.0f / 7.0f);
    s = fmaf(s, z2, 1.0f / 5.0f);
    s = fmaf(s, z2, 1.0f / 3.0f);
    return x * x * rr + 2.0f * z2 * z * s;   // 2 z^2 / (1 + z) = x^2 / ((1 + x)(2 + x))
  }
  return lg2_approx(1.0f + x) * 0.693147181f - __fdividef(x, 1.0f + x);
}

// Circular velocity squared of the halo at in-plane radius r.
__device__ __forceinline__ float halo_v2(const ModelConst& m, float r, float inv_r) {
  const float x = r * m.inv_rs;
  if (m.hern) {
    const float ix = rcp_approx(1.0f + x);
    return m.vh_c * x * ix * ix;
  }
  return m.vh_c * nfw_m(x) * inv_r;
}

// Projected density and Sigma sigma^2 of the bulge at sky radius R (kpc).
// With x = R / a, w = x / (x + 1) and node k at r = R cosh t_k:
//   rho(r) r^-1-part:  (x c)^-g (x c + 1)^(g-4) = x^-g (x+1)^(g-4) * c^-g q^(g-4),  q = 1 + w (c - 1)
//   rho M part:        (x c)^(3-2g) (x c + 1)^(2g-7) = x^(3-2g) (x+1)^(2g-7) * c^(3-2g) q^(2g-7)
// and q^(2g-7) = (q^(g-4))^2 q, so each node costs one lg2 and one ex2 of small arguments
// plus multiplications; the large per-point powers are taken once, accurately, outside the
// sum.  The products are grouped as (W E)(E c^3 q) so that no intermediate leaves the float
// range while its term still matters.
template <int NQ>
__device__ __forceinline__ void bulge_projected(const ModelConst& m, float R, float& Sigma, float& SigS2) {
  constexpr int base = NodeBase<NQ>::value;
  const float x = R * m.inv_a;
  const float xp1 = x + 1.0f;
  const float ix1 = rcp_approx(xp1);
  const float w = x * ix1;
  const float lw = lg2_approx(w);
  const float i2 = ix1 * ix1;
  const float ip4 = i2 * i2;
  const float pS = ex2_approx(m.ngam * lw) * ip4;
  const float pQ = ex2_approx(m.g3 * lw) * ip4;
  float S = 0.f, Q = 0.f;
#pragma unroll
  for (int k = 0; k < NQ; ++k) {
    const float cm1 = kNodeCm1[base + k];
    const float q = fmaf(w, cm1, 1.0f);
    const float d = lg2_approx(q);
    const float E = ex2_approx(fmaf(m.g4, d, m.ngam * kNodeLc[base + k]));   // c^-g q^(g-4)
    const float c = cm1 + 1.0f;
    S = fmaf(kNodeWs[base + k], E, S);
    Q = fmaf(kNodeWq[base + k] * E, E * (c * c) * (c * q), Q);
  }
  Sigma = m.cS * x * pS * S;
  SigS2 = m.cQ * pQ * Q;
}

// Projected density and Sigma sigma^2 of the closed-form bulges (bulge_kind 1 Hernquist,
// 2 Jaffe; Eqs. 4-6, B4-B5) from the fits of bulge_fit.h: Sigma = (M / a^2) F_S(s),
// Sigma sigma^2 = (G M^2 / a^3) F_Q(s), s = R / a, log2 F = E_k + p_k(u) on unit pieces of
// t = log2 s.  With sS, sQ also the slopes d ln F / d ln s (the adjoint's).
__device__ __forceinline__ void bulge_closed(const ModelConst& m, float R, float& Sigma, float& SigS2,
                                             float* sS = nullptr, float* sQ = nullptr) {
  const int kind = m.bulge_fit - 1;
  const float t = lg2_approx(R * m.inv_a) - (float)BANG_BULGE_FIT_T0;
  int k = (int)floorf(t);
  k = k < 0 ? 0 : (k > BANG_BULGE_FIT_N - 1 ? BANG_BULGE_FIT_N - 1 : k);
  // beyond the fitted range (s outside [2^-48, 2^32)) the edge values hold, with zero slope
  const bool inside = t >= 0.f && t < (float)BANG_BULGE_FIT_N;
  const float u = fminf(fmaxf(t - (float)k, 0.f), 1.f);
  const float* cS = kBulgeFitC[kind][0][k];
  const float* cQ = kBulgeFitC[kind][1][k];
  float pS = cS[BANG_BULGE_FIT_DEG], pQ = cQ[BANG_BULGE_FIT_DEG], dS = 0.f, dQ = 0.f;
#pragma unroll
  for (int i = BANG_BULGE_FIT_DEG - 1; i >= 0; --i) {
    if (sS) {
      dS = fmaf(dS, u, pS);
      dQ = fmaf(dQ, u, pQ);
    }
    pS = fmaf(pS, u, cS[i]);
    pQ = fmaf(pQ, u, cQ[i]);
  }
  Sigma = m.cS * kBulgeFitScale[kind][0][k] * ex2_approx(pS);
  SigS2 = m.cQ * kBulgeFitScale[kind][1][k] * ex2_approx(pQ);
  if (sS) {
    *sS = inside ? dS : 0.f;
    *sQ = inside ? dQ : 0.f;
  }
}

// ---------------------------------------------------------------- radial table (option)
// Per parameter vector, the projected density Sigma and Q = Sigma sigma^2 of the bulge are
// computed by the same radial quadrature at T radii uniformly spaced in t = log2(R / a),
// node k at t0 + k h, covering the 1e-6 kpc floor to the farthest fine point.  A fine point
// then interpolates with the 4-point Lagrange rule in t.  To keep float32 precision the
// table holds the values V_k and the log-ratios D_k = log2(V_{k+1} / V_k) (|D_k| < 1): the
// interpolant is V_i 2^d with d = -w0 D_{i-1} + (w2 + w3) D_i + w3 D_{i+1}, all small.
// For the adjoint the table also holds the logarithmic slopes s = R dln/dR and
// g = dln/dgamma of both quantities (O(1) values, interpolated directly).
// Layout of one row's table (floats): [t0, 1/h, -, -][V_S][D_S][V_Q][D_Q][s_S][s_Q][g_S][g_Q].
constexpr int kTabHdr = 4;
enum { TAB_VS = 0, TAB_DS, TAB_VQ, TAB_DQ, TAB_SS, TAB_SQ, TAB_GS, TAB_GQ };

struct TabPos {
  int i;
  float w0, w2, w3, wv[4];
};

__device__ __forceinline__ TabPos table_pos(const float* __restrict__ tab, int T, float x) {
  const float t = log2f(x);
  const float u = (t - tab[0]) * tab[1];
  int i = (int)floorf(u);
  i = i < 1 ? 1 : (i > T - 3 ? T - 3 : i);
  const float f = u - (float)i;
  TabPos p;
  p.i = i;
  const float fm1 = f - 1.0f, fm2 = f - 2.0f, fp1 = f + 1.0f;
  p.w0 = -f * fm1 * fm2 * (1.0f / 6.0f);
  p.w2 = -fp1 * f * fm2 * 0.5f;
  p.w3 = fp1 * f * fm1 * (1.0f / 6.0f);
  p.wv[0] = p.w0;
  p.wv[1] = fp1 * fm1 * fm2 * 0.5f;
  p.wv[2] = p.w2;
  p.wv[3] = p.w3;
  return p;
}

// value of table q (V_S or V_Q with its log-ratios in the next table) at position p
__device__ __forceinline__ float table_value(const float* __restrict__ tab, int T, int q, const TabPos& p) {
  const float* V = tab + kTabHdr + q * T;
  const float* D = V + T;
  const float d = fmaf(-p.w0, D[p.i - 1], fmaf(p.w2 + p.w3, D[p.i], p.w3 * D[p.i + 1]));
  return V[p.i] * ex2_approx(d);
}

// plain 4-point interpolation of an O(1) table (slopes)
__device__ __forceinline__ float table_plain(const float* __restrict__ tab, int T, int q, const TabPos& p) {
  const float* Y = tab + kTabHdr + q * T + p.i - 1;
  return fmaf(p.wv[0], Y[0], fmaf(p.wv[1], Y[1], fmaf(p.wv[2], Y[2], p.wv[3] * Y[3])));
}

// The same sums with the per-model node factors folded into weights staged in shared
// memory, two nodes at a time: nw[k/2] = (ws_k, ws_k+1, wq_k, wq_k+1) with
// ws_k = w_k cosh t_k c_k^-g and wq_k = w_k tanh^2 t_k c_k^(3-2g).  e = q^(g-4) gives both
// q^(g-4) and q^(2g-7) = e^2 q, so a node needs one lg2 and one ex2; the FP32 work of a
// pair of nodes (q, the exponent, the two sums) runs as packed two-lane FMA / MUL
// instructions (one issue slot for both nodes, each lane rounded like fmaf), and one
// 128-bit shared load brings the pair's four weights.  Even and odd nodes accumulate in
// the two lanes, added at the end.
// Nodes [K0, K1) of the paired-weight sums (K0, K1 even).
template <int NQ, int K0, int K1>
__device__ __forceinline__ void node_pairs(const ModelConst& m, const float4* __restrict__ nw, float w, float2& S,
                                           float2& Q) {
  constexpr int base = NodeBase<NQ>::value;
  const float2 w2 = make_float2(w, w), g2 = make_float2(m.g4, m.g4), one2 = make_float2(1.0f, 1.0f);
#pragma unroll
  for (int k = K0; k < K1; k += 2) {
    const float2 q = __ffma2_rn(w2, make_float2(kNodeCm1[base + k], kNodeCm1[base + k + 1]), one2);
    const float2 d = make_float2(lg2_approx(q.x), lg2_approx(q.y));
    float4 wk;   // kept in the loop: hoisting 2 NQ invariant weights would exhaust the registers
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(wk.x), "=f"(wk.y), "=f"(wk.z), "=f"(wk.w)
                 : "r"((unsigned)__cvta_generic_to_shared(nw + k / 2)));
    const float2 t = __fmul2_rn(g2, d);
    const float2 e = make_float2(ex2_approx(t.x), ex2_approx(t.y));
    S = __ffma2_rn(make_float2(wk.x, wk.y), e, S);
    Q = __ffma2_rn(__fmul2_rn(make_float2(wk.z, wk.w), e), __fmul2_rn(e, q), Q);
  }
}

// With `tail` (kTailSet coefficient pairs: fill_tail_coeffs for both levels), the upper
// nodes of points away from the bulge centre come from a series: k >= KF where
// w (cosh t_KF - 1) >= kFarZ, else k >= K where w (cosh t_K - 1) >= kTailZ; without it, or
// for points nearer the centre, every node is summed.
template <int NQ>
__device__ __forceinline__ void bulge_projected_w(const ModelConst& m, const float4* __restrict__ nw, float R,
                                                  float& Sigma, float& SigS2, const float2* __restrict__ tail = nullptr) {
  constexpr int base = NodeBase<NQ>::value, K = TailRule<NQ>::K, KF = TailRule<NQ>::KF;
  const float x = R * m.inv_a;
  const float xp1 = x + 1.0f;
  const float ix1 = rcp_approx(xp1);
  const float w = x * ix1;
  const float lw = lg2_approx(w);
  const float i2 = ix1 * ix1;
  const float ip4 = i2 * i2;
  const float pS = ex2_approx(m.ngam * lw) * ip4;
  const float pQ = ex2_approx(m.g3 * lw) * ip4;
  float2 S = make_float2(0.f, 0.f), Q = make_float2(0.f, 0.f);
  const bool far = tail && w * kNodeCm1[base + KF] >= kFarZ;
  const bool mid = !far && tail && w * kNodeCm1[base + K] >= kTailZ;
  node_pairs<NQ, 0, KF>(m, nw, w, S, Q);
  if (!far) node_pairs<NQ, KF, K>(m, nw, w, S, Q);
  if (!far && !mid) node_pairs<NQ, K, NQ>(m, nw, w, S, Q);
  if (far || mid) {
    // upper nodes: w^n P(1 / w) for both sums, P by Horner in packed pairs (the mid set's
    // top coefficients are zero)
    const float2* c = far ? tail : tail + kFarTerms;
    const float u = xp1 * rcp_approx(x);   // 1 / w
    const float2 u2 = make_float2(u, u);
    float2 P;
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(P.x), "=f"(P.y)
                 : "r"((unsigned)__cvta_generic_to_shared(c + kFarTerms - 1)));
#pragma unroll
    for (int j = kFarTerms - 2; j >= 0; --j) {
      float2 cj;
      asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(cj.x), "=f"(cj.y)
                   : "r"((unsigned)__cvta_generic_to_shared(c + j)));
      P = __ffma2_rn(P, u2, cj);
    }
    S.x = fmaf(ex2_approx(m.g4 * lw), P.x, S.x);                    // w^(g-4)
    Q.x = fmaf(ex2_approx(fmaf(2.0f, m.g4, 1.0f) * lw), P.y, Q.x);  // w^(2g-7)
  }
  Sigma = m.cS * x * pS * (S.x + S.y);
  SigS2 = m.cQ * pQ * (Q.x + Q.y);
}

// ---------------------------------------------------------------- upper nodes as a series
// For the upper nodes k >= K of the radial rule (cosh t_k - 1 = m_k large), a point's
// q_k = 1 + w m_k = w m_k (1 + z_k) with z_k = 1 / (w m_k) small, so that
//   q_k^n = (w m_k)^n sum_j binom(n, j) z_k^j     (binomial series, |z_k| < 1)
// and the upper part of each projected sum collapses into a polynomial in 1 / w:
//   sum_{k>=K} W_k q_k^n = w^n sum_j binom(n, j) A_j w^-j,   A_j = sum_{k>=K} W_k m_k^(n-j),
// with n = g - 4, W_k = ws_k c_k^-g for Sigma and n = 2g - 7, W_k = wq_k c_k^(3-2g) for
// Sigma sigma^2 (the same terms as the per-node sums).  A_j depends on the model only.  It is
// the same discrete sum up to the series' truncation, which stays below 1e-9 of the whole
// sum for every gamma in [0, 3) at both levels (a float64 check over the parameter range is
// a CPU test): the far level splits at t_KF ~ 3 and takes fourteen terms where
// w m_KF >= kFarZ = 7 (R above ~2.2 bulge scales, most of a grid); the mid level splits at
// t_K ~ 5.1 and takes eight terms where w m_K >= kTailZ = 16 (R above ~0.2 bulge scales);
// a point closer to the bulge centre takes the upper nodes one by one.

// The series' per-model coefficients (binom(n, j) A_j for Sigma, for Sigma sigma^2) of the
// split at node K, T terms, as pairs, by the 32 lanes of one warp: lane l takes the upper
// nodes K + l, K + l + 32, ..., and the lanes' partial sums are combined by a fixed shuffle
// tree (the same bits on every call).  Float32 suffices: the upper nodes' share of either
// sum is small (their terms fall like cosh^-3 t: < 2.4e-4 above the mid split, < 1.5e-3
// above the far one), so the coefficients' float32 rounding and the float32 Horner move a
// sum by < 1e-9 (a CPU test emulates both).
template <int NQ, int K, int T>
__device__ __noinline__ void fill_tail_level(const ModelConst& m, float2* tail, int lane) {
  constexpr int base = NodeBase<NQ>::value;
  const float nS = m.g4, nQ = fmaf(2.0f, m.g4, 1.0f);   // g - 4 and 2g - 7
  float aS[T], aQ[T];
#pragma unroll
  for (int j = 0; j < T; ++j) aS[j] = aQ[j] = 0.f;
  for (int k = K + lane; k < NQ; k += 32) {
    const float lm = kNodeLm[base + k], lc = kNodeLc[base + k];
    const float r = 1.0f / kNodeCm1[base + k];
    float eS = kNodeWs[base + k] * exp2f(fmaf(m.ngam, lc, nS * lm));   // W_k m_k^n for Sigma
    float eQ = kNodeWq[base + k] * exp2f(fmaf(m.g3, lc, nQ * lm));     // and for Sigma sigma^2
#pragma unroll
    for (int j = 0; j < T; ++j) {
      aS[j] += eS;
      aQ[j] += eQ;
      eS *= r;
      eQ *= r;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int j = 0; j < T; ++j) {
      aS[j] += __shfl_xor_sync(0xffffffffu, aS[j], o);
      aQ[j] += __shfl_xor_sync(0xffffffffu, aQ[j], o);
    }
  }
  if (lane < T) {   // lane j: binom(n, j) by the product formula
    float bS = 1.0f, bQ = 1.0f, vS = aS[0], vQ = aQ[0];
#pragma unroll
    for (int j = 1; j < T; ++j) {
      bS *= (nS - (j - 1)) / j;
      bQ *= (nQ - (j - 1)) / j;
      if (j == lane) {
        vS = bS * aS[j];
        vQ = bQ * aQ[j];
      }
    }
    tail[lane] = make_float2(vS, vQ);
  }
}

// Both levels' coefficients into tail[kTailSet] (one warp): the far set, then the mid set
// padded with zeros to kFarTerms.
template <int NQ>
__device__ __forceinline__ void fill_tail_coeffs(const ModelConst& m, float2* tail, int lane) {
  fill_tail_level<NQ, TailRule<NQ>::KF, kFarTerms>(m, tail, lane);
  fill_tail_level<NQ, TailRule<NQ>::K, kTailTerms>(m, tail + kFarTerms, lane);
  if (lane >= kTailTerms && lane < kFarTerms) tail[kFarTerms + lane] = make_float2(0.f, 0.f);
}

// The adjoint's series (three packed coefficient sets of kTailTerms pairs, Sigma in .x and
// Sigma sigma^2 in .y).  Besides each sum sum W q^n, the adjoint carries the sums weighted by
// u / w = c / q and by log2(u / w) = log2 c - log2 q (see bang_adjoint.cu).  With
// A_j = sum_{k>=K} W_k m_k^(n-j), A'_j = sum_{k>=K} W_k log2(c_k / m_k) m_k^(n-j) and
// log2 q = log2 w + log2 m + log2(1 + z):
//   sum W q^n c / q          = w^(n-1) sum_j binom(n-1, j) (A_j + A_{j+1}) w^-j   (c = m + 1)
//   sum W q^n log2(c / q) + log2 w sum W q^n
//                            = w^n sum_j [binom(n, j) A'_j - f_j(n) A_j] w^-j,
// f_j(n) = (d/dn binom(n, j)) / ln 2 = binom(n, j) sum_{i<j} 1 / (n - i) / ln 2, the
// coefficients of (1 + z)^n log2(1 + z).  For the split at node K with T terms, set c of
// stride ST (T <= ST, the entries from T on zero): tail[0..ST) hold binom(n, j) A_j (the
// sums), tail[ST..2ST) binom(n-1, j) (A_j + A_{j+1}), tail[2ST..3ST) the log-weighted ones.
template <int NQ, int K, int T, int ST>
__device__ __noinline__ void fill_tail_level_adj(const ModelConst& m, float2* tail, int lane) {
  constexpr int base = NodeBase<NQ>::value;
  constexpr float kInvLn2 = 1.44269504088896341f;
  for (int fam = 0; fam < 2; ++fam) {   // 0: Sigma (n = g - 4), 1: Sigma sigma^2 (n = 2g - 7)
    const float n = fam == 0 ? m.g4 : fmaf(2.0f, m.g4, 1.0f);
    const float pc = fam == 0 ? m.ngam : m.g3;   // power of c in W
    float A[T + 1], Ap[T];
#pragma unroll
    for (int j = 0; j <= T; ++j) A[j] = 0.f;
#pragma unroll
    for (int j = 0; j < T; ++j) Ap[j] = 0.f;
    for (int k = K + lane; k < NQ; k += 32) {
      const float lcm = kNodeLcm[base + k], r = 1.0f / kNodeCm1[base + k];
      const float W = fam == 0 ? kNodeWs[base + k] : kNodeWq[base + k];
      float e = W * exp2f(fmaf(pc, kNodeLc[base + k], n * kNodeLm[base + k]));   // W_k m_k^n
#pragma unroll
      for (int j = 0; j <= T; ++j) {
        A[j] += e;
        if (j < T) Ap[j] = fmaf(e, lcm, Ap[j]);
        e *= r;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
      for (int j = 0; j <= T; ++j) A[j] += __shfl_xor_sync(0xffffffffu, A[j], o);
#pragma unroll
      for (int j = 0; j < T; ++j) Ap[j] += __shfl_xor_sync(0xffffffffu, Ap[j], o);
    }
    if (lane < T) {   // lane j: the three coefficient sets of pair j
      float b = 1.0f, b1 = 1.0f, hs = 0.f;   // binom(n, j), binom(n - 1, j), sum_{i<j} 1 / (n - i)
      float v0 = A[0], v1 = A[0] + A[1], v2 = Ap[0];
#pragma unroll
      for (int j = 1; j < T; ++j) {
        b *= (n - (j - 1)) / j;
        b1 *= (n - 1.0f - (j - 1)) / j;
        hs += 1.0f / (n - (j - 1));
        if (j == lane) {
          v0 = b * A[j];
          v1 = b1 * (A[j] + A[j + 1]);
          v2 = b * (Ap[j] - hs * kInvLn2 * A[j]);
        }
      }
      reinterpret_cast<float*>(tail + lane)[fam] = v0;
      reinterpret_cast<float*>(tail + ST + lane)[fam] = v1;
      reinterpret_cast<float*>(tail + 2 * ST + lane)[fam] = v2;
    } else if (lane < ST) {
      reinterpret_cast<float*>(tail + lane)[fam] = 0.f;
      reinterpret_cast<float*>(tail + ST + lane)[fam] = 0.f;
      reinterpret_cast<float*>(tail + 2 * ST + lane)[fam] = 0.f;
    }
  }
}

// The adjoint's coefficients into tail[kTailSetAdj] (one warp): the mid level only, three
// sets of kTailTerms pairs.  (With the far level as well, the adjoint's three longer Horner
// chains and extra node-loop segment raised its spills at 64 and 80 registers, and logL +
// gradient ran 5.5% slower: 88.2k against 93.3k evaluations per second.)
constexpr int kTailSetAdj = 3 * kTailTerms;
template <int NQ>
__device__ __forceinline__ void fill_tail_coeffs_adj(const ModelConst& m, float2* tail, int lane) {
  fill_tail_level_adj<NQ, TailRule<NQ>::K, kTailTerms, kTailTerms>(m, tail, lane);
}

// Per-model node weights for bulge_projected_w, paired as (ws_k, ws_k+1, wq_k, wq_k+1)
// (threads of a block fill them together).
template <int NQ>
__device__ __forceinline__ void fill_node_pairs(const ModelConst& m, float4* nw, int tid, int nthreads) {
  constexpr int base = NodeBase<NQ>::value;
  for (int j = tid; j < NQ / 2; j += nthreads) {
    const int k = base + 2 * j;
    nw[j] = make_float4(kNodeWs[k] * exp2f(m.ngam * kNodeLc[k]), kNodeWs[k + 1] * exp2f(m.ngam * kNodeLc[k + 1]),
                        kNodeWq[k] * exp2f(m.g3 * kNodeLc[k]), kNodeWq[k + 1] * exp2f(m.g3 * kNodeLc[k + 1]));
  }
}

// The four observables at one padded fine grid point: (B, v_los, sigma_los, <L/M>); in the
// flux-weighted PSF mode the quantities that are convolved instead: (B, B v_los,
// B (sigma_los^2 + v_los^2), 1e-6 Sigma_tot), so that after the PSF v = C1 / C0,
// sigma^2 = C2 / C0 - v^2 and M/L = C3 / C0.
template <int NQ, int ND>
__device__ __forceinline__ float4 eval_point(const ModelConst& m, float X, float Y, const float* tab = nullptr,
                                             int T = 0, const float4* nodew = nullptr,
                                             const float2* tail = nullptr) {
  // Sec. 2.1: rotate the major axis onto x; deproject the razor-thin discs by 1 / cos i
  const float xr = fmaf(X, m.cpa, Y * m.spa);
  const float yr = fmaf(Y, m.cpa, -X * m.spa);
  const float R2 = fmaf(X, X, Y * Y);
  const float yd = yr * m.inv_ci;
  const float r2 = fmaf(xr, xr, yd * yd);
  const float R = sqrt_approx(fmaxf(R2, kR2Floor));
  const float r2c = fmaxf(r2, kR2Floor);
  const float inv_r = rsqrt_approx(r2c);   // r and 1 / r from one SFU operation
  const float r = r2c * inv_r;
  const float cphi = xr * inv_r;

  float Sb, SbS2;
  if (tab) {
    const TabPos tp = table_pos(tab, T, R * m.inv_a);
    Sb = table_value(tab, T, TAB_VS, tp);
    SbS2 = table_value(tab, T, TAB_VQ, tp);
  } else if (m.bulge_fit) {
    bulge_closed(m, R, Sb, SbS2);
  } else if (nodew) {
    bulge_projected_w<NQ>(m, nodew, R, Sb, SbS2, tail);
  } else {
    bulge_projected<NQ>(m, R, Sb, SbS2);
  }

  // circular velocities in the disc plane (Eq. 10)
  const float xa = r * m.inv_a;
  const float ub = xa * rcp_approx(xa + 1.0f);
  float vint2 = m.vb_r * ex2_approx(m.three_mg * lg2_approx(ub)) * inv_r;   // vb_c u^(3-g) / (r / a)
  vint2 += halo_v2(m, r, inv_r);
  float Sd[ND];
#pragma unroll
  for (int j = 0; j < ND; ++j) {
    vint2 += m.vd_c[j] * disc_F(r * m.half_inv_Rd[j], m.two_Rd[j] * inv_r);
    Sd[j] = m.Sd_c[j] * ex2_approx(-r * m.inv_Rd[j] * 1.44269504f);
  }
  const float vint = sqrt_approx(vint2);

  // light weighting (Eqs. 13-15, 19)
  const float Bb = Sb * m.Lb;
  float B = Bb, Bv = 0.f, Bs2 = SbS2 * m.Lb, Stot = Sb;
#pragma unroll
  for (int j = 0; j < ND; ++j) {
    const float Bd = Sd[j] * m.Ld[j];
    B += Bd;
    Bv = fmaf(Bd, m.ks[j] * cphi * vint, Bv);
    Bs2 = fmaf(Bd, m.omk[j] * vint2, Bs2);
    Stot += Sd[j];
  }
  const float iB = rcp_approx(B);
  if (m.flux) return make_float4(B, Bv, fmaf(Bv * iB, Bv, Bs2), 1e-6f * Stot);
  return make_float4(B, Bv * iB, sqrt_approx(Bs2 * iB), __fdividef(B * 1e6f, Stot));
}

}  // namespace bang
