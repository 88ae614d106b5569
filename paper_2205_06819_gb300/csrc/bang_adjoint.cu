// Hand-written adjoint of the log-likelihood: d logL / d theta.
//
// Input: the per-spaxel seeds lambda_c(s) = d logL / d F_c(s) written by the forward kernel
// (kModeSeed), F_c the PSF-convolved, binned channel c (B, v, sigma, <L/M>).  Because
// F_c(s) = sum_p K(s, p) f_c(p) is linear in the fine-grid field f, the seed of fine point p
// is a_c(p) = sum_s K(s, p) lambda_c(s): the transposed PSF (x) box stencil.  For the
// separable Gaussian this is a vertical pass (spaxel rows -> fine row) followed by a
// horizontal one; for the Moffat PSF the two-dimensional weights are applied directly.
// Each fine point then runs the vector-Jacobian product of the point model
// (Sec. 2.1-2.4): the forward values are recomputed, the radial quadrature included, and
// the seeds are pushed back through the light weighting, the Satoh decomposition, the
// circular velocities and the geometry onto the per-model constants.  The quadrature
// carries, besides its two sums, the sums weighted by u = r / (r + a) and by ln u, from
// which d/dR, d/da and d/dgamma of both projected integrals follow in closed form:
//   Sigma = 2 R sum w c rho(R c),   rho ~ r^-g (r + a)^(g-4):
//     R dSigma/dR = (1 - g) Sigma + (g - 4) Su,   a dSigma/da = (g - 3) Sigma + (4 - g) Su,
//     dSigma/dg = -Sigma / (3 - g) - Sl,
//   Sigma sigma^2 = 2 G sum w tanh^2 rho M,   rho M ~ r^(3-2g) (r + a)^(2g-7):
//     R dQ/dR = (3 - 2g) Q + (2g - 7) Qu,   a dQ/da = (2g - 6) Q + (7 - 2g) Qu,
//     dQ/dg = -Q / (3 - g) - 2 Ql,
// with Su, Qu the u-weighted and Sl, Ql the (ln u)-weighted sums.  Nothing is stored
// between the forward and the backward evaluation: the quadrature is recomputed.
// Work items are bands of fine rows (no halo is needed: the seeds live in global memory).
// Per-thread float32 partials are reduced per block (sums of four lanes in float32, the
// rest in float64) into the work item's own slots; grad_out_kernel sums a row's items in
// item order (no atomics) and maps the per-model constants to theta in float64.
#include <cuda_runtime.h>

#include <cmath>

#include "bang_device.cuh"
#include "bang_internal.h"

namespace bang {
namespace {

constexpr int kAdjThreads = 256;
constexpr float kLn2 = 0.69314718055994531f;

// Next work item: from the shared counter when the launch has one (dynamic scheduling),
// otherwise the fixed grid stride.  Always a block-wide barrier, so that thread 0 may
// overwrite the shared item state afterwards.
#define BANG_NEXT_ITEM(it)                                                     \
  do {                                                                         \
    if (a.queue) {                                                             \
      if (threadIdx.x == 0) next_item = atomicAdd(a.queue, 1) + (int)gridDim.x; \
      __syncthreads();                                                         \
      it = next_item;                                                          \
    } else {                                                                   \
      __syncthreads();                                                         \
      it += (int)gridDim.x;                                                    \
    }                                                                          \
  } while (0)

// adjoint accumulators (per thread), adjoints of the per-model constants
enum {
  A_X0 = 0,   // d/dX0 (X0 = xoff - x0)
  A_Y0,
  A_PA,       // d/dPA through the rotation
  A_INVCI,    // d/d(1/cos i)
  A_LB,       // d/dLb,  Lb = 1e-6 / (M/L)_b
  A_A,        // d/da   (bulge scale)
  A_G,        // d/dgamma
  A_MB,       // Mb d/dMb
  A_VHC,      // d/dvh_c
  A_IRS,      // d/d(1/rs)
  A_D0        // per disc: SDC, VDC, IRD, HIRD, LD, KS, OMK
};
constexpr int kPerDisc = 7;
enum { D_SDC = 0, D_VDC, D_IRD, D_HIRD, D_LD, D_KS, D_OMK };

// One level of a warp reduce-scatter: a lane holds the partial sums of 2h slots and keeps
// the half its lane bit o selects (upper if set), adding the partner lane's copy of it.
template <int H, typename T>
__device__ __forceinline__ void scatter_level(const T* v, T* out, int lane, int o) {
  const bool up = (lane & o) != 0;
#pragma unroll
  for (int j = 0; j < H; ++j) {
    const T keep = up ? v[j + H] : v[j], send = up ? v[j] : v[j + H];
    out[j] = keep + __shfl_xor_sync(0xffffffffu, send, o);
  }
}

// Warp sum of each of N <= 32 per-lane float32 accumulators, as a reduce-scatter: lane k
// returns the sum over the warp's 32 lanes of acc[k] (lanes k >= N return 0).  The first
// two levels (sums of 2 and 4 lanes) add in float32, the last three in float64, in a fixed
// order.  A float64 add issues at 1/64 the float32 rate here, and a full-width float64
// shuffle sum of every accumulator (5 adds each) took a fifth of the FP64 pipe's time;
// this form needs 8 conversions and 7 float64 adds per lane whatever N is.
template <int N>
__device__ __forceinline__ double warp_sum_scatter(const float* acc, int lane) {
  static_assert(N > 16 && N <= 32, "the reduce-scatter expects 17 to 32 accumulators");
  float v32[32], v16[16], v8[8];
#pragma unroll
  for (int j = 0; j < 32; ++j) v32[j] = j < N ? acc[j] : 0.f;
  scatter_level<16>(v32, v16, lane, 16);
  scatter_level<8>(v16, v8, lane, 8);
  double d8[8], d4[4], d2[2], d1[1];
#pragma unroll
  for (int j = 0; j < 8; ++j) d8[j] = (double)v8[j];
  scatter_level<4>(d8, d4, lane, 4);
  scatter_level<2>(d4, d2, lane, 2);
  scatter_level<1>(d2, d1, lane, 1);
  return lane < N ? d1[0] : 0.0;
}

struct BulgeDer {
  float Sb, Qb, dSb_dR, dQb_dR, dSb_da, dQb_da, dSb_dg, dQb_dg;
};

// Nodes [K0, K1) of the six sums (paired weights, packed two-lane instructions): even and
// odd nodes accumulate in the two lanes.
template <int NQ, int K0, int K1>
__device__ __forceinline__ void adj_node_pairs(const ModelConst& m, const float4* __restrict__ nw, float w,
                                               float2& S2, float2& Su2, float2& Sl2, float2& Q2, float2& Qu2,
                                               float2& Ql2) {
  constexpr int base = NodeBase<NQ>::value;
  const float2 w2 = make_float2(w, w), g2 = make_float2(m.g4, m.g4), one2 = make_float2(1.0f, 1.0f);
  const float2 neg2 = make_float2(-1.0f, -1.0f);
#pragma unroll
  for (int k = K0; k < K1; k += 2) {
    const float2 q = __ffma2_rn(w2, make_float2(kNodeCm1[base + k], kNodeCm1[base + k + 1]), one2);
    const float2 d = make_float2(lg2_approx(q.x), lg2_approx(q.y));
    float4 wk;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(wk.x), "=f"(wk.y), "=f"(wk.z), "=f"(wk.w)
                 : "r"((unsigned)__cvta_generic_to_shared(nw + k / 2)));
    const float2 t = __fmul2_rn(g2, d);
    const float2 e = make_float2(ex2_approx(t.x), ex2_approx(t.y));   // q^(g-4); q^(2g-7) = e^2 q
    const float2 t1 = __fmul2_rn(make_float2(wk.x, wk.y), e);
    const float2 t2 = __fmul2_rn(__fmul2_rn(make_float2(wk.z, wk.w), e), __fmul2_rn(e, q));
    const float2 mk = __ffma2_rn(d, neg2, make_float2(kNodeLc[base + k], kNodeLc[base + k + 1]));   // log2(u / w)
    const float2 uw = make_float2(ex2_approx(mk.x), ex2_approx(mk.y));                             // u / w
    S2 = __fadd2_rn(S2, t1);
    Su2 = __ffma2_rn(t1, uw, Su2);
    Sl2 = __ffma2_rn(t1, mk, Sl2);
    Q2 = __fadd2_rn(Q2, t2);
    Qu2 = __ffma2_rn(t2, uw, Qu2);
    Ql2 = __ffma2_rn(t2, mk, Ql2);
  }
}

// Horner of one packed coefficient set (kTailTerms pairs in shared memory) at u.
__device__ __forceinline__ float2 tail_poly(const float2* __restrict__ c, float2 u2) {
  float2 P;
  asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(P.x), "=f"(P.y)
               : "r"((unsigned)__cvta_generic_to_shared(c + kTailTerms - 1)));
#pragma unroll
  for (int j = kTailTerms - 2; j >= 0; --j) {
    float2 cj;
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(cj.x), "=f"(cj.y)
                 : "r"((unsigned)__cvta_generic_to_shared(c + j)));
    P = __ffma2_rn(P, u2, cj);
  }
  return P;
}

template <int NQ>
__device__ __forceinline__ BulgeDer bulge_projected_vjp(const ModelConst& m, float R, const float4* nw = nullptr,
                                                         const float2* tail = nullptr) {
  constexpr int base = NodeBase<NQ>::value, K = TailRule<NQ>::K;
  const float x = R * m.inv_a;
  const float xp1 = x + 1.0f;
  const float ix1 = rcp_approx(xp1);
  const float w = x * ix1;
  const float lw = lg2_approx(w);
  const float i2 = ix1 * ix1;
  const float ip4 = i2 * i2;
  const float pS = ex2_approx(m.ngam * lw) * ip4;
  const float pQ = ex2_approx(m.g3 * lw) * ip4;
  // u_k = r_k / (r_k + a) = w 2^(lc_k - d_k): the per-point factors w and log2 w are taken
  // out of the sums, which carry t u / w and t (log2 u - log2 w)
  float S = 0.f, Su = 0.f, Sl = 0.f, Q = 0.f, Qu = 0.f, Ql = 0.f;
  bool series = false;
  if (nw) {
    // per-model node factors folded into shared-memory weights, two nodes at a time in
    // packed two-lane FP32 instructions (see bulge_projected_w); with the series
    // coefficients, the upper nodes k >= K of points away from the centre come from the
    // mid-level series (the forward's far level is not used here: fill_tail_coeffs_adj)
    float2 S2 = make_float2(0.f, 0.f), Su2 = S2, Sl2 = S2, Q2 = S2, Qu2 = S2, Ql2 = S2;
    series = tail && w * kNodeCm1[base + K] >= kTailZ;
    if (series) adj_node_pairs<NQ, 0, K>(m, nw, w, S2, Su2, Sl2, Q2, Qu2, Ql2);
    else adj_node_pairs<NQ, 0, NQ>(m, nw, w, S2, Su2, Sl2, Q2, Qu2, Ql2);
    S = S2.x + S2.y;
    Su = Su2.x + Su2.y;
    Sl = Sl2.x + Sl2.y;
    Q = Q2.x + Q2.y;
    Qu = Qu2.x + Qu2.y;
    Ql = Ql2.x + Ql2.y;
  } else {
#pragma unroll
    for (int k = 0; k < NQ; ++k) {
      const float lc = kNodeLc[base + k];
      const float q = fmaf(w, kNodeCm1[base + k], 1.0f);
      const float d = lg2_approx(q);
      const float E = ex2_approx(fmaf(m.g4, d, m.ngam * lc));   // c^-g q^(g-4)
      const float c = kNodeCm1[base + k] + 1.0f;
      const float t1 = kNodeWs[base + k] * E;
      const float t2 = (kNodeWq[base + k] * E) * (E * (c * c) * (c * q));
      const float mk = lc - d;                         // log2(u_k / w)
      const float uw = ex2_approx(mk);                 // u_k / w
      S += t1;
      Su = fmaf(t1, uw, Su);
      Sl = fmaf(t1, mk, Sl);
      Q += t2;
      Qu = fmaf(t2, uw, Qu);
      Ql = fmaf(t2, mk, Ql);
    }
  }
  Su *= w;
  Qu *= w;
  Sl = fmaf(lw, S, Sl);
  Ql = fmaf(lw, Q, Ql);
  if (series) {   // the upper nodes: w^n times the three polynomials in 1 / w (fill_tail_coeffs_adj)
    const float2 u2 = make_float2(xp1 * rcp_approx(x), xp1 * rcp_approx(x));
    const float2 P0 = tail_poly(tail, u2), P1 = tail_poly(tail + kTailTerms, u2),
                 P2 = tail_poly(tail + 2 * kTailTerms, u2);
    const float pwS = ex2_approx(m.g4 * lw), pwQ = ex2_approx(fmaf(2.0f, m.g4, 1.0f) * lw);   // w^(g-4), w^(2g-7)
    S = fmaf(pwS, P0.x, S);
    Q = fmaf(pwQ, P0.y, Q);
    Su = fmaf(pwS, P1.x, Su);
    Qu = fmaf(pwQ, P1.y, Qu);
    Sl = fmaf(pwS, P2.x, Sl);
    Ql = fmaf(pwQ, P2.y, Ql);
  }
  const float fS = m.cS * x * pS, fQ = m.cQ * pQ;
  const float g = -m.ngam;
  const float inv3g = rcp_approx(m.three_mg);
  BulgeDer o;
  o.Sb = fS * S;
  o.Qb = fQ * Q;
  const float SU = fS * Su, SL = fS * Sl * kLn2, QU = fQ * Qu, QL = fQ * Ql * kLn2;
  const float iR = rcp_approx(R);
  o.dSb_dR = ((1.0f - g) * o.Sb + (g - 4.0f) * SU) * iR;
  o.dSb_da = ((g - 3.0f) * o.Sb + (4.0f - g) * SU) * m.inv_a;
  o.dSb_dg = -o.Sb * inv3g - SL;
  o.dQb_dR = ((3.0f - 2.0f * g) * o.Qb + (2.0f * g - 7.0f) * QU) * iR;
  o.dQb_da = ((2.0f * g - 6.0f) * o.Qb + (7.0f - 2.0f * g) * QU) * m.inv_a;
  o.dQb_dg = -o.Qb * inv3g - 2.0f * QL;
  return o;
}

// The same derivatives from the row's radial table: Sigma = M a^-2 F(R/a, g) and
// Q = M^2 a^-3 G(R/a, g) give a dSigma/da = -(2 + s_S) Sigma and a dQ/da = -(3 + s_Q) Q,
// with s = R dln/dR the tabulated slopes; d/dgamma from the tabulated g = dln/dgamma.
__device__ __forceinline__ BulgeDer bulge_table_vjp(const ModelConst& m, const float* __restrict__ tab, int T,
                                                     float R) {
  const TabPos p = table_pos(tab, T, R * m.inv_a);
  BulgeDer o;
  o.Sb = table_value(tab, T, TAB_VS, p);
  o.Qb = table_value(tab, T, TAB_VQ, p);
  const float sS = table_plain(tab, T, TAB_SS, p), sQ = table_plain(tab, T, TAB_SQ, p);
  const float gS = table_plain(tab, T, TAB_GS, p), gQ = table_plain(tab, T, TAB_GQ, p);
  const float iR = rcp_approx(R);
  o.dSb_dR = o.Sb * sS * iR;
  o.dQb_dR = o.Qb * sQ * iR;
  o.dSb_da = -o.Sb * (2.0f + sS) * m.inv_a;
  o.dQb_da = -o.Qb * (3.0f + sQ) * m.inv_a;
  o.dSb_dg = o.Sb * gS;
  o.dQb_dg = o.Qb * gQ;
  return o;
}

// The same derivatives for the closed-form bulges: Sigma = M a^-2 F_S(R/a) and
// Q = G M^2 a^-3 F_Q(R/a) with the fitted slopes s = d ln F / d ln(R/a); gamma is fixed.
__device__ __forceinline__ BulgeDer bulge_closed_vjp(const ModelConst& m, float R) {
  BulgeDer o;
  float sS, sQ;
  bulge_closed(m, R, o.Sb, o.Qb, &sS, &sQ);
  const float iR = rcp_approx(R);
  o.dSb_dR = o.Sb * sS * iR;
  o.dQb_dR = o.Qb * sQ * iR;
  o.dSb_da = -o.Sb * (2.0f + sS) * m.inv_a;
  o.dQb_da = -o.Qb * (3.0f + sQ) * m.inv_a;
  o.dSb_dg = 0.f;
  o.dQb_dg = 0.f;
  return o;
}

// Vector-Jacobian product of one fine point: adds sum_c a_c d f_c / d(constants) to acc.
template <int NQ, int ND>
__device__ __forceinline__ void point_vjp(const ModelConst& m, float X, float Y, float4 a, float* acc,
                                          const float* tab, int T, const float4* nodew, const float2* tail) {
  // ---- forward (Sec. 2.1-2.4), keeping what the reverse sweep needs
  const float xr = fmaf(X, m.cpa, Y * m.spa);
  const float yr = fmaf(Y, m.cpa, -X * m.spa);
  const float R2 = fmaf(X, X, Y * Y);
  const float yd = yr * m.inv_ci;
  const float r2 = fmaf(xr, xr, yd * yd);
  const bool Rfree = R2 > kR2Floor, rfree = r2 > kR2Floor;
  const float R = sqrt_approx(fmaxf(R2, kR2Floor));
  const float r2c = fmaxf(r2, kR2Floor);
  const float inv_r = rsqrt_approx(r2c);   // r and 1 / r from one SFU operation
  const float r = r2c * inv_r;
  const float cphi = xr * inv_r;

  const BulgeDer bd = tab ? bulge_table_vjp(m, tab, T, R)
                           : (m.bulge_fit ? bulge_closed_vjp(m, R) : bulge_projected_vjp<NQ>(m, R, nodew, tail));

  const float xa = r * m.inv_a;
  const float ub = xa * rcp_approx(xa + 1.0f);
  const float lub = lg2_approx(ub);
  const float vb2 = m.vb_r * ex2_approx(m.three_mg * lub) * inv_r;   // vb_c u^(3-g) / (r / a)
  const float xh = r * m.inv_rs;
  const float ixh1 = rcp_approx(1.0f + xh);
  // NFW: vh2 = vh_c m(x) / r; Hernquist: vh2 = vh_c h(x), h = x / (1 + x)^2
  const float mh = m.hern ? xh * ixh1 * ixh1 : nfw_m(xh);
  const float vh2 = m.hern ? m.vh_c * mh : m.vh_c * mh * inv_r;
  float vint2 = vb2 + vh2;
  float Fd[ND], dFd[ND], ex[ND], Sd[ND];
#pragma unroll
  for (int j = 0; j < ND; ++j) {
    disc_F_d(r * m.half_inv_Rd[j], m.two_Rd[j] * inv_r, Fd[j], dFd[j]);
    vint2 = fmaf(m.vd_c[j], Fd[j], vint2);
    ex[j] = ex2_approx(-r * m.inv_Rd[j] * 1.44269504f);
    Sd[j] = m.Sd_c[j] * ex[j];
  }
  const float vint = sqrt_approx(vint2);
  float B = bd.Sb * m.Lb, Bv = 0.f, Bs2 = bd.Qb * m.Lb, Stot = bd.Sb;
#pragma unroll
  for (int j = 0; j < ND; ++j) {
    const float Bd = Sd[j] * m.Ld[j];
    B += Bd;
    Bv = fmaf(Bd, m.ks[j] * cphi * vint, Bv);
    Bs2 = fmaf(Bd, m.omk[j] * vint2, Bs2);
    Stot += Sd[j];
  }
  const float iB = rcp_approx(B);
  const float f1 = Bv * iB;
  const float f2 = sqrt_approx(Bs2 * iB);
  const float iS = rcp_approx(Stot);
  const float f3 = B * 1e6f * iS;

  // ---- reverse
  float gB, gBv, gBs2, gStot;
  if (m.flux) {   // point values (B, Bv, Bs2 + Bv^2 / B, 1e-6 Stot)
    gB = a.x - a.z * f1 * f1;
    gBv = fmaf(2.0f * a.z, f1, a.y);
    gBs2 = a.z;
    gStot = 1e-6f * a.w;
  } else {        // point values (B, Bv / B, sqrt(Bs2 / B), 1e6 B / Stot)
    gB = a.x - a.y * f1 * iB - 0.5f * a.z * f2 * iB + a.w * f3 * iB;
    gBv = a.y * iB;
    gBs2 = f2 > 0.f ? __fdividef(0.5f * a.z, f2 * B) : 0.f;
    gStot = -a.w * f3 * iS;
  }
  const float gSb = fmaf(gB, m.Lb, gStot);
  const float gQb = gBs2 * m.Lb;
  acc[A_LB] += fmaf(gB, bd.Sb, gBs2 * bd.Qb);
  float gcphi = 0.f, gvint = 0.f, gvint2 = 0.f, gr = 0.f;
#pragma unroll
  for (int j = 0; j < ND; ++j) {
    float* dj = acc + A_D0 + kPerDisc * j;
    const float Bd = Sd[j] * m.Ld[j];
    const float gBd = gB + gBv * m.ks[j] * cphi * vint + gBs2 * m.omk[j] * vint2;
    const float gSd = fmaf(gBd, m.Ld[j], gStot);
    dj[D_LD] += gBd * Sd[j];
    dj[D_KS] += gBv * Bd * cphi * vint;
    dj[D_OMK] += gBs2 * Bd * vint2;
    gcphi = fmaf(gBv * Bd, m.ks[j] * vint, gcphi);
    gvint = fmaf(gBv * Bd, m.ks[j] * cphi, gvint);
    gvint2 = fmaf(gBs2 * Bd, m.omk[j], gvint2);
    dj[D_SDC] += gSd * ex[j];
    gr -= gSd * Sd[j] * m.inv_Rd[j];
    dj[D_IRD] -= gSd * Sd[j] * r;
  }
  gvint2 += __fdividef(0.5f * gvint, vint);
#pragma unroll
  for (int j = 0; j < ND; ++j) {
    float* dj = acc + A_D0 + kPerDisc * j;
    dj[D_VDC] += gvint2 * Fd[j];
    const float gy = gvint2 * m.vd_c[j] * dFd[j];
    gr = fmaf(gy, m.half_inv_Rd[j], gr);
    dj[D_HIRD] += gy * r;
  }
  if (m.hern) {
    // Hernquist halo: vh2 = vh_c h(x), x = r / R_h, h'(x) = (1 - x) / (1 + x)^3
    acc[A_VHC] += gvint2 * mh;
    const float gxh = gvint2 * m.vh_c * (1.0f - xh) * ixh1 * ixh1 * ixh1;
    gr += gxh * m.inv_rs;
    acc[A_IRS] += gxh * r;
  } else {
    // NFW halo: vh2 = vh_c m(x) / r, x = r / rs, m'(x) = x / (1 + x)^2
    acc[A_VHC] += gvint2 * mh * inv_r;
    const float gxh = gvint2 * m.vh_c * (xh * ixh1 * ixh1) * inv_r;
    gr += gxh * m.inv_rs - gvint2 * vh2 * inv_r;
    acc[A_IRS] += gxh * r;
  }
  // bulge circular velocity: vb2 = G Mb u^(3-g) / r, u = r / (r + a)
  const float omu = 1.0f - ub;
  gr += gvint2 * vb2 * inv_r * (m.three_mg * omu - 1.0f);
  acc[A_A] -= gvint2 * vb2 * m.three_mg * omu * m.inv_a;
  acc[A_G] -= gvint2 * vb2 * lub * kLn2;
  acc[A_MB] += gvint2 * vb2;
  // bulge projected density and dispersion
  acc[A_A] += gSb * bd.dSb_da + gQb * bd.dQb_da;
  acc[A_G] += gSb * bd.dSb_dg + gQb * bd.dQb_dg;
  acc[A_MB] += gSb * bd.Sb + 2.0f * gQb * bd.Qb;
  const float gR = gSb * bd.dSb_dR + gQb * bd.dQb_dR;
  // geometry
  float gxr = gcphi * inv_r;
  gr -= gcphi * cphi * inv_r;
  float gyd = 0.f;
  if (rfree) {
    gxr = fmaf(gr * inv_r, xr, gxr);
    gyd = gr * inv_r * yd;
  }
  const float gyr = gyd * m.inv_ci;
  acc[A_INVCI] += gyd * yr;
  float gX = gxr * m.cpa - gyr * m.spa;
  float gY = gxr * m.spa + gyr * m.cpa;
  if (Rfree) {
    const float iR = rcp_approx(R);
    gX = fmaf(gR * iR, X, gX);
    gY = fmaf(gR * iR, Y, gY);
  }
  acc[A_X0] += gX;
  acc[A_Y0] += gY;
  acc[A_PA] += gxr * yr - gyr * xr;
}

// d logL / d theta from the reduced constant adjoints and the row's decode terms T
// (float64, one thread).
__device__ void constants_to_theta(const float* __restrict__ th, const float* T, int nd, int halo_kind,
                                   int bulge_kind, const double* s, double* g) {
  const double ln10 = 2.302585092994045684;
  const double ci = T[0], si = T[1];
  const double a = T[5];
  g[0] = -s[A_X0];
  g[1] = -s[A_Y0];
  g[2] = s[A_PA];
  double gi = s[A_INVCI] * si / (ci * ci);
  g[4] = ln10 * s[A_MB];
  g[5] = ln10 * a * s[A_A];
  g[6] = bulge_kind == 0 ? s[A_G] : 0.0;   // a fixed gamma has no slot to differentiate
  g[10] = -s[A_LB] * (1e-6 / th[10]) / th[10];
  if (halo_kind == 0) {   // NFW: vh_c = G M200 / m(c), 1/rs = c / r200(M200)
    const double M200 = T[6], c = th[13], r200 = T[7], mc = T[8];
    const double dmc = c / ((1.0 + c) * (1.0 + c));
    const double vh_c = kG * M200 / mc, inv_rs = c / r200;
    g[12] = ln10 * (s[A_VHC] * vh_c - s[A_IRS] * inv_rs / 3.0);
    g[13] = -s[A_VHC] * vh_c * dmc / mc + s[A_IRS] * inv_rs / c;
  } else {                // Hernquist: vh_c = G M_h / R_h, 1/rs = 1 / R_h
    const double Mh = T[6], Rh = T[7];
    const double vh_c = kG * Mh / Rh, inv_rs = 1.0 / Rh;
    g[12] = ln10 * s[A_VHC] * vh_c;
    g[13] = -ln10 * (s[A_VHC] * vh_c + s[A_IRS] * inv_rs);
  }
  for (int j = 0; j < nd; ++j) {
    const double* dj = s + A_D0 + kPerDisc * j;
    const int o = j == 0 ? 7 : 15;
    const double Md = T[9 + 2 * j], Rd = T[10 + 2 * j], k = th[o + 2];
    const double ml = j == 0 ? th[11] : th[18];
    const double Sd_c = Md / (2.0 * kPi * Rd * Rd * ci), vd_c = 2.0 * kG * Md / Rd;
    g[o] = ln10 * (dj[D_SDC] * Sd_c + dj[D_VDC] * vd_c);
    g[o + 1] = ln10 * (-2.0 * dj[D_SDC] * Sd_c - dj[D_VDC] * vd_c - dj[D_IRD] / Rd - dj[D_HIRD] * 0.5 / Rd);
    g[o + 2] = -dj[D_KS] * si - dj[D_OMK] * 2.0 * k / 3.0;
    g[j == 0 ? 11 : 18] = -dj[D_LD] * (1e-6 / ml) / ml;
    gi += dj[D_SDC] * Sd_c * si / ci - dj[D_KS] * k * ci;
  }
  g[3] = gi;
}

// MINB blocks per SM: 4 (64 registers) for the one-disc quadrature form, whose spills cost
// less than the extra warps gain; 3 (80 registers) for two discs and for the radial-table
// mode, whose shared memory holds 3 blocks per SM anyway.
template <int NQ, int ND, int PSF, int MINB>
__global__ void __launch_bounds__(kAdjThreads, MINB) adjoint_kernel(AdjArgs a) {
  constexpr int NACC = A_D0 + kPerDisc * ND;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ ModelConst mc;
  __shared__ GalDev gs;
  __shared__ double red[kAdjThreads / 32][NACC];

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  __shared__ int next_item;
  __shared__ float4 nodew[NQ / 2];
  __shared__ float2 tailc[kTailSetAdj];
  // first item by block index, then either the next one from the shared counter (dynamic
  // scheduling, longest items first) or a fixed stride
  for (int it = blockIdx.x; it < a.n_items;) {
    const int item_id = a.order ? a.order[it] : it;
    if (!BANG_IN(item_id, a.n_items, kSiteAdjItem)) {
      BANG_NEXT_ITEM(it);
      continue;
    }
    WorkItem w;
    if (a.items) {
      w = a.items[item_id];
    } else {   // implicit item: fine rows [k rows, (k + 1) rows) of row b, the row's galaxy read on the device
      const int b = item_id / a.nb, k = item_id - b * a.nb;
      const int g = a.gal_idx ? __ldg(a.gal_idx + b) : 0;
      const bool bad = (unsigned)g >= (unsigned)a.n_gal;   // decode marked the row invalid
      const int H = bad ? 0 : __ldg(&a.gals[g].H);
      const int y0 = k * a.rows_per_item;
      w = WorkItem{b, bad ? 0 : g, y0, min(H, y0 + a.rows_per_item)};
    }
    if (!BANG_IN(w.b, a.B, kSiteAdjRow) || !BANG_IN(w.g, a.n_gal, kSiteAdjGal)) {
      BANG_NEXT_ITEM(it);
      continue;
    }
    if (tid == 0) {
      gs = a.gals[w.g];
      mc = a.consts[w.b];
    }
    __syncthreads();
    if (!mc.valid) {   // outside the domain or without a galaxy: grad_out_kernel does not read the row's items
      BANG_NEXT_ITEM(it);
      continue;
    }
    if (w.j1 <= w.j0) {   // an empty band past the last fine row of a smaller galaxy: zero adjoints
      if (tid < kAdjSlots) a.acc_partial[(size_t)item_id * kAdjSlots + tid] = 0.0;
      BANG_NEXT_ITEM(it);
      continue;
    }
    const int L = gs.L, os = gs.os, W = gs.W, nx = gs.nx, ny = gs.ny, n = nx * ny;
    const float inv_os = 1.0f / (float)os, inv_nx = 1.0f / (float)nx;
    const int64_t soff = a.out_off ? a.out_off[w.b] : (int64_t)w.b * a.out_stride;
    const float* seed = a.seed + soff;
    // separable taps stored twice, (t, t): a 64-bit load gives the pair the packed
    // two-lane FMAs need; the L x L two-dimensional taps once (shared memory)
    float2* taps = reinterpret_cast<float2*>(smem_raw);
    float* taps2d = reinterpret_cast<float*>(smem_raw);
    const int ntaps = PSF == 0 ? L : L * L;
    float4* lam = reinterpret_cast<float4*>(smem_raw + (((size_t)ntaps * (PSF == 0 ? 8 : 4) + 15) / 16) * 16);
    const int nj_max = (a.G + L - 1) / os + 2;
    float4* V = lam + (size_t)nj_max * nx;
    float* tab = a.tables ? reinterpret_cast<float*>(V + (PSF == 0 ? (size_t)a.G * nx : 0)) : nullptr;
    // checked build: the layout fits the launch's shared memory; the item's fine rows, the
    // row's seed block and radial table are in range
    if (!BANG_IN((tab ? reinterpret_cast<const unsigned char*>(tab + kTabHdr + 8 * a.table_T)
                      : reinterpret_cast<const unsigned char*>(V + (PSF == 0 ? (size_t)a.G * nx : 0))) - smem_raw - 1,
                 dynamic_smem_bytes(), kSiteAdjSmem) ||
        !BANG_IN(w.j0, w.j1, kSiteAdjItem) || !BANG_IN(w.j1 - 1, gs.H, kSiteAdjItem) ||
        !BANG_IN(soff + 4ll * n - 1, a.seed_total, kSiteAdjSeed) ||
        (tab && !BANG_IN((long long)w.b * a.table_stride + kTabHdr + 8 * a.table_T - 1,
                         (long long)a.B * a.table_stride, kSiteAdjTable))) {
      BANG_NEXT_ITEM(it);
      continue;
    }
    for (int t = tid; t < ntaps; t += kAdjThreads) {
      const float tv = __ldg(gs.taps + t);
      if (PSF == 0) taps[t] = make_float2(tv, tv);
      else taps2d[t] = tv;
    }
    if (tab) {
      const float* src = a.tables + (size_t)w.b * a.table_stride;
      const int nt = kTabHdr + 8 * a.table_T;
      for (int t = tid; t < nt; t += kAdjThreads) tab[t] = __ldg(src + t);
    } else if (!mc.bulge_fit) {
      fill_node_pairs<NQ>(mc, nodew, tid, kAdjThreads);
      if (tid < 32) fill_tail_coeffs_adj<NQ>(mc, tailc, tid);
    }

    float acc[NACC];
#pragma unroll
    for (int k = 0; k < NACC; ++k) acc[k] = 0.f;
    const float pk = gs.pitch_kpa;
    for (int y0 = w.j0; y0 < w.j1; y0 += a.G) {
      const int G = min(a.G, w.j1 - y0);
      int jlo = y0 - L + 1 <= 0 ? 0 : (y0 - L + os) / os;
      const int jhi = min(ny - 1, (y0 + G - 1) / os);
      const int nj = jhi - jlo + 1;
      __syncthreads();   // taps loaded / previous chunk's lam and V no longer read
      if (!BANG_IN(nj, nj_max + 1, kSiteAdjLam)) break;   // uniform: every thread leaves the item's loop
      for (int t = tid; t < nj * nx; t += kAdjThreads) {
        const int tj = floor_div(t, inv_nx);
        const int s = (jlo + tj) * nx + (t - tj * nx);
        lam[t] = make_float4(__ldg(seed + s), __ldg(seed + n + s), __ldg(seed + 2 * n + s), __ldg(seed + 3 * n + s));
      }
      __syncthreads();
      if (PSF == 0) {
        // vertical transposed pass: V[g][i] = sum_j T[y - j os] lambda(i, j)
        for (int t = tid; t < G * nx; t += kAdjThreads) {
          const int gr = floor_div(t, inv_nx), i = t - gr * nx;
          const int y = y0 + gr;
          int j0 = y - L + 1 <= 0 ? 0 : floor_div(y - L + os, inv_os);
          const int j1 = min(ny - 1, floor_div(y, inv_os));
          float2 vxy = make_float2(0.f, 0.f), vzw = vxy;
          for (int j = j0; j <= j1; ++j) {
            if (!BANG_IN(y - j * os, L, kSiteAdjTap) || !BANG_IN(j - jlo, nj, kSiteAdjLam)) continue;
            const float2 tv = taps[y - j * os];
            const float4 l = lam[(j - jlo) * nx + i];
            vxy = __ffma2_rn(tv, make_float2(l.x, l.y), vxy);
            vzw = __ffma2_rn(tv, make_float2(l.z, l.w), vzw);
          }
          V[t] = make_float4(vxy.x, vxy.y, vzw.x, vzw.y);
        }
        __syncthreads();
      }
      // point VJPs, 32 points per grab from the shared counter (balances the warps)
      const int npts = G * W;
      const float inv_W = 1.0f / (float)W;
      // 32-point batches in a fixed order (warp w takes batches w, w + 8, ...): every
      // accumulation order is fixed, so the gradient is the same bits on every call
      for (int base = warp * 32; base < npts; base += kAdjThreads) {
        const int p = base + lane;
        if (p >= npts) continue;
        const int gr = __float2int_rz(((float)p + 0.5f) * inv_W);   // p + 1/2 is never a multiple of W
        const int qx = p - gr * W;
        const int y = y0 + gr;
        int i0 = qx - L + 1 <= 0 ? 0 : floor_div(qx - L + os, inv_os);
        const int i1 = min(nx - 1, floor_div(qx, inv_os));
        float2 sxy = make_float2(0.f, 0.f), szw = sxy;
        if (PSF == 0) {
          for (int i = i0; i <= i1; ++i) {
            if (!BANG_IN(qx - i * os, L, kSiteAdjTap) || !BANG_IN(gr * nx + i, G * nx, kSiteAdjV)) continue;
            const float2 th_ = taps[qx - i * os];
            const float4 v = V[gr * nx + i];
            sxy = __ffma2_rn(th_, make_float2(v.x, v.y), sxy);
            szw = __ffma2_rn(th_, make_float2(v.z, v.w), szw);
          }
        } else {
          int j0 = y - L + 1 <= 0 ? 0 : floor_div(y - L + os, inv_os);
          const int j1 = min(ny - 1, floor_div(y, inv_os));
          for (int j = j0; j <= j1; ++j) {
            if (!BANG_IN(y - j * os, L, kSiteAdjTap) || !BANG_IN(j - jlo, nj, kSiteAdjLam)) continue;
            const float* wrow = taps2d + (y - j * os) * L;
            for (int i = i0; i <= i1; ++i) {
              if (!BANG_IN(qx - i * os, L, kSiteAdjTap)) continue;
              const float2 tw = make_float2(wrow[qx - i * os], wrow[qx - i * os]);
              const float4 l = lam[(j - jlo) * nx + i];
              sxy = __ffma2_rn(tw, make_float2(l.x, l.y), sxy);
              szw = __ffma2_rn(tw, make_float2(l.z, l.w), szw);
            }
          }
        }
        const float X = fmaf((float)qx, pk, mc.X0);
        const float Y = fmaf((float)y, pk, mc.Y0);
        point_vjp<NQ, ND>(mc, X, Y, make_float4(sxy.x, sxy.y, szw.x, szw.y), acc, tab, a.table_T, nodew, tailc);
      }
    }
    // block reduction of the adjoints: lane k of each warp ends with the warp's sum of
    // accumulator k, then one thread per accumulator sums the warps in float64
    {
      const double v = warp_sum_scatter<NACC>(acc, lane);
      if (lane < NACC) red[warp][lane] = v;
    }
    __syncthreads();
    if (tid < NACC) {   // one thread per accumulator: sum over warps into the item's slots
      double sum = 0.0;
      for (int q = 0; q < kAdjThreads / 32; ++q) sum += red[q][tid];
      a.acc_partial[(size_t)item_id * kAdjSlots + tid] = sum;
    }
    BANG_NEXT_ITEM(it);
  }
}

// One warp per row: the constant adjoints of the row's work items, summed in item order
// (lane k < kAdjSlots sums slot k, lane kVsysSlot the forward items' d logL / d v_sys),
// then mapped to d logL / d theta (float64), or zero for a row outside the parameter
// domain.  As in decode_kernel, lane i < kDecodeTerms also evaluates decode term i and
// lane 0 does the rest.  No atomics: the gradient is the same bits on every call.
// adj_row_first / row_first NULL: row b's items are [b adj_nb, (b + 1) adj_nb) and
// [b nb, (b + 1) nb); gal_idx (may be NULL): a row whose galaxy index is outside [0, n_gal)
// gets a zero gradient.
__global__ void grad_out_kernel(const float* __restrict__ theta, int P, int nd, int halo_kind, int bulge_kind,
                                const double* __restrict__ acc_partial, const int* __restrict__ adj_row_first,
                                const double* __restrict__ vsys_partial, const int* __restrict__ row_first, int B,
                                int n_items, int adj_items, int adj_nb, int nb, const int* __restrict__ gal_idx,
                                int n_gal, double l10k, float* __restrict__ grad) {
  const int b = (int)((blockIdx.x * (unsigned)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (b >= B) return;   // whole warps
  const float* th = theta + (size_t)b * P;
  const bool ok = theta_in_domain(th, nd, halo_kind, bulge_kind) &&
                  (!gal_idx || (unsigned)gal_idx[b] < (unsigned)n_gal);
  const float v = (ok && lane < kDecodeTerms) ? decode_term(lane, th, nd, halo_kind, l10k) : 0.f;
  float T[kDecodeTerms];
#pragma unroll
  for (int i = 0; i < kDecodeTerms; ++i) T[i] = __shfl_sync(0xffffffffu, v, i);
  double sum = 0.0;
  if (ok && lane < kAdjSlots) {
    const int i0 = adj_row_first ? adj_row_first[b] : b * adj_nb;
    const int i1 = adj_row_first ? adj_row_first[b + 1] : (b + 1) * adj_nb;
    for (int i = i0; i < i1; ++i)
      if (BANG_IN(i, adj_items, kSiteFinalizeItem)) sum += acc_partial[(size_t)i * kAdjSlots + lane];
  } else if (ok && lane == kVsysSlot) {
    const int i0 = row_first ? row_first[b] : b * nb, i1 = row_first ? row_first[b + 1] : (b + 1) * nb;
    for (int i = i0; i < i1; ++i)
      if (BANG_IN(i, n_items, kSiteFinalizeItem)) sum += vsys_partial[i];
  }
  double s[kVsysSlot + 1];
#pragma unroll
  for (int k = 0; k <= kVsysSlot; ++k) s[k] = __shfl_sync(0xffffffffu, sum, k);
  if (lane != 0) return;
  double g[kMaxParams];
  for (int p = 0; p < kMaxParams; ++p) g[p] = 0.0;
  if (ok) {
    constants_to_theta(th, T, nd, halo_kind, bulge_kind, s, g);
    g[14] = s[kVsysSlot];
  }
  for (int p = 0; p < P; ++p) grad[(size_t)b * P + p] = (float)g[p];
}

// Radial table of one row per block: Sigma and Q (and, for the adjoint, their slopes in
// ln R and ln-derivatives in gamma) by the radial quadrature at T radii, t = log2(R / a)
// uniform from the 1e-6 kpc floor to 1% beyond the farthest fine point; then the
// log-ratios of neighbouring values.  Node positions are formed in float64 so that the
// lookup's t0 + k h holds to float32 rounding.
template <int NQ>
__global__ void table_kernel(const ModelConst* __restrict__ consts, const GalDev* __restrict__ gals,
                             const int* __restrict__ row_g, int n_gal, int T, int derivs, float* __restrict__ tables,
                             int64_t stride) {
  const int b = blockIdx.x;
  __shared__ ModelConst m;
  __shared__ double t0h[2];
  if (threadIdx.x == 0) {
    m = consts[b];
    const int gi = row_g ? row_g[b] : 0;
    const bool gal_ok = (unsigned)gi < (unsigned)n_gal && BANG_IN(gi, n_gal, kSiteDecodeGal);
    if (!gal_ok || !BANG_IN(kTabHdr + (derivs ? 8 : 4) * T - 1, stride, kSiteTable)) m.valid = 0;
    const GalDev g = gals[gal_ok ? gi : 0];
    const double xa = m.X0, xb = m.X0 + (double)(g.W - 1) * g.pitch_kpa;
    const double ya = m.Y0, yb = m.Y0 + (double)(g.H - 1) * g.pitch_kpa;
    const double rmax = sqrt(fmax(xa * xa, xb * xb) + fmax(ya * ya, yb * yb));
    const double inv_a = m.inv_a;
    const double t_lo = log2(1e-6 * inv_a);
    double t_hi = log2(fmax(rmax * 1.01, 2e-6) * inv_a);
    if (t_hi < t_lo + 1.0) t_hi = t_lo + 1.0;
    const double h = (t_hi - t_lo) / (T - 4);
    // the float32 header the lookup uses; node positions follow from it exactly
    t0h[0] = (double)(float)(t_lo - h);
    t0h[1] = (double)(float)(1.0 / h);
  }
  __syncthreads();
  if (!m.valid) return;
  float* tab = tables + (size_t)b * stride;
  if (threadIdx.x == 0) {
    tab[0] = (float)t0h[0];
    tab[1] = (float)t0h[1];
    tab[2] = 0.f;
    tab[3] = 0.f;
  }
  float* VS = tab + kTabHdr + TAB_VS * T;
  float* VQ = tab + kTabHdr + TAB_VQ * T;
  for (int k = threadIdx.x; k < T; k += blockDim.x) {
    // the lookup maps R to u = (log2(R / a) - t0) / h; node k sits at u = k
    const double tk = t0h[0] + (double)k / t0h[1];
    const float R = (float)(exp2(tk) / (double)m.inv_a);
    if (derivs) {
      const BulgeDer d = bulge_projected_vjp<NQ>(m, R);
      VS[k] = d.Sb;
      VQ[k] = d.Qb;
      tab[kTabHdr + TAB_SS * T + k] = R * d.dSb_dR / d.Sb;
      tab[kTabHdr + TAB_SQ * T + k] = R * d.dQb_dR / d.Qb;
      tab[kTabHdr + TAB_GS * T + k] = d.dSb_dg / d.Sb;
      tab[kTabHdr + TAB_GQ * T + k] = d.dQb_dg / d.Qb;
    } else {
      float S, Q;
      bulge_projected<NQ>(m, R, S, Q);
      VS[k] = S;
      VQ[k] = Q;
    }
  }
  __syncthreads();
  float* DS = tab + kTabHdr + TAB_DS * T;
  float* DQ = tab + kTabHdr + TAB_DQ * T;
  for (int k = threadIdx.x; k < T; k += blockDim.x) {
    DS[k] = k + 1 < T ? log2f(VS[k + 1] / VS[k]) : 0.f;
    DQ[k] = k + 1 < T ? log2f(VQ[k + 1] / VQ[k]) : 0.f;
  }
}

constexpr int adj_min_blocks(int nd, bool table) { return nd == 1 && !table ? 4 : 3; }

// minb 3 runs the one-disc quadrature form at 3 blocks per SM (80 registers, the table
// form's instance, which handles tables == NULL by the per-point quadrature)
template <int NQ, int ND>
cudaError_t launch_nd(const AdjArgs& a, int psf2d, int minb, int grid, size_t smem, cudaStream_t st) {
  constexpr int kQuad = adj_min_blocks(ND, false), kTab = adj_min_blocks(ND, true);
  if (a.tables || minb == kTab) {
    if (psf2d) adjoint_kernel<NQ, ND, 1, kTab><<<grid, kAdjThreads, smem, st>>>(a);
    else adjoint_kernel<NQ, ND, 0, kTab><<<grid, kAdjThreads, smem, st>>>(a);
  } else {
    if (psf2d) adjoint_kernel<NQ, ND, 1, kQuad><<<grid, kAdjThreads, smem, st>>>(a);
    else adjoint_kernel<NQ, ND, 0, kQuad><<<grid, kAdjThreads, smem, st>>>(a);
  }
  return cudaGetLastError();
}

}  // namespace

int adjoint_threads() { return kAdjThreads; }

size_t adjoint_smem_bytes(int L, int os, int nx, int G, int psf2d, int table_T) {
  const int ntaps = psf2d ? L * L : L;
  const int nj_max = (G + L - 1) / os + 2;
  return (((size_t)ntaps * (psf2d ? 4 : 8) + 15) / 16) * 16 + (size_t)nj_max * nx * 16 + (psf2d ? 0 : (size_t)G * nx * 16) +
         (table_T > 0 ? sizeof(float) * (size_t)(kTabHdr + 8 * table_T) : 0);
}

int64_t table_row_floats(int T, int derivs) { return kTabHdr + (int64_t)(derivs ? 8 : 4) * T; }

int adjoint_minb(int n_discs, int table, int want) {
  if (n_discs == 1 && !table && (want == 3 || want == 4)) return want;
  return adj_min_blocks(n_discs, table != 0);
}

const void* adjoint_kernel_ptr(int n_quad, int n_discs, int psf2d, int table, int minb) {
#define BANG_PICK(NQ, ND, PSF)                                                                        \
  if (n_quad == NQ && n_discs == ND && psf2d == PSF)                                                  \
    return (table || minb == adj_min_blocks(ND, true))                                                \
               ? (const void*)adjoint_kernel<NQ, ND, PSF, adj_min_blocks(ND, true)>                   \
               : (const void*)adjoint_kernel<NQ, ND, PSF, adj_min_blocks(ND, false)>;
  BANG_PICK(64, 1, 0) BANG_PICK(64, 1, 1) BANG_PICK(64, 2, 0) BANG_PICK(64, 2, 1)
  BANG_PICK(128, 1, 0) BANG_PICK(128, 1, 1) BANG_PICK(128, 2, 0) BANG_PICK(128, 2, 1)
#undef BANG_PICK
  return nullptr;
}

cudaError_t launch_adjoint(const AdjArgs& a, int n_quad, int n_discs, int psf2d, int minb, int grid, size_t smem,
                           cudaStream_t st) {
  if (n_quad == 64)
    return n_discs == 2 ? launch_nd<64, 2>(a, psf2d, minb, grid, smem, st) : launch_nd<64, 1>(a, psf2d, minb, grid, smem, st);
  return n_discs == 2 ? launch_nd<128, 2>(a, psf2d, minb, grid, smem, st) : launch_nd<128, 1>(a, psf2d, minb, grid, smem, st);
}

cudaError_t launch_tables(const ModelConst* consts, const GalDev* gals, const int* row_g, int n_gal, int B, int n_quad,
                          int T, int derivs, float* tables, int64_t stride, cudaStream_t st) {
  if (n_quad == 64) table_kernel<64><<<B, 256, 0, st>>>(consts, gals, row_g, n_gal, T, derivs, tables, stride);
  else table_kernel<128><<<B, 256, 0, st>>>(consts, gals, row_g, n_gal, T, derivs, tables, stride);
  return cudaGetLastError();
}

BANG_DEFINE_FAULT_TAKER(take_fault_adjoint)

cudaError_t launch_grad_out(const float* theta, int P, int n_discs, int halo_kind, int bulge_kind,
                            const double* acc_partial, const int* adj_row_first, const double* vsys_partial,
                            const int* row_first, int B, int n_items, int adj_items, float* grad, cudaStream_t st,
                            int adj_nb, int nb, const int* gal_idx, int n_gal) {
  constexpr int kRowsPerBlock = 4;   // 4 warps, one row each
  const double l10k = std::log10(3.0 / (4.0 * kPi * 200.0 * kRhoCrit));
  grad_out_kernel<<<(B + kRowsPerBlock - 1) / kRowsPerBlock, 32 * kRowsPerBlock, 0, st>>>(
      theta, P, n_discs, halo_kind, bulge_kind, acc_partial, adj_row_first, vsys_partial, row_first, B, n_items,
      adj_items, adj_nb, nb, gal_idx, n_gal, l10k, grad);
  return cudaGetLastError();
}

cudaError_t upload_nodes_adjoint(const float* cm1, const float* lc, const float* ws, const float* wq) {
  float lm[192], lcm[192];   // the series' log tables, from the float32 m_k
  for (int k = 0; k < 192; ++k) {
    const double mk = (double)cm1[k];
    lm[k] = (float)std::log2(mk);
    lcm[k] = (float)std::log2(1.0 + 1.0 / mk);
  }
  cudaError_t e = cudaMemcpyToSymbol(kNodeCm1, cm1, 192 * sizeof(float));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(kNodeLm, lm, sizeof lm);
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(kNodeLcm, lcm, sizeof lcm);
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(kNodeLc, lc, 192 * sizeof(float));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(kNodeWs, ws, 192 * sizeof(float));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(kNodeWq, wq, 192 * sizeof(float));
  return e;
}

}  // namespace bang
