// Float64 check path (bang_loglike_fp64): the same discrete model as the float32 kernels
// (padded fine grid, fixed radial rule, PSF (x) box taps, chi-square), every step in
// float64 and in its plainest form, one kernel per step.  It compares the GPU's
// discretisation with the float64 oracle without float32 rounding in between; it is not
// built for speed.
//   1. fp64_points: one thread per padded fine point evaluates the point model of
//      Sec. 2.1-2.4: the radial quadrature node by node from the definitions
//      Sigma = 2 sum_k w_k rho(R c_k) R c_k and Sigma sigma^2 = 2 G sum_k w_k tanh^2 t_k
//      rho(R c_k) M(R c_k) with c_k = cosh t_k; the Freeman disc velocity from the
//      modified Bessel functions; the NFW or Hernquist halo; the four observables.
//   2. fp64_spaxels: one thread per spaxel: the PSF (x) box window sum (Eq. 21), the
//      residuals against the data and the spaxel's chi-square.
//   3. fp64_sum: one block: the spaxels' chi-square summed in a fixed order, then logL.
#include <cuda_runtime.h>

#include <cmath>

#include "bang_device.cuh"
#include "bang_internal.h"

namespace bang {
namespace {

constexpr int kFp64Threads = 128;
constexpr int kFp64SumThreads = 256;
constexpr double kR2Floor64 = 1e-12;   // radii floored at 1e-6 kpc

// K0(x) and K1(x), x > 0, from K_nu(x) = int_0^inf exp(-x cosh t) cosh(nu t) dt by the
// trapezoid rule.  The integrand is entire and decays doubly exponentially, so the rule
// converges spectrally: step 0.1, narrowed to 0.1 sqrt(10 / x) beyond x = 10 where the
// integrand's width shrinks like 1 / sqrt(x); the sum stops where x cosh t > 745 and the
// exponential underflows.  Relative error below 2e-14 for x in [1e-6, 200] (checked
// against an independent library on the host).
__device__ void bessel_k01(double x, double& k0, double& k1) {
  const double h = x <= 10.0 ? 0.1 : 0.1 * sqrt(10.0 / x);
  const double tmax = x < 745.0 ? acosh(745.0 / x) : 0.0;
  const int n = (int)ceil(tmax / h) + 1;
  double s0 = 0.5 * exp(-x), s1 = s0;
  for (int i = 1; i <= n; ++i) {
    const double t = i * h, c = cosh(t), e = exp(-x * c);
    s0 += e;
    s1 += e * c;
  }
  k0 = h * s0;
  k1 = h * s1;
}

// I0(y) K0(y) - I1(y) K1(y) for y > 25 from the large-argument expansion of the products
// I_nu K_nu (DLMF 10.40.6): I_nu(y) K_nu(y) ~ (1 / 2y) sum_k (-1)^k c_k p_k(nu) / (2y)^(2k),
// c_k = (1 3 ... (2k-1)) / (2 4 ... 2k), p_k(nu) = prod_{j<=k} (4 nu^2 - (2j-1)^2).  The
// k = 0 terms of nu = 0 and 1 cancel exactly, so the difference is summed term by term
// without the cancellation of the direct form; twelve terms give double precision from
// y = 25 on (the leading term is 1 / (4 y^3)).
__device__ double freeman_bessel_series(double y) {
  const double z2 = 1.0 / (4.0 * y * y);
  double s = 0.0, c = 1.0, p0 = 1.0, p1 = 1.0, zk = 1.0;
  for (int k = 1; k <= 12; ++k) {
    const double o = (2.0 * k - 1.0) * (2.0 * k - 1.0);
    c *= (2.0 * k - 1.0) / (2.0 * k);
    p0 *= -o;          // nu = 0
    p1 *= 4.0 - o;     // nu = 1
    zk *= z2;
    s += ((k & 1) ? -c : c) * (p0 - p1) * zk;
  }
  return s / (2.0 * y);
}

// I0(y) K0(y) - I1(y) K1(y) of the Freeman disc: the Bessel functions themselves up to
// y = 25 (where the difference has lost ~y^2 x 1e-16 to cancellation), the expansion beyond
// (I0 would overflow near y = 700).
__device__ double freeman_bessel(double y) {
  if (y > 25.0) return freeman_bessel_series(y);
  double k0, k1;
  bessel_k01(y, k0, k1);
  return cyl_bessel_i0(y) * k0 - cyl_bessel_i1(y) * k1;
}

// The model's parameters from theta (slot layout of include/bang.h).
struct Const64 {
  double X0, Y0, cpa, spa, ci, si;
  double Mb, a, gam, Lb;
  double Mh, rh, mc;   // NFW: M_200, r_s, ln(1 + c) - c / (1 + c); Hernquist: M_h, R_h
  double Md[2], Rd[2], k[2], Ld[2];
  double vsys;
};

__device__ Const64 decode64(const double* __restrict__ th, int nd, int halo_kind, const Gal64& g) {
  Const64 m;
  m.X0 = g.xoff - th[0];
  m.Y0 = g.yoff - th[1];
  m.cpa = cos(th[2]);
  m.spa = sin(th[2]);
  m.ci = cos(th[3]);
  m.si = sin(th[3]);
  m.Mb = exp10(th[4]);
  m.a = exp10(th[5]);
  m.gam = th[6];
  m.Lb = 1e-6 / th[10];
  if (halo_kind == 0) {   // NFW: r_200 = (3 M_200 / (4 pi 200 rho_c))^(1/3), r_s = r_200 / c
    const double c = th[13];
    m.Mh = exp10(th[12]);
    m.rh = cbrt(3.0 * m.Mh / (4.0 * kPi * 200.0 * kRhoCrit)) / c;
    m.mc = log1p(c) - c / (1.0 + c);
  } else {                // Hernquist (M_h, R_h)
    m.Mh = exp10(th[12]);
    m.rh = exp10(th[13]);
    m.mc = 1.0;
  }
  for (int j = 0; j < 2; ++j) {
    const int o = j == 0 ? 7 : 15;
    const bool on = j < nd;
    m.Md[j] = on ? exp10(th[o]) : 0.0;
    m.Rd[j] = on ? exp10(th[o + 1]) : 1.0;
    m.k[j] = on ? th[o + 2] : 0.0;
    m.Ld[j] = on ? 1e-6 / (j == 0 ? th[11] : th[18]) : 0.0;
  }
  m.vsys = th[14];
  return m;
}

__global__ void fp64_points(const double* __restrict__ th, int nd, int halo_kind, Nodes64 nodes, Gal64 g,
                            double* __restrict__ f) {
  const int N = g.W * g.H;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= N) return;
  const Const64 m = decode64(th, nd, halo_kind, g);
  const int qy = p / g.W, qx = p - qy * g.W;
  // Sec. 2.1: sky offsets from the centre, rotated onto the major axis; disc plane by 1 / cos i
  const double X = m.X0 + qx * g.pitch, Y = m.Y0 + qy * g.pitch;
  const double xr = X * m.cpa + Y * m.spa, yr = Y * m.cpa - X * m.spa;
  const double yd = yr / m.ci;
  const double R = sqrt(fmax(X * X + Y * Y, kR2Floor64));
  const double r = sqrt(fmax(xr * xr + yd * yd, kR2Floor64));
  const double cphi = xr / r;

  // bulge (Dehnen): rho(r) = (3 - g) M a / (4 pi r^g (r + a)^(4 - g)), M(r) = M (r / (r + a))^(3 - g)
  const double g3 = 3.0 - m.gam;
  double S = 0.0, Q = 0.0;
  for (int k = 0; k < nodes.n; ++k) {
    const double rk = R * nodes.ch[k];
    const double rho = g3 * m.Mb * m.a / (4.0 * kPi * pow(rk, m.gam) * pow(rk + m.a, 4.0 - m.gam));
    const double Mr = m.Mb * pow(rk / (rk + m.a), g3);
    S += nodes.w[k] * rho * rk;
    Q += nodes.w[k] * nodes.th2[k] * rho * Mr;
  }
  const double Sb = 2.0 * S, Qb = 2.0 * kG * Q;   // Sigma_b and Sigma_b sigma_b^2

  // circular velocities in the disc plane (Eq. 10)
  double vint2 = kG * m.Mb * pow(r / (r + m.a), g3) / r;
  if (halo_kind == 0) {
    const double x = r / m.rh;
    vint2 += kG * m.Mh * (log1p(x) - x / (1.0 + x)) / (m.mc * r);
  } else {
    vint2 += kG * m.Mh * r / ((r + m.rh) * (r + m.rh));
  }
  double Sd[2] = {0.0, 0.0};
  for (int j = 0; j < nd; ++j) {
    const double y = r / (2.0 * m.Rd[j]);
    vint2 += 2.0 * kG * m.Md[j] / m.Rd[j] * y * y * freeman_bessel(y);
    Sd[j] = m.Md[j] * exp(-r / m.Rd[j]) / (2.0 * kPi * m.Rd[j] * m.Rd[j] * m.ci);
  }
  const double vint = sqrt(vint2);

  // light weighting (Eqs. 13-15, 19)
  double B = Sb * m.Lb, Bv = 0.0, Bs2 = Qb * m.Lb, Stot = Sb;
  for (int j = 0; j < nd; ++j) {
    const double Bd = Sd[j] * m.Ld[j];
    B += Bd;
    Bv += Bd * (-m.k[j] * m.si * cphi * vint);
    Bs2 += Bd * (1.0 - m.k[j] * m.k[j]) / 3.0 * vint2;
    Stot += Sd[j];
  }
  f[p] = B;
  f[N + p] = Bv / B;
  f[2 * N + p] = sqrt(Bs2 / B);
  f[3 * N + p] = B * 1e6 / Stot;
}

__global__ void fp64_spaxels(const double* __restrict__ th, Gal64 g, const double* __restrict__ f,
                             double* __restrict__ chi) {
  const int n = g.nx * g.ny;
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const int j = s / g.nx, i = s - j * g.nx;
  const int N = g.W * g.H, L = g.L;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int cy = 0; cy < L; ++cy)
    for (int cx = 0; cx < L; ++cx) {
      const double wgt = g.psf2d ? g.taps[cy * L + cx] : g.taps[cy] * g.taps[cx];
      const int q = (j * g.os + cy) * g.W + i * g.os + cx;
      for (int c = 0; c < 4; ++c) acc[c] += wgt * f[c * N + q];
    }
  const double model[4] = {acc[0], acc[1] + th[14], acc[2], 1.0 / acc[3]};
  double c2 = 0.0;
  for (int c = 0; c < 4; ++c) {
    const double iv = g.iv[c * n + s];
    if (iv == 0.0) continue;   // masked
    const double res = model[c] - (double)g.data[c * n + s];
    c2 += iv * res * res;
  }
  chi[s] = c2;
}

__global__ void fp64_sum(const double* __restrict__ chi, int n, double norm_const, double* __restrict__ logL) {
  __shared__ double red[kFp64SumThreads];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += kFp64SumThreads) s += chi[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = kFp64SumThreads / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *logL = isnan(red[0]) ? -INFINITY : -0.5 * red[0] - norm_const;
}

}  // namespace

size_t fp64_scratch_bytes(int N, int n) { return sizeof(double) * ((size_t)4 * N + (size_t)n) + 256; }

cudaError_t launch_fp64_row(const double* theta, int nd, int halo_kind, const Nodes64& nodes, const Gal64& g,
                            void* scratch, double* logL, cudaStream_t st) {
  const int N = g.W * g.H, n = g.nx * g.ny;
  double* f = static_cast<double*>(scratch);
  double* chi = f + (size_t)4 * N;
  fp64_points<<<(N + kFp64Threads - 1) / kFp64Threads, kFp64Threads, 0, st>>>(theta, nd, halo_kind, nodes, g, f);
  fp64_spaxels<<<(n + kFp64Threads - 1) / kFp64Threads, kFp64Threads, 0, st>>>(theta, g, f, chi);
  fp64_sum<<<1, kFp64SumThreads, 0, st>>>(chi, n, g.norm_const, logL);
  return cudaGetLastError();
}

}  // namespace bang
