// The paper's execution form (App. A, Alg. 2), kept as the comparison baseline.
//
// For every parameter vector: a serial chain of kernels, one per task of the model, each
// with one thread per padded fine point and 64 threads per block; intermediate arrays live
// in device memory; the PSF kernel has one thread per spaxel summing over its window; the
// chi-square is a block reduction plus float64 atomics.  The arithmetic is the same as the
// fused kernel's (bang_device.cuh); only the execution form differs.
#include <cuda_runtime.h>

#include "bang_device.cuh"
#include "bang_internal.h"

namespace bang {
namespace {

constexpr int kPlainThreads = 64;   // App. A: 64 threads per block in the paper's execution form

struct PlainBufs {
  float *R, *r, *cphi, *Sb, *Qb, *vint2, *Sd0, *Sd1, *f;   // [N] each, f [4][N]
  float* F;                                                 // [4][nx*ny]
  double* chi;                                              // [1]
  ModelConst* mc;                                           // [1]
};

__global__ void plain_decode(const float* __restrict__ theta, int nd, int halo_kind, const GalDev* __restrict__ gal,
                             ModelConst* __restrict__ mc, double* __restrict__ chi) {
  ModelConst m;
  m.valid = decode_model(theta, nd, halo_kind, *gal, m);
  *mc = m;
  *chi = 0.0;
}

// task 1: coordinates (Sec. 2.1)
__global__ void plain_coords(const GalDev* __restrict__ gal, const ModelConst* __restrict__ mcp, PlainBufs b) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  const GalDev& g = *gal;
  if (p >= g.W * g.H || !mcp->valid) return;
  const ModelConst& m = *mcp;
  const int qy = p / g.W, qx = p - qy * g.W;
  const float X = fmaf((float)qx, g.pitch_kpa, m.X0);
  const float Y = fmaf((float)qy, g.pitch_kpa, m.Y0);
  const float xr = fmaf(X, m.cpa, Y * m.spa);
  const float yr = fmaf(Y, m.cpa, -X * m.spa);
  const float R2 = fmaf(X, X, Y * Y);
  const float yd = yr * m.inv_ci;
  const float r2 = fmaf(xr, xr, yd * yd);
  b.R[p] = sqrtf(fmaxf(R2, kR2Floor));
  const float r = sqrtf(fmaxf(r2, kR2Floor));
  b.r[p] = r;
  b.cphi[p] = xr * (1.0f / r);
}

// task 2: bulge projected density and dispersion (Sec. 2.2)
template <int NQ>
__global__ void plain_bulge(const GalDev* __restrict__ gal, const ModelConst* __restrict__ mcp, PlainBufs b) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= gal->W * gal->H || !mcp->valid) return;
  float S, Q;
  if (mcp->bulge_fit) bulge_closed(*mcp, b.R[p], S, Q);
  else bulge_projected<NQ>(*mcp, b.R[p], S, Q);
  b.Sb[p] = S;
  b.Qb[p] = Q;
}

// task 3: circular velocities (Eq. 10)
template <int ND>
__global__ void plain_velocity(const GalDev* __restrict__ gal, const ModelConst* __restrict__ mcp, PlainBufs b) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= gal->W * gal->H || !mcp->valid) return;
  const ModelConst& m = *mcp;
  const float r = b.r[p];
  const float xa = r * m.inv_a;
  const float ub = xa / (xa + 1.0f);
  float v2 = m.vb_c * exp2f(m.three_mg * log2f(ub)) / xa;
  v2 += halo_v2(m, r, 1.0f / r);
#pragma unroll
  for (int j = 0; j < ND; ++j) v2 += m.vd_c[j] * disc_F(r * m.half_inv_Rd[j]);
  b.vint2[p] = v2;
}

// task 4: disc surface densities (Eqs. 7-8)
template <int ND>
__global__ void plain_discs(const GalDev* __restrict__ gal, const ModelConst* __restrict__ mcp, PlainBufs b) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= gal->W * gal->H || !mcp->valid) return;
  const ModelConst& m = *mcp;
  const float r = b.r[p];
  b.Sd0[p] = m.Sd_c[0] * expf(-r * m.inv_Rd[0]);
  if (ND == 2) b.Sd1[p] = m.Sd_c[1] * expf(-r * m.inv_Rd[1]);
}

// task 5: light-weighted observables (Eqs. 11-15, 19)
template <int ND>
__global__ void plain_combine(const GalDev* __restrict__ gal, const ModelConst* __restrict__ mcp, PlainBufs b) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  const int N = gal->W * gal->H;
  if (p >= N || !mcp->valid) return;
  const ModelConst& m = *mcp;
  const float vint2 = b.vint2[p];
  const float vint = sqrtf(vint2);
  const float cphi = b.cphi[p];
  const float Sb = b.Sb[p];
  const float Sd[2] = {b.Sd0[p], ND == 2 ? b.Sd1[p] : 0.f};
  float B = Sb * m.Lb, Bv = 0.f, Bs2 = b.Qb[p] * m.Lb, Stot = Sb;
#pragma unroll
  for (int j = 0; j < ND; ++j) {
    const float Bd = Sd[j] * m.Ld[j];
    B += Bd;
    Bv = fmaf(Bd, m.ks[j] * cphi * vint, Bv);
    Bs2 = fmaf(Bd, m.omk[j] * vint2, Bs2);
    Stot += Sd[j];
  }
  const float iB = 1.0f / B;
  b.f[p] = B;
  if (m.flux) {   // flux-weighted PSF mode: B v, B (sigma^2 + v^2), 1e-6 Sigma_tot
    b.f[N + p] = Bv;
    b.f[2 * N + p] = fmaf(Bv * iB, Bv, Bs2);
    b.f[3 * N + p] = 1e-6f * Stot;
    return;
  }
  b.f[N + p] = Bv * iB;
  b.f[2 * N + p] = sqrtf(Bs2 * iB);
  b.f[3 * N + p] = B * 1e6f / Stot;
}

// task 6: PSF + binning, one thread per spaxel summing over its (os + 2h)^2 window (Eq. 21)
template <int PSF>
__global__ void plain_psf(const GalDev* __restrict__ gal, const ModelConst* __restrict__ mcp, PlainBufs b) {
  const GalDev& g = *gal;
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= g.nx * g.ny || !mcp->valid) return;
  const int j = s / g.nx, i = s - j * g.nx;
  const int N = g.W * g.H, L = g.L;
  // checked build: the spaxel's last window point lies on the padded fine grid
  if (!BANG_IN((long long)(j * g.os + L - 1) * g.W + i * g.os + L - 1, N, kSitePlain) ||
      !BANG_IN(i * g.os + L - 1, g.W, kSitePlain))
    return;
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int cy = 0; cy < L; ++cy) {
    const int qy = j * g.os + cy;
    for (int cx = 0; cx < L; ++cx) {
      const float wgt = PSF == 0 ? g.taps[cy] * g.taps[cx] : g.taps[cy * L + cx];
      const int q = qy * g.W + i * g.os + cx;
      acc.x = fmaf(wgt, b.f[q], acc.x);
      acc.y = fmaf(wgt, b.f[N + q], acc.y);
      acc.z = fmaf(wgt, b.f[2 * N + q], acc.z);
      acc.w = fmaf(wgt, b.f[3 * N + q], acc.w);
    }
  }
  const int n = g.nx * g.ny;
  b.F[s] = acc.x;
  b.F[n + s] = acc.y;
  b.F[2 * n + s] = acc.z;
  b.F[3 * n + s] = acc.w;
}

// task 7: chi-square (Eq. 18), float32 per spaxel, float64 across spaxels
__global__ void plain_chi2(const GalDev* __restrict__ gal, const ModelConst* __restrict__ mcp, PlainBufs b) {
  __shared__ double red[kPlainThreads / 32];
  const GalDev& g = *gal;
  const int n = g.nx * g.ny;
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  double v = 0.0;
  if (s < n && mcp->valid) {
    float model[4] = {b.F[s], b.F[n + s] + mcp->vsys, b.F[2 * n + s], 1.0f / b.F[3 * n + s]};
    if (mcp->flux) {   // v = C1/C0, sigma^2 = C2/C0 - v^2, M/L = C3/C0
      const float iC0 = 1.0f / b.F[s], v = b.F[n + s] * iC0;
      model[1] = v + mcp->vsys;
      model[2] = sqrtf(fmaxf(b.F[2 * n + s] * iC0 - v * v, 0.f));
      model[3] = b.F[3 * n + s] * iC0;
    }
    float c2 = 0.f;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const float r = model[c] - g.data[c * n + s];
      c2 = fmaf(r * g.iv[c * n + s], r, c2);
    }
    v = c2;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < kPlainThreads / 32; ++k) t += red[k];
    atomicAdd(b.chi, t);
  }
}

__global__ void plain_logl(const GalDev* __restrict__ gal, const ModelConst* __restrict__ mcp, PlainBufs b,
                           double* __restrict__ logL) {
  *logL = mcp->valid ? -0.5 * (*b.chi) - gal->norm_const : -INFINITY;
}

inline int blocks_for(int n) { return (n + kPlainThreads - 1) / kPlainThreads; }

template <int NQ, int ND, int PSF>
cudaError_t chain(const float* theta, int P, int halo_kind, const GalDev* d_gal, const GalDev& h_gal, PlainBufs bufs,
                  double* logL, cudaStream_t st) {
  const int N = h_gal.W * h_gal.H, n = h_gal.nx * h_gal.ny;
  plain_decode<<<1, 1, 0, st>>>(theta, ND, halo_kind, d_gal, bufs.mc, bufs.chi);
  plain_coords<<<blocks_for(N), kPlainThreads, 0, st>>>(d_gal, bufs.mc, bufs);
  plain_bulge<NQ><<<blocks_for(N), kPlainThreads, 0, st>>>(d_gal, bufs.mc, bufs);
  plain_velocity<ND><<<blocks_for(N), kPlainThreads, 0, st>>>(d_gal, bufs.mc, bufs);
  plain_discs<ND><<<blocks_for(N), kPlainThreads, 0, st>>>(d_gal, bufs.mc, bufs);
  plain_combine<ND><<<blocks_for(N), kPlainThreads, 0, st>>>(d_gal, bufs.mc, bufs);
  plain_psf<PSF><<<blocks_for(n), kPlainThreads, 0, st>>>(d_gal, bufs.mc, bufs);
  plain_chi2<<<blocks_for(n), kPlainThreads, 0, st>>>(d_gal, bufs.mc, bufs);
  plain_logl<<<1, 1, 0, st>>>(d_gal, bufs.mc, bufs, logL);
  (void)P;
  return cudaGetLastError();
}

}  // namespace

size_t plain_scratch_bytes(int N, int n) {
  return sizeof(float) * ((size_t)N * 12 + (size_t)n * 4) + 256 + sizeof(ModelConst) + 64;
}

int plain_launches_per_row() { return 9; }

cudaError_t launch_plain_row(const float* theta, int P, int n_quad, int n_discs, int halo_kind, const GalDev* d_gal,
                             const GalDev& h_gal, void* scratch, double* logL, cudaStream_t st) {
  const int N = h_gal.W * h_gal.H, n = h_gal.nx * h_gal.ny;
  float* base = static_cast<float*>(scratch);
  PlainBufs b;
  b.R = base;
  b.r = b.R + N;
  b.cphi = b.r + N;
  b.Sb = b.cphi + N;
  b.Qb = b.Sb + N;
  b.vint2 = b.Qb + N;
  b.Sd0 = b.vint2 + N;
  b.Sd1 = b.Sd0 + N;
  b.f = b.Sd1 + N;                 // 4 N
  b.F = b.f + 4 * (size_t)N;       // 4 n
  char* tail = reinterpret_cast<char*>(b.F + 4 * (size_t)n);
  tail = reinterpret_cast<char*>(((uintptr_t)tail + 255) & ~(uintptr_t)255);
  b.chi = reinterpret_cast<double*>(tail);
  b.mc = reinterpret_cast<ModelConst*>(tail + 64);
  const int psf2d = h_gal.psf_kind;
#define BANG_CHAIN(NQ, ND)                                                                    \
  if (n_quad == NQ && n_discs == ND)                                                          \
    return psf2d ? chain<NQ, ND, 1>(theta, P, halo_kind, d_gal, h_gal, b, logL, st)           \
                 : chain<NQ, ND, 0>(theta, P, halo_kind, d_gal, h_gal, b, logL, st);
  BANG_CHAIN(64, 1) BANG_CHAIN(64, 2) BANG_CHAIN(128, 1) BANG_CHAIN(128, 2)
#undef BANG_CHAIN
  return cudaErrorInvalidValue;
}

BANG_DEFINE_FAULT_TAKER(take_fault_plain)

cudaError_t upload_nodes_plain(const float* cm1, const float* lc, const float* ws, const float* wq) {
  cudaError_t e = cudaMemcpyToSymbol(kNodeCm1, cm1, 192 * sizeof(float));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(kNodeLc, lc, 192 * sizeof(float));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(kNodeWs, ws, 192 * sizeof(float));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(kNodeWq, wq, 192 * sizeof(float));
  return e;
}

}  // namespace bang
