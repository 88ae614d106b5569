// Fused forward kernel: model evaluation -> PSF -> binning -> chi-square, one launch.
//
// Each block takes work items (row b, galaxy g, spaxel rows [j0, j1)) and streams the fine
// rows those spaxel rows depend on from top to bottom, G rows at a time:
//   1. every thread evaluates points of the G x W chunk (the per-point model, Sec. 2.1-2.4)
//      into a shared-memory stage of float4 (B, v, sigma, <L/M>);
//   2. the combined PSF (x) box filter (Eq. 21 followed by the os x os average) is applied:
//      separable Gaussian - one thread per spaxel column forms the horizontal sum of each
//      fine row and scatters it with the vertical weights into the accumulators of the
//      spaxel rows still open; Moffat - one thread per (open spaxel row, column) applies
//      the two-dimensional weights row by row;
//   3. a spaxel row whose last fine row has arrived is finished at once: residuals against
//      the data, chi-square in float32 per spaxel, float64 per thread, then a warp-shuffle
//      tree and a cross-warp float64 sum per work item.
// The fine field never leaves shared memory.  Only ceil((os + 2h) / os) spaxel rows of
// accumulators are live at any time.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <mutex>

#include "bang_device.cuh"
#include "bang_internal.h"

namespace bang {

namespace {

constexpr int kThreads = 256;

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

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Taps part, part + R, ... of the separable stencil's horizontal pass over one staged fine
// row (two packed lanes per float4); R a compile-time stride so that the loop unrolls.
template <int R>
__device__ __forceinline__ void hpass(const float2* taps, const float4* srow, int L, int part, float2& hxy,
                                      float2& hzw) {
  for (int k = part; k < L; k += R) {
    const float2 tw = taps[k];
    const float4 v = srow[k];
    hxy = __ffma2_rn(tw, make_float2(v.x, v.y), hxy);
    hzw = __ffma2_rn(tw, make_float2(v.z, v.w), hzw);
  }
}

// Residual terms of spaxel (i, j) of galaxy g from the filtered value F = (B, v, sigma, <L/M>)
// (flux-weighted mode: the filtered moments).  Writes the model maps / adjoint seeds when
// requested and d logL / d v_lam in lam_v.  Returns chi^2 of the four maps.
template <int MODE>
__device__ __forceinline__ float finish_spaxel(const GalDev& g, const ModelConst& m, float4 F, int i, int j,
                                               float* __restrict__ out, float& lam_v) {
  const int n = g.nx * g.ny;
  const int s = j * g.nx + i;
  if (!BANG_IN(s, n, kSiteFwdSpaxel)) {
    lam_v = 0.f;
    return 0.f;
  }
  float model[4];
  float v = 0.f, sig = 0.f, iC0 = 0.f;
  if (g.flux) {   // flux-weighted moments: v = C1/C0, sigma^2 = C2/C0 - v^2, M/L = C3/C0
    iC0 = 1.0f / F.x;
    v = F.y * iC0;
    sig = sqrtf(fmaxf(fmaf(F.z, iC0, -v * v), 0.f));
    model[0] = F.x;
    model[1] = v + m.vsys;
    model[2] = sig;
    model[3] = F.w * iC0;
  } else {        // each quantity convolved on its own; M/L = 1 / F_l
    model[0] = F.x;
    model[1] = F.y + m.vsys;
    model[2] = F.z;
    model[3] = 1.0f / F.w;
  }
  float chi = 0.f, lam[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const float iv = __ldg(g.iv + c * n + s);
    const float r = model[c] - __ldg(g.data + c * n + s);
    chi = fmaf(r * iv, r, chi);
    lam[c] = -r * iv;   // d logL / d model_c
    if (MODE == kModeMaps) out[c * n + s] = model[c];
  }
  lam_v = lam[1];       // the model velocity map is v + v_sys: d logL / d v_sys sums these
  if (MODE == kModeSeed) {   // d logL / dF_c for each filtered channel
    if (g.flux) {
      // dv = (dC1 - v dC0) / C0; dsigma = (dC2 - 2 v dC1 + (2 v^2 - C2/C0) dC0) / (2 sigma C0);
      // dML = (dC3 - ML dC0) / C0
      const float hs = sig > 0.f ? 0.5f * lam[2] / sig : 0.f;
      out[s] = lam[0] + iC0 * (-v * lam[1] + hs * (2.0f * v * v - F.z * iC0) - model[3] * lam[3]);
      out[n + s] = iC0 * (lam[1] - 2.0f * v * hs);
      out[2 * n + s] = iC0 * hs;
      out[3 * n + s] = iC0 * lam[3];
    } else {
#pragma unroll
      for (int c = 0; c < 3; ++c) out[c * n + s] = lam[c];
      out[3 * n + s] = -lam[3] * model[3] * model[3];
    }
  }
  return chi;
}

template <int NQ, int ND, int PSF, int MODE>
__global__ void __launch_bounds__(kThreads, MODE == kModeLogL2 ? 3 : 4) forward_kernel(FwdArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ ModelConst mc;
  __shared__ GalDev gs;
  __shared__ double red[kThreads / 32];

  const int tid = threadIdx.x;
  __shared__ int next_item;
  __shared__ int chunk_ctr[2];
  __shared__ float4 nodew[NQ / 2];
  __shared__ float2 tailc[kTailSet];
  const int lane = threadIdx.x & 31;
  // first item by block index, then either the next one from the shared counter (dynamic
  // scheduling, longest items first) or a fixed stride
  for (int it = blockIdx.x; it < a.n_items;) {
    const int item_id = a.order ? a.order[it] : it;
    if (!BANG_IN(item_id, a.n_items, kSiteFwdItem)) {
      BANG_NEXT_ITEM(it);
      continue;
    }
    WorkItem w;
    bool bad_gal = false;
    if (a.items) {
      w = a.items[item_id];
    } else {   // implicit item: band k of row b, the row's galaxy read on the device
      const int b = item_id / a.nb, k = item_id - b * a.nb;
      const int g = a.gal_idx ? __ldg(a.gal_idx + b) : 0;
      bad_gal = (unsigned)g >= (unsigned)a.n_gal;
      const int ny = bad_gal ? 0 : __ldg(&a.gals[g].ny);
      w = WorkItem{b, bad_gal ? 0 : g, (int)((long long)ny * k / a.nb), (int)((long long)ny * (k + 1) / a.nb)};
    }
    if (!BANG_IN(w.b, a.B, kSiteFwdRow) || !BANG_IN(w.g, a.n_gal, kSiteFwdGal)) {
      BANG_NEXT_ITEM(it);
      continue;
    }
    if (bad_gal || w.j1 <= w.j0) {   // a row without a galaxy, or an empty band of a galaxy with fewer rows
      if (tid == 0) {
        a.partial[item_id] = bad_gal ? __longlong_as_double(0x7ff8000000000000ll) : 0.0;
        if (MODE == kModeSeed) a.vsys_partial[item_id] = 0.0;
      }
      BANG_NEXT_ITEM(it);
      continue;
    }
    if (a.consts) {
      if (tid == 0) {
        gs = a.gals[w.g];
        mc = a.consts[w.b];
      }
    } else if (tid < 32) {   // warp 0 decodes the row (a few microseconds, once per item)
      if (tid == 0) gs = a.gals[w.g];
      decode_row_warp(a.theta + (size_t)w.b * a.P, ND, a.halo_kind, a.gals[w.g], true, a.l10k, tid, mc);
    }
    __syncthreads();
    // the gradient's forward pass leaves each row's constants for the adjoint (first band)
    if (a.consts_out && tid == 0 && w.j0 == 0) a.consts_out[w.b] = mc;
    const int L = gs.L, os = gs.os, W = gs.W, nx = gs.nx;
    const int NA = (L + os - 1) / os;                       // open spaxel rows
    const float inv_os = 1.0f / (float)os, inv_nx = 1.0f / (float)nx, inv_NA = 1.0f / (float)NA;
    // separable taps stored twice, (t, t): a 64-bit load gives the pair the packed
    // two-lane FMAs need; of the L x L two-dimensional taps only the Lq x Lq quadrant
    // (Lq = (L + 1) / 2): every two-dimensional window here is even in dx and dy about the
    // window's centre, and so is the os x os mean, so tap (cy, cx) equals tap (L-1-cy, cx)
    // and (cy, L-1-cx)
    float2* taps = reinterpret_cast<float2*>(smem_raw);
    float* taps2d = reinterpret_cast<float*>(smem_raw);
    const int Lq = (L + 1) / 2;
    const int ntaps = PSF == 0 ? L : Lq * Lq;
    float4* acc = reinterpret_cast<float4*>(smem_raw + (((size_t)ntaps * (PSF == 0 ? 8 : 4) + 15) / 16) * 16);
    float4* stage = acc + (size_t)NA * nx;
    // fine rows per chunk: a.G, or for a narrower galaxy of a mixed batch the rows that
    // hold the widest galaxy's a.chunk_pts points, as far as the launch's shared memory
    // goes (fewer barriers, and whole 64-point grabs for every warp between them)
    int Gc = a.G;
    if (a.chunk_pts > 0) {
      const size_t used = (size_t)(reinterpret_cast<unsigned char*>(stage) - smem_raw) +
                          (a.tables ? sizeof(float) * (size_t)(kTabHdr + 4 * a.table_T) : 0);
      const size_t dyn = dynamic_smem_bytes();
      const int cap = dyn > used ? (int)((dyn - used) / (2 * sizeof(float4) * (size_t)W)) : 0;
      Gc = max(a.G, min(a.chunk_pts / W, cap));
    }
    float* tab = a.tables ? reinterpret_cast<float*>(stage + 2 * (size_t)Gc * W) : nullptr;
    float* out = nullptr;
    const int64_t ooff = a.out_off ? a.out_off[w.b] : (int64_t)w.b * a.out_stride;
    if (MODE == kModeMaps) out = a.maps + ooff;
    if (MODE == kModeSeed) out = a.seed + ooff;
    // checked build: the layout fits the launch's shared memory, a fine row holds every
    // stencil read, the item's spaxel rows, output block and radial table are in range
    if (!BANG_IN((tab ? reinterpret_cast<const unsigned char*>(tab + kTabHdr + 4 * a.table_T)
                      : reinterpret_cast<const unsigned char*>(stage + 2 * (size_t)Gc * W)) - smem_raw - 1,
                 dynamic_smem_bytes(), kSiteFwdSmem) ||
        !BANG_IN((nx - 1) * os + L - 1, W, kSiteFwdStencil) || !BANG_IN(w.j0, w.j1, kSiteFwdSpaxel) ||
        !BANG_IN(w.j1 - 1, gs.ny, kSiteFwdSpaxel) ||
        ((MODE == kModeMaps || MODE == kModeSeed) && !BANG_IN(ooff + 4ll * nx * gs.ny - 1, a.out_total, kSiteFwdOut)) ||
        (tab && !BANG_IN((long long)w.b * a.table_stride + kTabHdr + 4 * a.table_T - 1,
                         (long long)a.B * a.table_stride, kSiteFwdTable))) {
      BANG_NEXT_ITEM(it);
      continue;
    }

    if (!mc.valid) {
      if (MODE == kModeMaps) {
        for (int s = tid; s < 4 * (w.j1 - w.j0) * nx; s += kThreads) {
          const int c = s / ((w.j1 - w.j0) * nx), rem = s - c * (w.j1 - w.j0) * nx;
          out[c * nx * gs.ny + w.j0 * nx + rem] = __int_as_float(0x7fc00000);
        }
      }
      if (MODE == kModeSeed) {
        for (int s = tid; s < 4 * (w.j1 - w.j0) * nx; s += kThreads) {
          const int c = s / ((w.j1 - w.j0) * nx), rem = s - c * (w.j1 - w.j0) * nx;
          out[c * nx * gs.ny + w.j0 * nx + rem] = 0.f;
        }
      }
      if (tid == 0) {
        a.partial[item_id] = __longlong_as_double(0x7ff8000000000000ll);
        if (MODE == kModeSeed) a.vsys_partial[item_id] = 0.0;
      }
      BANG_NEXT_ITEM(it);
      continue;
    }

    for (int t = tid; t < ntaps; t += kThreads) {
      if (PSF == 0) {
        const float tv = __ldg(gs.taps + t);
        taps[t] = make_float2(tv, tv);
      } else {
        const int ty = t / Lq, tx = t - ty * Lq;
        taps2d[t] = __ldg(gs.taps + ty * L + tx);
      }
    }
    for (int t = tid; t < NA * nx; t += kThreads) acc[t] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (tab) {   // this row's radial table: header, values and log-ratios of Sigma and Q
      const float* src = a.tables + (size_t)w.b * a.table_stride;
      const int nt = kTabHdr + 4 * a.table_T;
      for (int t = tid; t < nt; t += kThreads) tab[t] = __ldg(src + t);
    }
    if (tid < 2) chunk_ctr[tid] = 0;
    if (!tab && !mc.bulge_fit) {
      fill_node_pairs<NQ>(mc, nodew, tid, kThreads);
      if (tid < 32) fill_tail_coeffs<NQ>(mc, tailc, tid);
    }
    __syncthreads();

    double chi_thread = 0.0, vsys_thread = 0.0;
    const int y_begin = w.j0 * os;
    const int y_end = (w.j1 - 1) * os + L;                   // exclusive
    const int nchunks = (y_end - y_begin + Gc - 1) / Gc;
    const float pk = gs.pitch_kpa;
    const float inv_W = 1.0f / (float)W;

    // Evaluation of chunk c (Gc fine rows) into stage buffer c & 1.  Warps take 32 points
    // at a time from the chunk's shared counter, so warps that are busy with the stencil
    // of the previous chunk simply take fewer points.
    auto eval_chunk = [&](int c) {
      const int y0 = y_begin + c * Gc;
      const int npts = min(Gc, y_end - y0) * W;
      float4* st = stage + (size_t)(c & 1) * Gc * W;
      if (!BANG_IN(npts, Gc * W + 1, kSiteFwdStage)) return;
      if constexpr (MODE == kModeLogL2) {   // two points per thread: their independent chains interleave
        for (;;) {
          int base = 0;
          if (lane == 0) base = atomicAdd(&chunk_ctr[c & 1], 64);
          base = __shfl_sync(0xffffffffu, base, 0);
          if (base >= npts) break;
          const int pA = base + lane;
          if (pA < npts) {
            const int pB = min(base + 32 + lane, npts - 1);   // a lane past the end repeats the last point
            const int grA = __float2int_rz(((float)pA + 0.5f) * inv_W);
            const int grB = __float2int_rz(((float)pB + 0.5f) * inv_W);
            const float XA = fmaf((float)(pA - grA * W), pk, mc.X0), YA = fmaf((float)(y0 + grA), pk, mc.Y0);
            const float XB = fmaf((float)(pB - grB * W), pk, mc.X0), YB = fmaf((float)(y0 + grB), pk, mc.Y0);
            const float4 oA = eval_point<NQ, ND>(mc, XA, YA, tab, a.table_T, nodew, tailc);
            const float4 oB = eval_point<NQ, ND>(mc, XB, YB, tab, a.table_T, nodew, tailc);
            st[pA] = oA;
            if (base + 32 + lane < npts) st[pB] = oB;
          }
        }
      } else {
        for (;;) {
          int base = 0;
          if (lane == 0) base = atomicAdd(&chunk_ctr[c & 1], 32);
          base = __shfl_sync(0xffffffffu, base, 0);
          if (base >= npts) break;
          const int p = base + lane;
          if (p < npts) {
            const int gr = __float2int_rz(((float)p + 0.5f) * inv_W);   // p + 1/2 is never a multiple of W
            const int qx = p - gr * W;
            const float X = fmaf((float)qx, pk, mc.X0);
            const float Y = fmaf((float)(y0 + gr), pk, mc.Y0);
            st[p] = eval_point<NQ, ND>(mc, X, Y, tab, a.table_T, nodew, tailc);
          }
        }
      }
    };

    eval_chunk(0);
    __syncthreads();
    for (int c = 0; c < nchunks; ++c) {
      // stage c & 1 holds chunk c; its counter is free again (next used by chunk c + 2)
      if (tid == 0) chunk_ctr[c & 1] = 0;
      const int y0 = y_begin + c * Gc;
      const int G = min(Gc, y_end - y0);
      const float4* stage_c = stage + (size_t)(c & 1) * Gc * W;
      // filter chunk c into the open spaxel rows; finish the rows that complete
      if (PSF == 0) {
        // With a.col_lanes, r lanes per spaxel column (a power of two, r nx <= kThreads,
        // r <= 8) split the horizontal pass's taps (k = part, part + r, ...) and a fixed
        // shuffle tree adds the parts, so that a column's dependent FMA chain is L / r long;
        // lane part 0 then scatters into the open spaxel rows (otherwise r = 1: one thread
        // per column).  Whole warps run the loop (the shuffles).  The autotuner chooses
        // for the one-point forms: the uneven batch gains 4.3% with it, the gradient's
        // forward pass loses; in the two-point form it cost the batched workload 1.7% even
        // switched off, so that form has none.
        int lr = 0;
        if constexpr (MODE != kModeLogL2) {   // the two-point form keeps one thread per column
          if (a.col_lanes)
            while (lr < 3 && (2 << lr) * nx <= kThreads) ++lr;
        }
        const int r = 1 << lr, nu = nx << lr, nu_w = (nu + 31) & ~31;
        for (int u = tid; u < nu_w; u += kThreads) {
          const bool act = u < nu;
          const int i = act ? u >> lr : 0, part = u & (r - 1);
          for (int gr = 0; gr < G; ++gr) {
            const int y = y0 + gr;
            const float4* srow = stage_c + gr * W + i * os;
            float2 hxy = make_float2(0.f, 0.f), hzw = hxy;   // (B, v) and (sigma, <L/M>) lanes
            if (act) {
              if (lr == 0) hpass<1>(taps, srow, L, part, hxy, hzw);
              else if (lr == 1) hpass<2>(taps, srow, L, part, hxy, hzw);
              else if (lr == 2) hpass<4>(taps, srow, L, part, hxy, hzw);
              else hpass<8>(taps, srow, L, part, hxy, hzw);
            }
            for (int o = 1; o < r; o <<= 1) {
              hxy.x += __shfl_xor_sync(0xffffffffu, hxy.x, o);
              hxy.y += __shfl_xor_sync(0xffffffffu, hxy.y, o);
              hzw.x += __shfl_xor_sync(0xffffffffu, hzw.x, o);
              hzw.y += __shfl_xor_sync(0xffffffffu, hzw.y, o);
            }
            if (!act || part != 0) continue;
            int jlo = y - L + 1 <= 0 ? 0 : floor_div(y - L + os, inv_os);  // ceil((y - L + 1) / os)
            jlo = max(jlo, w.j0);
            const int jhi = min(floor_div(y, inv_os), w.j1 - 1);
            int ring = jlo - NA * floor_div(jlo, inv_NA);         // jlo % NA, then kept in step
            for (int j = jlo; j <= jhi; ++j) {
              if (BANG_IN(y - j * os, L, kSiteFwdTap)) {
                const float2 tv = taps[y - j * os];
                float4& A = acc[ring * nx + i];
                const float2 axy = __ffma2_rn(tv, hxy, make_float2(A.x, A.y));
                const float2 azw = __ffma2_rn(tv, hzw, make_float2(A.z, A.w));
                A = make_float4(axy.x, axy.y, azw.x, azw.y);
              }
              ring = ring + 1 == NA ? 0 : ring + 1;
            }
            const int yl = y - L + 1;                             // spaxel row ending here
            const int jl = yl >= 0 ? floor_div(yl, inv_os) : -1;
            if (yl >= 0 && jl * os == yl) {
              const int j = jl;
              if (j >= w.j0 && j < w.j1) {
                float4& A = acc[(j - NA * floor_div(j, inv_NA)) * nx + i];
                float lam_v;
                chi_thread += (double)finish_spaxel<MODE>(gs, mc, A, i, j, out, lam_v);
                if (MODE == kModeSeed) vsys_thread += (double)lam_v;
                A = make_float4(0.f, 0.f, 0.f, 0.f);
              }
            }
          }
        }
      } else {
        // open spaxel rows touched by this chunk
        const int ylast = y0 + G - 1;
        int jlo = y0 - L + 1 <= 0 ? 0 : (y0 - L + os) / os;
        jlo = max(jlo, w.j0);
        const int jhi = min(ylast / os, w.j1 - 1);
        const int nj = jhi - jlo + 1;
        for (int t = tid; t < nj * nx; t += kThreads) {
          const int tj = floor_div(t, inv_nx);
          const int j = jlo + tj;
          const int i = t - tj * nx;
          const int rj = j - NA * floor_div(j, inv_NA);           // j % NA
          float4 A = acc[rj * nx + i];
          const int ga = max(0, j * os - y0);
          const int gb = min(G - 1, j * os + L - 1 - y0);
          for (int gr = ga; gr <= gb; ++gr) {
            const int cy = y0 + gr - j * os;
            if (!BANG_IN(cy, L, kSiteFwdTap)) continue;
            const float* wrow = taps2d + min(cy, L - 1 - cy) * Lq;
            const float4* srow = stage_c + gr * W + i * os;
            float2 axy = make_float2(A.x, A.y), azw = make_float2(A.z, A.w);
            // columns k and L-1-k share a tap: their points are summed first
            for (int k = 0; k < L / 2; ++k) {
              const float2 tw = make_float2(wrow[k], wrow[k]);
              const float4 v = srow[k], u = srow[L - 1 - k];
              axy = __ffma2_rn(tw, __fadd2_rn(make_float2(v.x, v.y), make_float2(u.x, u.y)), axy);
              azw = __ffma2_rn(tw, __fadd2_rn(make_float2(v.z, v.w), make_float2(u.z, u.w)), azw);
            }
            if (L & 1) {
              const float2 tw = make_float2(wrow[L / 2], wrow[L / 2]);
              const float4 v = srow[L / 2];
              axy = __ffma2_rn(tw, make_float2(v.x, v.y), axy);
              azw = __ffma2_rn(tw, make_float2(v.z, v.w), azw);
            }
            A = make_float4(axy.x, axy.y, azw.x, azw.y);
          }
          if (j * os + L - 1 <= ylast) {
            float lam_v;
            chi_thread += (double)finish_spaxel<MODE>(gs, mc, A, i, j, out, lam_v);
            if (MODE == kModeSeed) vsys_thread += (double)lam_v;
            A = make_float4(0.f, 0.f, 0.f, 0.f);
          }
          acc[rj * nx + i] = A;
        }
      }
      // meanwhile (and after its share of the stencil) every warp evaluates chunk c + 1
      if (c + 1 < nchunks) eval_chunk(c + 1);
      __syncthreads();
    }

    // float64 reduction of the work item's chi^2: warp shuffles, then across warps
    double v = warp_sum(chi_thread);
    if ((tid & 31) == 0) red[tid >> 5] = v;
    __syncthreads();
    if (tid == 0) {
      double s = 0.0;
      for (int k = 0; k < kThreads / 32; ++k) s += red[k];
      a.partial[item_id] = s;
    }
    if (MODE == kModeSeed) {   // the item's share of d logL / d v_sys (summed per row in fixed order later)
      __syncthreads();         // red is reused
      const double u = warp_sum(vsys_thread);
      if ((tid & 31) == 0) red[tid >> 5] = u;
      __syncthreads();
      if (tid == 0) {
        double s = 0.0;
        for (int k = 0; k < kThreads / 32; ++k) s += red[k];
        a.vsys_partial[item_id] = s;
      }
    }
    BANG_NEXT_ITEM(it);
  }
}

// One warp per row (decode_row_warp): the rows' constants ahead of the radial tables, which
// are built from them.
__global__ void decode_kernel(const float* __restrict__ theta, int P, int nd, int halo_kind,
                              const GalDev* __restrict__ gals, const int* __restrict__ row_g, int n_gal, int B,
                              double l10k, ModelConst* __restrict__ out) {
  const int b = (int)((blockIdx.x * (unsigned)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (b >= B) return;   // whole warps: b is uniform across the warp
  const float* th = theta + (size_t)b * P;
  const int g = row_g ? row_g[b] : 0;
  const bool gal_ok = (unsigned)g < (unsigned)n_gal && BANG_IN(g, n_gal, kSiteDecodeGal);
  const GalDev& gal = gals[gal_ok ? g : 0];
  ModelConst m;
  decode_row_warp(th, nd, halo_kind, gal, gal_ok, l10k, lane, m);
  if (lane == 0) out[b] = m;
}

// logL[b] = -chi^2/2 - const from the per-item partial sums (items of row b are contiguous).
// row_first NULL: the items of row b are [b nb, (b + 1) nb); row_g NULL: galaxy 0.  With
// check_gal, a row whose galaxy index is outside [0, n_gal) gets NaN (its items were skipped).
__global__ void finalize_kernel(const double* __restrict__ partial, const int* __restrict__ row_first,
                                const int* __restrict__ row_g, const GalDev* __restrict__ gals, int B, int n_items,
                                int n_gal, int nb, int check_gal, double* __restrict__ logL) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const int g = row_g ? row_g[b] : 0;
  if (check_gal && (unsigned)g >= (unsigned)n_gal) {
    logL[b] = __longlong_as_double(0x7ff8000000000000ll);
    return;
  }
  double s = 0.0;
  bool bad = false;
  const int k0 = row_first ? row_first[b] : b * nb, k1 = row_first ? row_first[b + 1] : (b + 1) * nb;
  for (int k = k0; k < k1; ++k) {
    if (!BANG_IN(k, n_items, kSiteFinalizeItem)) continue;
    const double v = partial[k];
    bad |= isnan(v);
    s += v;
  }
  if (!BANG_IN(g, n_gal, kSiteDecodeGal)) return;
  logL[b] = bad ? -INFINITY : -0.5 * s - gals[g].norm_const;
}

// Execution order of implicit work items (nb per row), longest first: a counting sort of the
// rows by the rank of their galaxy's item cost (gal_rank[g] in [0, n_rank), 0 = costliest),
// the items of a row kept together.  Rows without a valid galaxy go last.  One block; the
// order within a rank follows the atomics (it changes which block runs an item, not any
// result: every item writes its own partial sums).
constexpr int kOrderThreads = 1024;
__global__ void __launch_bounds__(kOrderThreads) order_kernel(const int* __restrict__ gal_idx,
                                                              const int* __restrict__ gal_rank, int n_gal, int n_rank,
                                                              int B, int nb, int* __restrict__ order) {
  extern __shared__ int cnt[];   // n_rank + 1 counters
  __shared__ int part[kOrderThreads];
  const int tid = threadIdx.x, nr = n_rank + 1;
  for (int r = tid; r < nr; r += kOrderThreads) cnt[r] = 0;
  __syncthreads();
  auto rank_of = [&](int b) {
    const int g = gal_idx ? gal_idx[b] : 0;
    return (unsigned)g < (unsigned)n_gal ? gal_rank[g] : n_rank;
  };
  for (int b = tid; b < B; b += kOrderThreads) atomicAdd(&cnt[rank_of(b)], nb);
  __syncthreads();
  // exclusive scan of the counters: each thread a contiguous chunk, then the chunk totals
  const int per = (nr + kOrderThreads - 1) / kOrderThreads;
  const int r0 = min(nr, tid * per), r1 = min(nr, r0 + per);
  int local = 0;
  for (int r = r0; r < r1; ++r) local += cnt[r];
  part[tid] = local;
  __syncthreads();
  for (int off = 1; off < kOrderThreads; off <<= 1) {   // Hillis-Steele inclusive scan of part
    const int v = tid >= off ? part[tid - off] : 0;
    __syncthreads();
    part[tid] += v;
    __syncthreads();
  }
  int run = part[tid] - local;
  for (int r = r0; r < r1; ++r) {
    const int c = cnt[r];
    cnt[r] = run;
    run += c;
  }
  __syncthreads();
  for (int b = tid; b < B; b += kOrderThreads) {
    const int pos = atomicAdd(&cnt[rank_of(b)], nb);
    for (int k = 0; k < nb; ++k) order[pos + k] = b * nb + k;
  }
}

template <int NQ, int ND, int PSF, int MODE>
cudaError_t launch_t(const FwdArgs& a, int grid, size_t smem, cudaStream_t st) {
  forward_kernel<NQ, ND, PSF, MODE><<<grid, kThreads, smem, st>>>(a);
  return cudaGetLastError();
}

template <int NQ, int ND, int PSF>
cudaError_t launch_mode(const FwdArgs& a, int mode, int grid, size_t smem, cudaStream_t st) {
  switch (mode) {
    case kModeLogL: return launch_t<NQ, ND, PSF, kModeLogL>(a, grid, smem, st);
    case kModeLogL2: return launch_t<NQ, ND, PSF, kModeLogL2>(a, grid, smem, st);
    case kModeMaps: return launch_t<NQ, ND, PSF, kModeMaps>(a, grid, smem, st);
    default: return launch_t<NQ, ND, PSF, kModeSeed>(a, grid, smem, st);
  }
}

template <int NQ, int ND>
cudaError_t launch_psf(const FwdArgs& a, int psf2d, int mode, int grid, size_t smem, cudaStream_t st) {
  return psf2d ? launch_mode<NQ, ND, 1>(a, mode, grid, smem, st) : launch_mode<NQ, ND, 0>(a, mode, grid, smem, st);
}

}  // namespace

int forward_threads() { return kThreads; }

size_t forward_smem_bytes(int L, int os, int nx, int W, int G, int psf2d, int table_T) {
  const int ntaps = psf2d ? ((L + 1) / 2) * ((L + 1) / 2) : L;   // two-dimensional: the quadrant
  const int NA = (L + os - 1) / os;
  return (((size_t)ntaps * (psf2d ? 4 : 8) + 15) / 16) * 16 + (size_t)NA * nx * 16 + 2 * (size_t)G * W * 16 +
         (table_T > 0 ? sizeof(float) * (size_t)(kTabHdr + 4 * table_T) : 0);
}

const void* forward_kernel_ptr(int n_quad, int n_discs, int psf2d, int mode) {
#define BANG_PICK(NQ, ND, PSF)                                                    \
  if (n_quad == NQ && n_discs == ND && psf2d == PSF) {                            \
    if (mode == kModeLogL) return (const void*)forward_kernel<NQ, ND, PSF, kModeLogL>; \
    if (mode == kModeLogL2) return (const void*)forward_kernel<NQ, ND, PSF, kModeLogL2>; \
    if (mode == kModeMaps) return (const void*)forward_kernel<NQ, ND, PSF, kModeMaps>; \
    return (const void*)forward_kernel<NQ, ND, PSF, kModeSeed>;                   \
  }
  BANG_PICK(64, 1, 0) BANG_PICK(64, 1, 1) BANG_PICK(64, 2, 0) BANG_PICK(64, 2, 1)
  BANG_PICK(128, 1, 0) BANG_PICK(128, 1, 1) BANG_PICK(128, 2, 0) BANG_PICK(128, 2, 1)
#undef BANG_PICK
  return nullptr;
}

cudaError_t launch_forward(const FwdArgs& a, int n_quad, int n_discs, int psf2d, int mode, int grid, size_t smem,
                           cudaStream_t st) {
  if (n_quad == 64) {
    return n_discs == 2 ? launch_psf<64, 2>(a, psf2d, mode, grid, smem, st)
                        : launch_psf<64, 1>(a, psf2d, mode, grid, smem, st);
  }
  return n_discs == 2 ? launch_psf<128, 2>(a, psf2d, mode, grid, smem, st)
                      : launch_psf<128, 1>(a, psf2d, mode, grid, smem, st);
}

size_t model_const_bytes() { return sizeof(ModelConst); }

double decode_l10k_host() { return std::log10(3.0 / (4.0 * kPi * 200.0 * kRhoCrit)); }

cudaError_t launch_decode(const float* theta, int P, int n_discs, int halo_kind, const GalDev* gals, const int* row_g,
                          int n_gal, int B, ModelConst* out, cudaStream_t st) {
  constexpr int kRowsPerBlock = 4;   // 4 warps of 32 lanes, one row each
  const double l10k = decode_l10k_host();
  decode_kernel<<<(B + kRowsPerBlock - 1) / kRowsPerBlock, 32 * kRowsPerBlock, 0, st>>>(
      theta, P, n_discs, halo_kind, gals, row_g, n_gal, B, l10k, out);
  return cudaGetLastError();
}

// Rows of several grids of one galaxy: theta_x[b n + k] = theta[b] (expand), and
// logL[b] = sum_k logL_x[b n + k], grad[b] = sum_k grad_x[b n + k] (sum).
__global__ void expand_rows_kernel(const float* __restrict__ theta, int P, int B, int n, float* __restrict__ theta_x) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t total = (int64_t)B * n * P;
  if (t >= total) return;
  const int64_t row = t / P, p = t - row * P;
  theta_x[t] = theta[(row / n) * P + p];
}

__global__ void sum_rows_kernel(const double* __restrict__ logL_x, const float* __restrict__ grad_x, int P, int B, int n,
                                double* __restrict__ logL, float* __restrict__ grad) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  double s = 0.0;
  for (int k = 0; k < n; ++k) s += logL_x[(size_t)b * n + k];
  logL[b] = s;
  if (!grad) return;
  for (int p = 0; p < P; ++p) {
    double g = 0.0;
    for (int k = 0; k < n; ++k) g += (double)grad_x[((size_t)b * n + k) * P + p];
    grad[(size_t)b * P + p] = (float)g;
  }
}

cudaError_t launch_expand_rows(const float* theta, int P, int B, int n, float* theta_x, cudaStream_t st) {
  const int64_t total = (int64_t)B * n * P;
  expand_rows_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(theta, P, B, n, theta_x);
  return cudaGetLastError();
}

cudaError_t launch_sum_rows(const double* logL_x, const float* grad_x, int P, int B, int n, double* logL, float* grad,
                            cudaStream_t st) {
  sum_rows_kernel<<<(B + 127) / 128, 128, 0, st>>>(logL_x, grad_x, P, B, n, logL, grad);
  return cudaGetLastError();
}

cudaError_t launch_finalize(const double* partial, const int* row_first, const int* row_g, const GalDev* gals, int B,
                            int n_items, int n_gal, double* logL, cudaStream_t st, int nb, int check_gal) {
  finalize_kernel<<<(B + 127) / 128, 128, 0, st>>>(partial, row_first, row_g, gals, B, n_items, n_gal, nb, check_gal,
                                                   logL);
  return cudaGetLastError();
}

cudaError_t launch_order(const int* gal_idx, const int* gal_rank, int n_gal, int n_rank, int B, int nb, int* order,
                         cudaStream_t st) {
  order_kernel<<<1, kOrderThreads, sizeof(int) * (size_t)(n_rank + 1), st>>>(gal_idx, gal_rank, n_gal, n_rank, B, nb,
                                                                            order);
  return cudaGetLastError();
}

BANG_DEFINE_FAULT_TAKER(take_fault_forward)

namespace {
__global__ void check_selftest_kernel(long long i, long long n) { (void)BANG_IN(i, n, kSiteSelftest); }
}  // namespace

// One check of i against n on the device: in the checked build an out-of-range i is
// recorded as a fault of the selftest site; nothing is read or written at i.
cudaError_t launch_check_selftest(long long i, long long n, cudaStream_t st) {
  check_selftest_kernel<<<1, 1, 0, st>>>(i, n);
  return cudaGetLastError();
}

cudaError_t upload_nodes_forward(const float* cm1, const float* lc, const float* ws, const float* wq) {
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

// ============================================================================================
// bang_loglike_batch_noalloc: the forward launch with its scratch in a fixed device array.
//
// bang_loglike_batch keeps per-batch scratch (the work-item table and the per-item chi^2
// partial sums) in device memory that it allocates the first time it sees a batch shape.
// This variant allocates nothing: the same scratch lives in g_noalloc_scratch, a file-scope
// __device__ array of kNoAllocScratchBytes that every device which loads the library holds
// until the process exits.  Host code cannot use the array's name as a device address (it
// names a host-side shadow), so the address is looked up once per device with
// cudaGetSymbolAddress, with that device current, and passed to the kernels.
namespace bang {
namespace {

constexpr int kNoAllocMaxRows = 32768;
constexpr size_t align256(size_t x) { return (x + 255) / 256 * 256; }
constexpr size_t kNaItemsOff = 0;
constexpr size_t kNaPartialOff = align256(kNaItemsOff + sizeof(WorkItem) * kNoAllocMaxRows);
constexpr size_t kNaRowFirstOff = align256(kNaPartialOff + sizeof(double) * kNoAllocMaxRows);
constexpr size_t kNaRowGOff = align256(kNaRowFirstOff + sizeof(int) * (kNoAllocMaxRows + 1));
constexpr size_t kNaGalIdxOff = align256(kNaRowGOff + sizeof(int) * kNoAllocMaxRows);
constexpr size_t kNoAllocScratchBytes = align256(kNaGalIdxOff + sizeof(int) * kNoAllocMaxRows);   // ~1.2 MB

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kNaMaxDevices = 64;
std::mutex g_na_mu;
unsigned char* g_na_ptr[kNaMaxDevices] = {};

// One work item per row (whole spaxel grid), row b against galaxy gal[b] (0 when gal is NULL).
__global__ void noalloc_items_kernel(const int* __restrict__ gal, const GalDev* __restrict__ gals, int B,
                                     WorkItem* __restrict__ items, int* __restrict__ row_first,
                                     int* __restrict__ row_g) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const int g = gal ? gal[b] : 0;
  items[b] = WorkItem{b, g, 0, gals[g].ny};
  row_first[b] = b;
  row_g[b] = g;
  if (b == B - 1) row_first[B] = B;
}

}  // namespace
}  // namespace bang

extern "C" bang_status bang_loglike_batch_noalloc(bang_model* m, const float* theta, const int32_t* gal_idx, int B,
                                                  double* logL, void* stream) {
  using namespace bang;
  NvtxRange nvtx("bang_loglike_batch_noalloc");
  ModelView v;
  if (!model_view(m, &v)) return set_error(BANG_E_INVALID_ARG, "null model");
  if (v.bulge_table)
    return set_error(BANG_E_UNSUPPORTED, "bang_loglike_batch_noalloc: no radial-table mode (bulge_table)");
  if (!theta || !logL) return set_error(BANG_E_INVALID_ARG, "theta or logL is null");
  if (B < 1 || B > kNoAllocMaxRows)
    return set_error(BANG_E_INVALID_ARG, "bang_loglike_batch_noalloc: B = %d outside [1, %d] (fixed scratch of %zu bytes)",
                     B, kNoAllocMaxRows, kNoAllocScratchBytes);
  if (v.device < 0 || v.device >= kNaMaxDevices) return set_error(BANG_E_UNSUPPORTED, "device index %d", v.device);
  cudaError_t e = cudaSetDevice(v.device);
  if (e != cudaSuccess) return set_error(BANG_E_CUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
  for (const void* ptr : {(const void*)theta, (const void*)logL}) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess || at.type != cudaMemoryTypeDevice) {
      cudaGetLastError();
      return set_error(BANG_E_INVALID_ARG, "bang_loglike_batch_noalloc: theta and logL must be device memory");
    }
  }
  if (gal_idx) {   // this entry point schedules on the host: gal_idx must be host memory
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, gal_idx) != cudaSuccess) {
      cudaGetLastError();
    } else if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) {
      return set_error(BANG_E_INVALID_ARG, "bang_loglike_batch_noalloc: gal_idx must be host memory");
    }
  }
  int psf2d = -1;
  size_t smem = 0;
  for (int b = 0; b < B; ++b) {
    const int g = gal_idx ? gal_idx[b] : 0;
    if (g < 0 || g >= v.n_gal) return set_error(BANG_E_INVALID_ARG, "gal_idx[%d] = %d out of range", b, g);
    const GalDev& G = v.h_gals[g];
    if (psf2d < 0) psf2d = G.psf_kind;
    if (G.psf_kind != psf2d) return set_error(BANG_E_UNSUPPORTED, "a batch mixes Gaussian and Moffat PSF galaxies");
    smem = std::max(smem, forward_smem_bytes(G.L, G.os, G.nx, G.W, 4, psf2d));
    if (!gal_idx) break;
  }
  int rows_per_step = 4;
  const void* kp = forward_kernel_ptr(v.n_quad, v.n_discs, psf2d, kModeLogL);
  cudaFuncAttributes fa;
  if ((e = cudaFuncGetAttributes(&fa, kp)) != cudaSuccess)
    return set_error(BANG_E_CUDA, "cudaFuncGetAttributes: %s", cudaGetErrorString(e));
  if (smem + fa.sharedSizeBytes > (size_t)v.smem_optin) {
    rows_per_step = 1;
    smem = 0;
    for (int b = 0; b < B; ++b) {
      const GalDev& G = v.h_gals[gal_idx ? gal_idx[b] : 0];
      smem = std::max(smem, forward_smem_bytes(G.L, G.os, G.nx, G.W, 1, psf2d));
      if (!gal_idx) break;
    }
    if (smem + fa.sharedSizeBytes > (size_t)v.smem_optin)
      return set_error(BANG_E_UNSUPPORTED, "galaxy too large for one block's shared memory");
  }

  // set-up, once per device: the device address of the scratch array
  unsigned char* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_na_mu);
    if (!g_na_ptr[v.device]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p)
        return set_error(BANG_E_CUDA, "cudaGetSymbolAddress(g_noalloc_scratch): %s", cudaGetErrorString(e));
      g_na_ptr[v.device] = static_cast<unsigned char*>(p);
    }
    scratch = g_na_ptr[v.device];
  }
  if ((e = cudaFuncSetAttribute(kp, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                v.smem_optin - (int)fa.sharedSizeBytes)) != cudaSuccess)
    return set_error(BANG_E_CUDA, "cudaFuncSetAttribute: %s", cudaGetErrorString(e));
  int per_sm = 0;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kp, forward_threads(), smem)) != cudaSuccess ||
      per_sm < 1)
    return set_error(BANG_E_CUDA, "occupancy query failed");

  cudaStream_t st = static_cast<cudaStream_t>(stream);
  WorkItem* items = reinterpret_cast<WorkItem*>(scratch + kNaItemsOff);
  double* partial = reinterpret_cast<double*>(scratch + kNaPartialOff);
  int* row_first = reinterpret_cast<int*>(scratch + kNaRowFirstOff);
  int* row_g = reinterpret_cast<int*>(scratch + kNaRowGOff);
  int* gal_dev = nullptr;
  if (gal_idx) {
    gal_dev = reinterpret_cast<int*>(scratch + kNaGalIdxOff);
    if ((e = cudaMemcpyAsync(gal_dev, gal_idx, sizeof(int) * (size_t)B, cudaMemcpyHostToDevice, st)) != cudaSuccess)
      return set_error(BANG_E_CUDA, "copy of gal_idx: %s", cudaGetErrorString(e));
  }
  noalloc_items_kernel<<<(B + 127) / 128, 128, 0, st>>>(gal_dev, v.d_gals, B, items, row_first, row_g);
  if ((e = cudaGetLastError()) != cudaSuccess) return set_error(BANG_E_CUDA, "item kernel: %s", cudaGetErrorString(e));
  FwdArgs a{};
  a.theta = theta;
  a.P = v.P;
  a.halo_kind = v.halo_kind;
  a.gals = v.d_gals;
  a.items = items;
  a.order = nullptr;
  a.n_items = B;
  a.G = rows_per_step;
  a.partial = partial;
  a.out_off = nullptr;
  a.l10k = decode_l10k_host();
  a.B = B;
  a.n_gal = v.n_gal;
  const int grid = std::min(B, per_sm * v.num_sms);
  if ((e = launch_forward(a, v.n_quad, v.n_discs, psf2d, kModeLogL, grid, smem, st)) != cudaSuccess)
    return set_error(BANG_E_CUDA, "forward kernel: %s", cudaGetErrorString(e));
  if ((e = launch_finalize(partial, row_first, row_g, v.d_gals, B, B, v.n_gal, logL, st)) != cudaSuccess)
    return set_error(BANG_E_CUDA, "finalize kernel: %s", cudaGetErrorString(e));
  return check_faults(st);
}
