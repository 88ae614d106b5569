// Host side of libbang.so: the C ABI of include/bang.h.
//
// bang_model_create copies every galaxy's data to the device once (App. A allocates and
// loads the data a single time), builds the combined PSF (x) box-filter taps of Eq. 21 and
// the radial quadrature tables.  Each compute call turns the rows of a batch into a table of work
// items (row, galaxy, band of spaxel rows), cached per batch shape, and runs one persistent
// launch over it, replayed from a CUDA graph when the same buffers come back.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <list>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/bang.h"
#include "bang_device.cuh"
#include "bang_internal.h"

struct bang_model;

namespace {

thread_local std::string g_last_error;

bang_status fail(bang_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return s;
}

#define BANG_CUDA(call)                                                                         \
  do {                                                                                          \
    cudaError_t e_ = (call);                                                                    \
    if (e_ != cudaSuccess)                                                                      \
      return fail(e_ == cudaErrorMemoryAllocation ? BANG_E_OOM : BANG_E_CUDA, "%s: %s (%s:%d)", \
                  #call, cudaGetErrorString(e_), __FILE__, __LINE__);                           \
  } while (0)

constexpr double kPiD = 3.14159265358979323846;

// Gauss-Legendre rule on [-1, 1]: Newton's method on P_n from the Bonnet recurrence,
// starting from Tricomi's approximation of the k-th root.
void legendre_rule(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int k = 1; k <= n; ++k) {
    const double th = kPiD * (4.0 * k - 1.0) / (4.0 * n + 2.0);
    double z = (1.0 - (n - 1.0) / (8.0 * n * n * n)) * std::cos(th);
    double dp = 1.0;
    for (int it = 0; it < 60; ++it) {
      double pm = 1.0, p = z;
      for (int j = 1; j < n; ++j) {
        const double pn = ((2.0 * j + 1.0) * z * p - j * pm) / (j + 1.0);
        pm = p;
        p = pn;
      }
      dp = n * (pm - z * p) / (1.0 - z * z);
      const double dz = p / dp;
      z -= dz;
      if (std::fabs(dz) <= 1e-15 * std::fabs(z) + 1e-300) {
        // one more evaluation at the converged root for the weight
        pm = 1.0, p = z;
        for (int j = 1; j < n; ++j) {
          const double pn = ((2.0 * j + 1.0) * z * p - j * pm) / (j + 1.0);
          pm = p;
          p = pn;
        }
        dp = n * (pm - z * p) / (1.0 - z * z);
        break;
      }
    }
    x[n - k] = z;                              // ascending
    w[n - k] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

// Node tables for r = R cosh t, t in [0, 16]: rows [0, 64) for 64 nodes, [64, 192) for 128.
void node_tables(std::vector<float>& cm1, std::vector<float>& lc, std::vector<float>& ws, std::vector<float>& wq) {
  cm1.assign(192, 0.f);
  lc.assign(192, 0.f);
  ws.assign(192, 0.f);
  wq.assign(192, 0.f);
  const double T = 16.0;
  int base = 0;
  for (int n : {64, 128}) {
    std::vector<double> x, w;
    legendre_rule(n, x, w);
    for (int k = 0; k < n; ++k) {
      const double t = 0.5 * T * (x[k] + 1.0), wk = 0.5 * T * w[k];
      const double ch = std::cosh(t), th = std::tanh(t);
      const double sh = std::sinh(0.5 * t);
      cm1[base + k] = (float)(2.0 * sh * sh);   // cosh t - 1 without cancellation
      lc[base + k] = (float)std::log2(ch);
      ws[base + k] = (float)(wk * ch);
      wq[base + k] = (float)(wk * th * th);
    }
    base += n;
  }
}

// The same rule in float64 for the check path: cosh t_k, tanh^2 t_k, w_k, rows as above.
void node_tables64(std::vector<double>& ch, std::vector<double>& th2, std::vector<double>& w64) {
  ch.assign(192, 0.0);
  th2.assign(192, 0.0);
  w64.assign(192, 0.0);
  const double T = 16.0;
  int base = 0;
  for (int n : {64, 128}) {
    std::vector<double> x, w;
    legendre_rule(n, x, w);
    for (int k = 0; k < n; ++k) {
      const double t = 0.5 * T * (x[k] + 1.0), th = std::tanh(t);
      ch[base + k] = std::cosh(t);
      th2[base + k] = th * th;
      w64[base + k] = 0.5 * T * w[k];
    }
    base += n;
  }
}

int psf_halfwidth(double fwhm, double pitch) {
  if (!(fwhm > 0.0)) return 0;
  const double sig = fwhm / (2.0 * std::sqrt(2.0 * std::log(2.0)));
  return (int)std::floor(3.0 * sig / pitch);
}

// PSF taps, in fine pixels of pitch p.  The PSF g (Eq. 21's Gaussian, or Moffat) is cut
// to its window: the square |dx|, |dy| <= rho, rho = 3 sigma / p, or with the circular mode
// (psf_mode bit 1) the circle of radius rho that Eq. 21 names.
//  * Binning (default): spaxel column i averages fine columns h + i*os + m, m in [0, os);
//    each of those is the PSF-weighted mean over integer offsets in the window.  Their
//    composition weights padded fine column i*os + c, c in [0, os + 2h), by
//      T[c] = (1/os) sum_m g(c - m - h)    (g normalised to unit sum over the window).
//  * Centre sampling (psf_mode bit 2, App. A): spaxel (i, j) is the PSF-weighted mean of
//    the fine points around its centre, at offset c - h - (os-1)/2 from padded column
//    i*os + c: the points in the window, and always the one or two per axis nearest the
//    centre (|offset| <= 1/2), which alone are used (equal weights) without a PSF.
// Separable ([L], the two-axis weight is T[cy] T[cx]) for a Gaussian with the square
// window; otherwise the two-dimensional table W2[cy][cx] ([L][L]).
// (float64; the kernels take them rounded to float32, the float64 check path as they are)
std::vector<double> make_taps_d(int kind, double fwhm, double beta, int os, int h, double pitch, int mode) {
  const int L = os + 2 * h;
  const bool circle = (mode & BANG_PSF_CIRCLE) != 0, centre = (mode & BANG_PSF_CENTRE) != 0;
  const bool two_d = kind == 1 || circle;
  const bool psf = fwhm > 0.0;
  const double sig = fwhm / (2.0 * std::sqrt(2.0 * std::log(2.0)));
  const double rho = psf ? 3.0 * sig / pitch : 0.0;
  const double alpha = kind == 1 ? fwhm / (2.0 * std::sqrt(std::pow(2.0, 1.0 / beta) - 1.0)) : 1.0;
  auto value = [&](double dx, double dy) {
    const double d2 = (dx * dx + dy * dy) * pitch * pitch;
    return kind == 0 ? std::exp(-d2 / (2.0 * sig * sig)) : std::pow(1.0 + d2 / (alpha * alpha), -beta);
  };
  auto inside = [&](double dx, double dy) {
    return circle ? dx * dx + dy * dy <= rho * rho : std::fabs(dx) <= rho && std::fabs(dy) <= rho;
  };
  const double c0 = h + 0.5 * (os - 1);   // centre of spaxel 0 in padded fine columns
  if (!two_d) {
    std::vector<double> t(L, 0.0);
    double tot = 0.0;
    if (centre) {
      for (int c = 0; c < L; ++c) {
        const double d = c - c0;
        if (std::fabs(d) <= 0.5 || (psf && std::fabs(d) <= rho)) tot += (t[c] = psf ? value(d, 0.0) : 1.0);
      }
      for (double& v : t) v /= tot;
    } else {
      std::vector<double> g(2 * h + 1, 1.0);
      if (h > 0) {
        for (int d = -h; d <= h; ++d) tot += (g[d + h] = value(d, 0.0));
        for (double& v : g) v /= tot;
      }
      for (int c = 0; c < L; ++c) {
        for (int m = 0; m < os; ++m) {
          const int d = c - m - h;
          if (d >= -h && d <= h) t[c] += g[d + h];
        }
        t[c] /= os;
      }
    }
    return t;
  }
  std::vector<double> W2((size_t)L * L, 0.0);
  double tot = 0.0;
  if (centre) {
    for (int cy = 0; cy < L; ++cy)
      for (int cx = 0; cx < L; ++cx) {
        const double dx = cx - c0, dy = cy - c0;
        const bool nearest = std::fabs(dx) <= 0.5 && std::fabs(dy) <= 0.5;
        if (nearest || (psf && inside(dx, dy))) tot += (W2[(size_t)cy * L + cx] = psf ? value(dx, dy) : 1.0);
      }
    for (double& v : W2) v /= tot;
  } else {
    const int n = 2 * h + 1;
    std::vector<double> M((size_t)n * n, 0.0);
    if (h == 0) {
      M[0] = 1.0;
    } else {
      for (int dy = -h; dy <= h; ++dy)
        for (int dx = -h; dx <= h; ++dx)
          if (inside(dx, dy)) tot += (M[(size_t)(dy + h) * n + (dx + h)] = value(dx, dy));
      for (double& v : M) v /= tot;
    }
    for (int cy = 0; cy < L; ++cy)
      for (int cx = 0; cx < L; ++cx) {
        double acc = 0.0;
        for (int mn = 0; mn < os; ++mn)
          for (int mm = 0; mm < os; ++mm) {
            const int dy = cy - mn - h, dx = cx - mm - h;
            if (dy >= -h && dy <= h && dx >= -h && dx <= h) acc += M[(size_t)(dy + h) * n + (dx + h)];
          }
        W2[(size_t)cy * L + cx] = acc / ((double)os * os);
      }
  }
  return W2;
}

std::vector<float> make_taps(int kind, double fwhm, double beta, int os, int h, double pitch, int mode) {
  const std::vector<double> t = make_taps_d(kind, fwhm, beta, os, h, pitch, mode);
  return std::vector<float>(t.begin(), t.end());
}

// Device memory the library allocates while serving calls (plans, staging, scratch), with
// an optional cap set by bang_model_set_scratch_limit.  Entry points that may allocate
// install the model's budget for the calling thread (ScratchScope).
struct ScratchBudget {
  size_t limit = 0;   // 0: no cap
  size_t used = 0;
};
thread_local ScratchBudget* tl_budget = nullptr;

struct ScratchScope {
  ScratchBudget* prev;
  explicit ScratchScope(ScratchBudget* b) : prev(tl_budget) { tl_budget = b; }
  ~ScratchScope() { tl_budget = prev; }
};

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  ScratchBudget* charged = nullptr;
  ~DevBuf() { release(); }
  void release() {
    if (p) cudaFree(p);
    if (charged) charged->used -= bytes;
    p = nullptr;
    bytes = 0;
    charged = nullptr;
  }
  cudaError_t reserve(size_t b) {
    if (b <= bytes) return cudaSuccess;
    ScratchBudget* bud = tl_budget;
    if (bud && bud->limit && bud->used - (charged == bud ? bytes : 0) + b > bud->limit)
      return cudaErrorMemoryAllocation;   // over the caller's cap: nothing is freed or allocated
    release();
    cudaError_t e = cudaMalloc(&p, b);
    if (e != cudaSuccess) {
      p = nullptr;
      return e;
    }
    bytes = b;
    charged = bud;
    if (bud) bud->used += b;
    return e;
  }
  template <class T> T* as() const { return reinterpret_cast<T*>(p); }
};

// Batch shapes whose plans (and captured graphs) a model keeps, least recently used
// evicted: a sampler's calls come in a few dozen sizes, and an evicted plan frees device
// buffers (which synchronises) and is rebuilt and re-captured on its next use.
constexpr size_t kMaxPlans = 32;

// A batch shape: the work items of (gal_idx, B) and their device copies.
struct Plan {
  uint64_t key = 0;
  int B = 0, n_items = 0, G = 4, grid = 0, blocks_per_sm = 0;
  int max_W = 0;   // widest fine grid among the plan's galaxies (chunk_pts = G max_W)
  int col_lanes = 0;   // FwdArgs::col_lanes of the launch
  size_t smem = 0;
  int mode = 0;
  int kmode = 0;   // the forward kernel form launched (kModeLogL2 for a tuned logL batch)
  std::vector<bang::WorkItem> items;
  std::vector<int> order, row_first, row_g;
  std::vector<int64_t> out_off;
  int64_t out_total = 0;
  DevBuf d_items, d_order, d_row_first, d_row_g, d_out_off, d_partial, d_queue, d_consts, d_tables;
  int64_t table_stride = 0;   // floats per row of the radial tables (bulge_table option)
  int bands = 1;
  // adjoint sweep (kModeSeed plans only): bands of fine rows
  int adj_items = 0, adj_G = 4, adj_grid = 0, adj_minb = 0, adj_blocks_per_sm = 0;
  size_t adj_smem = 0;
  DevBuf d_adj_items, d_adj_order, d_adj_row_first;
  // device-index plan (gal_idx in device memory): implicit work items, nb per row and
  // adj_nb fine-row bands of adj_rows rows per row; seeds at a fixed stride per row; items
  // ordered on the device by the rank of their galaxy's cost (d_rank, d_adj_rank)
  bool implicit = false;
  int nb = 1, adj_nb = 1, n_rank = 0, n_adj_rank = 0;
  int64_t out_stride = 0;
  DevBuf d_rank, d_adj_rank;
  // graph replay
  cudaGraphExec_t graph = nullptr;
  const void* g_theta = nullptr;
  const void* g_out = nullptr;
  const void* g_out2 = nullptr;
  const void* g_gal = nullptr;
  ~Plan() {
    if (graph) cudaGraphExecDestroy(graph);
  }
};

uint64_t hash_bytes(const void* data, size_t n, uint64_t h = 1469598103934665603ull) {
  const unsigned char* p = static_cast<const unsigned char*>(data);
  for (size_t i = 0; i < n; ++i) {
    h ^= p[i];
    h *= 1099511628211ull;
  }
  return h;
}

bool is_device_pointer(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Where gal_idx lives: 0 host memory (or NULL), 1 device (or managed) memory the model's
// device can read, -1 device memory of another device.
int gal_idx_place(const int32_t* gal_idx, int device) {
  if (!gal_idx) return 0;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, gal_idx) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  if (at.type == cudaMemoryTypeManaged) return 1;
  if (at.type != cudaMemoryTypeDevice) return 0;
  return at.device == device ? 1 : -1;
}

// A host copy of gal_idx for the entry points that schedule on the host (synchronous).
bang_status host_gal_idx(const int32_t* gal_idx, int B, int device, std::vector<int32_t>& buf, const int32_t** out) {
  *out = gal_idx;
  const int place = gal_idx_place(gal_idx, device);
  if (place < 0) return fail(BANG_E_INVALID_ARG, "gal_idx is device memory of another device");
  if (place == 0) return BANG_OK;
  buf.resize((size_t)B);
  BANG_CUDA(cudaMemcpy(buf.data(), gal_idx, sizeof(int32_t) * (size_t)B, cudaMemcpyDeviceToHost));
  *out = buf.data();
  return BANG_OK;
}

}  // namespace

struct bang_model {
  int device = 0;
  bang_model_opts opts{};
  int P = 15;
  int num_sms = 0;
  int smem_optin = 0;
  std::vector<bang::GalDev> gals;   // host copy (device pointers inside)
  std::vector<bang_galaxy_desc> desc;
  std::vector<int> h_of;
  std::vector<std::unique_ptr<DevBuf>> owned;
  DevBuf d_gals;
  DevBuf stage_theta, stage_out, stage_out2, scratch_seed, scratch_grad, scratch_plain;
  DevBuf grids_in, grids_theta, grids_out;   // bang_loglike_grids: staged theta, expanded rows, sums
  std::mutex grids_mu;
  std::list<std::unique_ptr<Plan>> plans;   // most recently used first
  struct Tuning {
    int G = 4;       // fine rows per block step of the forward kernel
    int bands = 0;   // spaxel-row bands per batch row (0: default policy)
    int adj_G = 0;   // fine rows per band of the adjoint (0: default policy)
    int pair = 0;    // logL batches: 1 = the two-points-per-thread kernel form (kModeLogL2)
    int seed_G = 0;  // fine rows per block step of the gradient call's forward pass (0: G)
    int adj_minb = 0;  // blocks per SM of the one-disc quadrature adjoint, 3 or 4 (0: 4)
    int seed_bands = 0;  // spaxel-row bands per row of the gradient call's forward pass (0: bands)
    int lanes = 0;       // logL launch: several lanes per spaxel column in the separable stencil
    int seed_lanes = 0;  // the same for the gradient call's forward pass
  };
  std::map<uint64_t, Tuning> tuned;         // batch-shape key -> launch parameters
  std::mutex mu;
  ScratchBudget budget;
  cudaStream_t capture_stream = nullptr;
  cudaEvent_t last_work = nullptr;   // recorded after each call's device work (see CallOrder)
  bool use_graphs = true;
  // float64 check path (bang_loglike_fp64): float64 taps and 1/delta^2 kept from create,
  // uploaded with the float64 node rule on the first call
  std::vector<std::vector<double>> taps64, iv64;
  std::vector<double> pitch64;
  std::vector<bang::Gal64> g64;
  DevBuf nodes64, fp64_scratch, fp64_theta, fp64_out;
  std::mutex fp64_mu;
};

namespace {

bang_status validate_desc(const bang_galaxy_desc& d, int g) {
  if (d.nx < 1 || d.ny < 1 || d.oversample < 1) return fail(BANG_E_INVALID_ARG, "galaxy %d: bad grid size", g);
  if (!(d.spaxel_arcsec > 0.0) || !(d.kpc_per_arcsec > 0.0))
    return fail(BANG_E_INVALID_ARG, "galaxy %d: spaxel size and distance scale must be > 0", g);
  if (d.psf_kind != 0 && d.psf_kind != 1) return fail(BANG_E_INVALID_ARG, "galaxy %d: psf_kind must be 0 or 1", g);
  if (!(d.psf_fwhm_arcsec >= 0.0)) return fail(BANG_E_INVALID_ARG, "galaxy %d: psf_fwhm must be >= 0", g);
  if (d.psf_kind == 1 && !(d.moffat_beta > 0.0)) return fail(BANG_E_INVALID_ARG, "galaxy %d: moffat_beta must be > 0", g);
  if (!d.data || !d.err) return fail(BANG_E_INVALID_ARG, "galaxy %d: data and err are required", g);
  const int h = psf_halfwidth(d.psf_fwhm_arcsec, d.spaxel_arcsec / d.oversample);
  if (h > 64) return fail(BANG_E_INVALID_ARG, "galaxy %d: PSF window half-width %d exceeds 64 fine pixels", g, h);
  if ((long long)d.nx * d.oversample + 2 * h > 4096 || d.ny > 4096)
    return fail(BANG_E_INVALID_ARG, "galaxy %d: padded fine grid wider than 4096", g);
  const size_t n = (size_t)4 * d.nx * d.ny;
  for (size_t s = 0; s < n; ++s) {
    if (d.mask && !d.mask[s]) continue;
    if (!(d.err[s] > 0.f) || !std::isfinite(d.err[s]) || !std::isfinite(d.data[s]))
      return fail(BANG_E_INVALID_ARG, "galaxy %d: err must be finite and > 0 and data finite where used (entry %zu)",
                  g, s);
  }
  return BANG_OK;
}

template <class T>
bang_status upload(bang_model* m, const std::vector<T>& v, const T** out) {
  auto b = std::make_unique<DevBuf>();
  BANG_CUDA(b->reserve(std::max<size_t>(v.size() * sizeof(T), 16)));
  BANG_CUDA(cudaMemcpy(b->p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  *out = b->as<T>();
  m->owned.push_back(std::move(b));
  return BANG_OK;
}

template <class T>
cudaError_t copy_vec(DevBuf& d, const std::vector<T>& v) {
  cudaError_t e = d.reserve(std::max<size_t>(v.size() * sizeof(T), 16));
  if (e != cudaSuccess) return e;
  return cudaMemcpy(d.p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
}

// Bands of spaxel rows per batch row: 1 when the batch fills the GPU, otherwise enough to
// give every SM about two work items (each band re-evaluates its 2h-row halo).
int bands_for(const bang_model* m, int B, int ny, int forced) {
  if (forced > 0) return std::max(1, std::min(ny, forced));
  if (B >= m->num_sms) return 1;
  const int want = (2 * m->num_sms + B - 1) / B;
  return std::max(1, std::min(ny, want));
}

uint64_t shape_key(const int32_t* gal_idx, int B) {
  uint64_t key = hash_bytes(&B, sizeof B);
  if (gal_idx) key = hash_bytes(gal_idx, sizeof(int32_t) * (size_t)B, key);
  return key;
}

bang_status get_plan(bang_model* m, const int32_t* gal_idx, int B, int mode, Plan** out) {
  const uint64_t skey = shape_key(gal_idx, B);
  const uint64_t key = hash_bytes(&mode, sizeof mode, skey);
  bang_model::Tuning tune;
  {
    auto t = m->tuned.find(skey);
    if (t != m->tuned.end()) tune = t->second;
  }
  for (auto it = m->plans.begin(); it != m->plans.end(); ++it) {
    if ((*it)->key == key) {
      m->plans.splice(m->plans.begin(), m->plans, it);
      *out = m->plans.front().get();
      return BANG_OK;
    }
  }
  auto p = std::make_unique<Plan>();
  p->key = key;
  p->B = B;
  p->mode = mode;
  p->row_first.assign(B + 1, 0);
  p->row_g.assign(B, 0);
  p->out_off.assign(B, 0);
  std::vector<double> cost;
  int64_t off = 0;
  // bands per row from the model's tallest galaxy (a shorter galaxy's empty bands are
  // skipped), the policy of the device-index plans, so that both split a row alike
  int ny_model = 1, H_model = 1;
  for (const bang::GalDev& G : m->gals) {
    ny_model = std::max(ny_model, G.ny);
    H_model = std::max(H_model, G.H);
  }
  const int nb = bands_for(m, B, ny_model, mode == bang::kModeSeed && tune.seed_bands > 0 ? tune.seed_bands : tune.bands);
  for (int b = 0; b < B; ++b) {
    const int g = gal_idx ? gal_idx[b] : 0;
    if (g < 0 || g >= (int)m->gals.size()) return fail(BANG_E_INVALID_ARG, "gal_idx[%d] = %d out of range", b, g);
    const bang::GalDev& G = m->gals[g];
    p->row_g[b] = g;
    p->out_off[b] = off;
    off += (int64_t)4 * G.nx * G.ny;
    p->row_first[b] = (int)p->items.size();
    p->bands = std::max(p->bands, nb);
    for (int k = 0; k < nb; ++k) {
      const int j0 = (int)((long long)G.ny * k / nb), j1 = (int)((long long)G.ny * (k + 1) / nb);
      if (j1 <= j0) continue;
      p->items.push_back(bang::WorkItem{b, g, j0, j1});
      cost.push_back((double)((j1 - j0) * G.os + 2 * G.h) * G.W);
    }
  }
  p->row_first[B] = (int)p->items.size();
  p->out_total = off;
  p->n_items = (int)p->items.size();
  // longest items first, so that the persistent blocks finish together
  p->order.resize(p->n_items);
  for (int i = 0; i < p->n_items; ++i) p->order[i] = i;
  std::stable_sort(p->order.begin(), p->order.end(), [&](int a, int b) { return cost[a] > cost[b]; });

  int max_L = 0, max_os = 1, max_nx = 0, max_W = 0, psf2d = 0;
  for (int b = 0; b < B; ++b) {
    const bang::GalDev& G = m->gals[p->row_g[b]];
    max_L = std::max(max_L, G.L);
    max_os = std::max(max_os, G.os);
    max_nx = std::max(max_nx, G.nx);
    max_W = std::max(max_W, G.W);
    psf2d |= G.psf_kind;
  }
  for (int b = 0; b < B; ++b)
    if (m->gals[p->row_g[b]].psf_kind != psf2d)
      return fail(BANG_E_UNSUPPORTED, "a batch mixes Gaussian and Moffat PSF galaxies");
  p->max_W = max_W;
  p->G = (mode == bang::kModeSeed && tune.seed_G > 0) ? tune.seed_G : tune.G;
  // shared memory: the NA bound uses the smallest os among rows with the largest L, so
  // take it per galaxy
  size_t smem = 0;
  for (int b = 0; b < B; ++b) {
    const bang::GalDev& G = m->gals[p->row_g[b]];
    smem = std::max(smem, bang::forward_smem_bytes(G.L, G.os, G.nx, G.W, p->G, psf2d, m->opts.bulge_table));
  }
  if (smem > (size_t)m->smem_optin - 4096) {
    p->G = 1;
    smem = 0;
    for (int b = 0; b < B; ++b) {
      const bang::GalDev& G = m->gals[p->row_g[b]];
      smem = std::max(smem, bang::forward_smem_bytes(G.L, G.os, G.nx, G.W, 1, psf2d, m->opts.bulge_table));
    }
    if (smem > (size_t)m->smem_optin - 4096) return fail(BANG_E_UNSUPPORTED, "galaxy too large for one block's shared memory");
  }
  p->smem = smem;
  p->kmode = (mode == bang::kModeLogL && tune.pair) ? bang::kModeLogL2 : mode;
  p->col_lanes = mode == bang::kModeLogL ? tune.lanes : mode == bang::kModeSeed ? tune.seed_lanes : 0;
  const void* kp = bang::forward_kernel_ptr(m->opts.n_quad, m->opts.n_discs, psf2d, p->kmode);
  cudaFuncAttributes fa;
  BANG_CUDA(cudaFuncGetAttributes(&fa, kp));
  if (smem + fa.sharedSizeBytes > (size_t)m->smem_optin)
    return fail(BANG_E_UNSUPPORTED, "forward kernel needs %zu bytes of shared memory", smem + fa.sharedSizeBytes);
  BANG_CUDA(cudaFuncSetAttribute(kp, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 m->smem_optin - (int)fa.sharedSizeBytes));
  int per_sm = 0;
  BANG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kp, bang::forward_threads(), smem));
  if (per_sm < 1) return fail(BANG_E_UNSUPPORTED, "forward kernel does not fit on an SM (smem %zu)", smem);
  p->blocks_per_sm = per_sm;
  p->grid = std::min(p->n_items, per_sm * m->num_sms);

  if (mode == bang::kModeSeed) {
    // adjoint work items: bands of fine rows, sized for ~16 items per SM of B rows of the
    // model's tallest grid (as the device-index plans size them)
    const long long total_rows = (long long)B * H_model;
    // one staging step per band: rows per band = rows per block step (at most 16)
    const long long target = 16LL * m->num_sms;
    const int rows = tune.adj_G > 0 ? tune.adj_G
                                    : (int)std::max<long long>(1, std::min<long long>(16, (total_rows + target - 1) / target));
    p->adj_G = rows;
    std::vector<bang::WorkItem> ai;
    std::vector<double> acost;
    std::vector<int> arow_first(B + 1, 0);
    for (int b = 0; b < B; ++b) {
      const bang::GalDev& G = m->gals[p->row_g[b]];
      arow_first[b] = (int)ai.size();
      for (int y = 0; y < G.H; y += rows) {
        ai.push_back(bang::WorkItem{b, p->row_g[b], y, std::min(G.H, y + rows)});
        acost.push_back((double)(std::min(G.H, y + rows) - y) * G.W);
      }
    }
    arow_first[B] = (int)ai.size();
    std::vector<int> aorder(ai.size());
    for (size_t i = 0; i < ai.size(); ++i) aorder[i] = (int)i;
    std::stable_sort(aorder.begin(), aorder.end(), [&](int x, int y) { return acost[x] > acost[y]; });
    p->adj_items = (int)ai.size();
    size_t asmem = 0;
    for (int b = 0; b < B; ++b) {
      const bang::GalDev& G = m->gals[p->row_g[b]];
      asmem = std::max(asmem, bang::adjoint_smem_bytes(G.L, G.os, G.nx, p->adj_G, psf2d, m->opts.bulge_table));
    }
    p->adj_smem = asmem;
    p->adj_minb = bang::adjoint_minb(m->opts.n_discs, m->opts.bulge_table > 0, tune.adj_minb);
    const void* ak = bang::adjoint_kernel_ptr(m->opts.n_quad, m->opts.n_discs, psf2d, m->opts.bulge_table > 0,
                                              p->adj_minb);
    cudaFuncAttributes afa;
    BANG_CUDA(cudaFuncGetAttributes(&afa, ak));
    if (asmem + afa.sharedSizeBytes > (size_t)m->smem_optin)
      return fail(BANG_E_UNSUPPORTED, "adjoint kernel needs %zu bytes of shared memory", asmem + afa.sharedSizeBytes);
    BANG_CUDA(cudaFuncSetAttribute(ak, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   m->smem_optin - (int)afa.sharedSizeBytes));
    int aper = 0;
    BANG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&aper, ak, bang::adjoint_threads(), asmem));
    if (aper < 1) return fail(BANG_E_UNSUPPORTED, "adjoint kernel does not fit on an SM");
    p->adj_blocks_per_sm = aper;
    p->adj_grid = std::min(p->adj_items, aper * m->num_sms);
    BANG_CUDA(copy_vec(p->d_adj_items, ai));
    BANG_CUDA(copy_vec(p->d_adj_order, aorder));
    BANG_CUDA(copy_vec(p->d_adj_row_first, arow_first));
  }
  BANG_CUDA(copy_vec(p->d_items, p->items));
  BANG_CUDA(copy_vec(p->d_order, p->order));
  BANG_CUDA(copy_vec(p->d_row_first, p->row_first));
  BANG_CUDA(copy_vec(p->d_row_g, p->row_g));
  BANG_CUDA(copy_vec(p->d_out_off, p->out_off));
  BANG_CUDA(p->d_partial.reserve(sizeof(double) * std::max(1, p->n_items)));
  BANG_CUDA(p->d_queue.reserve(2 * sizeof(int)));
  BANG_CUDA(p->d_consts.reserve(bang::model_const_bytes() * (size_t)B));
  if (m->opts.bulge_table > 0) {
    p->table_stride = bang::table_row_floats(m->opts.bulge_table, mode == bang::kModeSeed);
    BANG_CUDA(p->d_tables.reserve(sizeof(float) * (size_t)p->table_stride * B));
  }
  m->plans.push_front(std::move(p));
  while (m->plans.size() > kMaxPlans) m->plans.pop_back();
  *out = m->plans.front().get();
  return BANG_OK;
}

// Ranks of the model's galaxies by the cost of one work item (0 = costliest), for the
// device-side ordering of implicit items.
std::vector<int> galaxy_ranks(const std::vector<double>& cost) {
  std::vector<int> idx(cost.size()), rank(cost.size());
  for (size_t i = 0; i < idx.size(); ++i) idx[i] = (int)i;
  std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return cost[a] > cost[b]; });
  for (size_t r = 0; r < idx.size(); ++r) rank[idx[r]] = (int)r;
  return rank;
}

constexpr int kMaxOrderedGalaxies = 8192;   // beyond, implicit items run in index order

uint64_t device_key(int B) {
  const uint64_t tag = 0x6465766963652d67ull;   // keys of device-index plans differ from any host shape
  return hash_bytes(&B, sizeof B, hash_bytes(&tag, sizeof tag));
}

// A plan for a batch whose gal_idx is device memory: nothing about the rows' galaxies is
// known on the host, so the launch is sized for every galaxy of the model (shared memory,
// bands: enough for the tallest galaxy, empty for shorter ones) and the work items are
// implicit (the kernels read the galaxy of each row on the device).
bang_status get_dplan(bang_model* m, int B, int mode, Plan** out) {
  const uint64_t skey = device_key(B);
  const uint64_t key = hash_bytes(&mode, sizeof mode, skey);
  bang_model::Tuning tune;
  {
    auto t = m->tuned.find(skey);
    if (t != m->tuned.end()) tune = t->second;
  }
  for (auto it = m->plans.begin(); it != m->plans.end(); ++it) {
    if ((*it)->key == key) {
      m->plans.splice(m->plans.begin(), m->plans, it);
      *out = m->plans.front().get();
      return BANG_OK;
    }
  }
  const int n_gal = (int)m->gals.size();
  int psf2d = m->gals[0].psf_kind, ny_max = 1, H_max = 1, n4_max = 4;
  for (const bang::GalDev& G : m->gals) {
    if (G.psf_kind != psf2d)
      return fail(BANG_E_UNSUPPORTED, "a device gal_idx needs galaxies of one PSF kind (the model mixes Gaussian and "
                                      "two-dimensional taps)");
    ny_max = std::max(ny_max, G.ny);
    H_max = std::max(H_max, G.H);
    n4_max = std::max(n4_max, 4 * G.nx * G.ny);
  }
  auto p = std::make_unique<Plan>();
  p->key = key;
  p->B = B;
  p->mode = mode;
  p->implicit = true;
  p->nb = bands_for(m, B, ny_max, mode == bang::kModeSeed && tune.seed_bands > 0 ? tune.seed_bands : tune.bands);
  p->bands = p->nb;
  p->n_items = B * p->nb;
  p->out_stride = n4_max;
  p->out_total = (int64_t)B * n4_max;
  p->G = (mode == bang::kModeSeed && tune.seed_G > 0) ? tune.seed_G : tune.G;
  for (const bang::GalDev& G : m->gals) p->max_W = std::max(p->max_W, G.W);
  size_t smem = 0;
  for (const bang::GalDev& G : m->gals)
    smem = std::max(smem, bang::forward_smem_bytes(G.L, G.os, G.nx, G.W, p->G, psf2d, m->opts.bulge_table));
  if (smem > (size_t)m->smem_optin - 4096) {
    p->G = 1;
    smem = 0;
    for (const bang::GalDev& G : m->gals)
      smem = std::max(smem, bang::forward_smem_bytes(G.L, G.os, G.nx, G.W, 1, psf2d, m->opts.bulge_table));
    if (smem > (size_t)m->smem_optin - 4096) return fail(BANG_E_UNSUPPORTED, "galaxy too large for one block's shared memory");
  }
  p->smem = smem;
  p->kmode = (mode == bang::kModeLogL && tune.pair) ? bang::kModeLogL2 : mode;
  p->col_lanes = mode == bang::kModeLogL ? tune.lanes : mode == bang::kModeSeed ? tune.seed_lanes : 0;
  const void* kp = bang::forward_kernel_ptr(m->opts.n_quad, m->opts.n_discs, psf2d, p->kmode);
  cudaFuncAttributes fa;
  BANG_CUDA(cudaFuncGetAttributes(&fa, kp));
  if (smem + fa.sharedSizeBytes > (size_t)m->smem_optin)
    return fail(BANG_E_UNSUPPORTED, "forward kernel needs %zu bytes of shared memory", smem + fa.sharedSizeBytes);
  BANG_CUDA(cudaFuncSetAttribute(kp, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 m->smem_optin - (int)fa.sharedSizeBytes));
  int per_sm = 0;
  BANG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kp, bang::forward_threads(), smem));
  if (per_sm < 1) return fail(BANG_E_UNSUPPORTED, "forward kernel does not fit on an SM (smem %zu)", smem);
  p->blocks_per_sm = per_sm;
  p->grid = std::min(p->n_items, per_sm * m->num_sms);
  const bool ordered = n_gal > 1 && n_gal <= kMaxOrderedGalaxies;
  if (ordered) {
    std::vector<double> cost(n_gal);
    for (int g = 0; g < n_gal; ++g) {
      const bang::GalDev& G = m->gals[g];
      cost[g] = (double)((G.ny + p->nb - 1) / p->nb * G.os + 2 * G.h) * G.W;
    }
    p->n_rank = n_gal;
    BANG_CUDA(copy_vec(p->d_rank, galaxy_ranks(cost)));
    BANG_CUDA(p->d_order.reserve(sizeof(int) * (size_t)p->n_items));
  }
  if (mode == bang::kModeSeed) {
    const long long target = 16LL * m->num_sms;
    const int rows = tune.adj_G > 0 ? tune.adj_G
                                    : (int)std::max<long long>(1, std::min<long long>(16, ((long long)B * H_max + target - 1) / target));
    p->adj_G = rows;
    p->adj_nb = (H_max + rows - 1) / rows;
    p->adj_items = B * p->adj_nb;
    size_t asmem = 0;
    for (const bang::GalDev& G : m->gals)
      asmem = std::max(asmem, bang::adjoint_smem_bytes(G.L, G.os, G.nx, p->adj_G, psf2d, m->opts.bulge_table));
    p->adj_smem = asmem;
    p->adj_minb = bang::adjoint_minb(m->opts.n_discs, m->opts.bulge_table > 0, tune.adj_minb);
    const void* ak = bang::adjoint_kernel_ptr(m->opts.n_quad, m->opts.n_discs, psf2d, m->opts.bulge_table > 0,
                                              p->adj_minb);
    cudaFuncAttributes afa;
    BANG_CUDA(cudaFuncGetAttributes(&afa, ak));
    if (asmem + afa.sharedSizeBytes > (size_t)m->smem_optin)
      return fail(BANG_E_UNSUPPORTED, "adjoint kernel needs %zu bytes of shared memory", asmem + afa.sharedSizeBytes);
    BANG_CUDA(cudaFuncSetAttribute(ak, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   m->smem_optin - (int)afa.sharedSizeBytes));
    int aper = 0;
    BANG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&aper, ak, bang::adjoint_threads(), asmem));
    if (aper < 1) return fail(BANG_E_UNSUPPORTED, "adjoint kernel does not fit on an SM");
    p->adj_blocks_per_sm = aper;
    p->adj_grid = std::min(p->adj_items, aper * m->num_sms);
    if (ordered) {
      std::vector<double> cost(n_gal);
      for (int g = 0; g < n_gal; ++g) cost[g] = (double)rows * m->gals[g].W;
      p->n_adj_rank = n_gal;
      BANG_CUDA(copy_vec(p->d_adj_rank, galaxy_ranks(cost)));
      BANG_CUDA(p->d_adj_order.reserve(sizeof(int) * (size_t)p->adj_items));
    }
  }
  BANG_CUDA(p->d_partial.reserve(sizeof(double) * std::max(1, p->n_items)));
  BANG_CUDA(p->d_queue.reserve(2 * sizeof(int)));
  BANG_CUDA(p->d_consts.reserve(bang::model_const_bytes() * (size_t)B));
  if (m->opts.bulge_table > 0) {
    p->table_stride = bang::table_row_floats(m->opts.bulge_table, mode == bang::kModeSeed);
    BANG_CUDA(p->d_tables.reserve(sizeof(float) * (size_t)p->table_stride * B));
  }
  p->row_g.assign(1, 0);   // psf2d_of: every galaxy of the model has the same PSF kind here
  m->plans.push_front(std::move(p));
  while (m->plans.size() > kMaxPlans) m->plans.pop_back();
  *out = m->plans.front().get();
  return BANG_OK;
}

int psf2d_of(const bang_model* m, const Plan* p) { return m->gals[p->row_g[0]].psf_kind; }

// dgal: the caller's device gal_idx for a device-index plan (p->implicit), else unused.
cudaError_t enqueue_forward(bang_model* m, Plan* p, const float* theta, int mode, double* logL, float* out,
                            cudaStream_t st, double* vsys_partial = nullptr, const int* dgal = nullptr) {
  bang::FwdArgs a{};
  a.theta = theta;
  a.P = m->P;
  a.gals = m->d_gals.as<bang::GalDev>();
  a.items = p->implicit ? nullptr : p->d_items.as<bang::WorkItem>();
  a.gal_idx = p->implicit ? dgal : nullptr;
  a.nb = p->nb;
  a.order = p->d_order.as<int>();
  a.n_items = p->n_items;
  a.G = p->G;
  a.chunk_pts = p->G * p->max_W;
  a.col_lanes = p->col_lanes;
  a.partial = p->d_partial.as<double>();
  a.maps = mode == bang::kModeMaps ? out : nullptr;
  a.seed = mode == bang::kModeSeed ? out : nullptr;
  a.vsys_partial = mode == bang::kModeSeed ? vsys_partial : nullptr;
  a.out_off = p->implicit ? nullptr : p->d_out_off.as<int64_t>();
  a.out_stride = p->out_stride;
  a.queue = p->d_queue.as<int>();
  a.halo_kind = m->opts.halo_kind;
  a.l10k = bang::decode_l10k_host();
  a.B = p->B;
  a.n_gal = (int)m->gals.size();
  a.out_total = p->out_total;
  const int* row_g = p->implicit ? dgal : p->d_row_g.as<int>();
  cudaError_t e = cudaSuccess;
  if (m->opts.bulge_table > 0) {   // the radial tables are built from the decoded rows
    a.consts = p->d_consts.as<bang::ModelConst>();
    e = bang::launch_decode(theta, m->P, m->opts.n_discs, m->opts.halo_kind, a.gals, row_g, a.n_gal, p->B,
                            p->d_consts.as<bang::ModelConst>(), st);
    if (e != cudaSuccess) return e;
  } else {                         // each item decodes its row; the adjoint reads what the seed pass stores
    a.consts_out = mode == bang::kModeSeed ? p->d_consts.as<bang::ModelConst>() : nullptr;
  }
  if (p->implicit && p->n_rank > 0) {
    e = bang::launch_order(dgal, p->d_rank.as<int>(), a.n_gal, p->n_rank, p->B, p->nb, p->d_order.as<int>(), st);
    if (e != cudaSuccess) return e;
  }
  if (m->opts.bulge_table > 0) {
    a.tables = p->d_tables.as<float>();
    a.table_T = m->opts.bulge_table;
    a.table_stride = p->table_stride;
    e = bang::launch_tables(a.consts, a.gals, row_g, a.n_gal, p->B, m->opts.n_quad, a.table_T,
                            mode == bang::kModeSeed, p->d_tables.as<float>(), p->table_stride, st);
    if (e != cudaSuccess) return e;
  }
  e = cudaMemsetAsync(a.queue, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  e = bang::launch_forward(a, m->opts.n_quad, m->opts.n_discs, psf2d_of(m, p), mode == bang::kModeLogL ? p->kmode : mode,
                           p->grid, p->smem, st);
  if (e != cudaSuccess || !logL) return e;
  if (p->implicit)
    return bang::launch_finalize(a.partial, nullptr, dgal, a.gals, p->B, p->n_items, a.n_gal, logL, st, p->nb, 1);
  return bang::launch_finalize(a.partial, p->d_row_first.as<int>(), p->d_row_g.as<int>(), a.gals, p->B, p->n_items,
                               a.n_gal, logL, st);
}

// Scratch of a gradient call: the forward items' d logL / d v_sys, then the adjoint items'
// constant adjoints (every slot is written before it is read: no zeroing).
size_t grad_scratch_bytes(const Plan* p) {
  return sizeof(double) * ((size_t)std::max(1, p->n_items) + (size_t)std::max(1, p->adj_items) * bang::kAdjSlots);
}

cudaError_t enqueue_grad(bang_model* m, Plan* p, const float* theta, double* logL, float* seed, double* scratch,
                         float* grad, cudaStream_t st, const int* dgal = nullptr) {
  double* vsys_partial = scratch;
  double* acc_partial = scratch + std::max(1, p->n_items);
  cudaError_t e = enqueue_forward(m, p, theta, bang::kModeSeed, logL, seed, st, vsys_partial, dgal);
  if (e != cudaSuccess) return e;
  bang::AdjArgs a{};
  a.theta = theta;
  a.P = m->P;
  a.gals = m->d_gals.as<bang::GalDev>();
  a.consts = p->d_consts.as<bang::ModelConst>();
  a.items = p->implicit ? nullptr : p->d_adj_items.as<bang::WorkItem>();
  a.gal_idx = p->implicit ? dgal : nullptr;
  a.nb = p->adj_nb;
  a.rows_per_item = p->adj_G;
  a.order = p->d_adj_order.as<int>();
  a.n_items = p->adj_items;
  a.G = p->adj_G;
  a.seed = seed;
  a.out_off = p->implicit ? nullptr : p->d_out_off.as<int64_t>();
  a.out_stride = p->out_stride;
  a.acc_partial = acc_partial;
  a.B = p->B;
  a.n_gal = (int)m->gals.size();
  a.seed_total = p->out_total;
  if (m->opts.bulge_table > 0) {
    a.tables = p->d_tables.as<float>();
    a.table_T = m->opts.bulge_table;
    a.table_stride = p->table_stride;
  }
  a.queue = p->d_queue.as<int>() + 1;
  if (p->implicit && p->n_adj_rank > 0) {
    e = bang::launch_order(dgal, p->d_adj_rank.as<int>(), a.n_gal, p->n_adj_rank, p->B, p->adj_nb,
                           p->d_adj_order.as<int>(), st);
    if (e != cudaSuccess) return e;
  }
  e = cudaMemsetAsync(a.queue, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  e = bang::launch_adjoint(a, m->opts.n_quad, m->opts.n_discs, psf2d_of(m, p), p->adj_minb, p->adj_grid, p->adj_smem,
                           st);
  if (e != cudaSuccess) return e;
  if (p->implicit)
    return bang::launch_grad_out(theta, m->P, m->opts.n_discs, m->opts.halo_kind, m->opts.bulge_kind, acc_partial,
                                 nullptr, vsys_partial, nullptr, p->B, p->n_items, p->adj_items, grad, st, p->adj_nb,
                                 p->nb, dgal, (int)m->gals.size());
  return bang::launch_grad_out(theta, m->P, m->opts.n_discs, m->opts.halo_kind, m->opts.bulge_kind, acc_partial,
                               p->d_adj_row_first.as<int>(), vsys_partial, p->d_row_first.as<int>(), p->B,
                               p->n_items, p->adj_items, grad, st);
}

}  // namespace

namespace bang {

bool model_view(const bang_model* m, ModelView* v) {
  if (!m || !v) return false;
  v->device = m->device;
  v->n_gal = (int)m->gals.size();
  v->n_quad = m->opts.n_quad;
  v->n_discs = m->opts.n_discs;
  v->halo_kind = m->opts.halo_kind;
  v->P = m->P;
  v->num_sms = m->num_sms;
  v->smem_optin = m->smem_optin;
  v->bulge_table = m->opts.bulge_table;
  v->h_gals = m->gals.data();
  v->d_gals = m->d_gals.as<GalDev>();
  return true;
}

bang_status set_error(bang_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return s;
}

bang_status check_faults(cudaStream_t st) {
  if constexpr (!kChecked) {
    (void)st;
    return BANG_OK;
  } else {
  BANG_CUDA(cudaStreamSynchronize(st));
  struct {
    const char* unit;
    cudaError_t (*take)(Fault*);
  } units[] = {{"forward", take_fault_forward}, {"adjoint", take_fault_adjoint}, {"plain", take_fault_plain}};
  for (const auto& u : units) {
    Fault f;
    BANG_CUDA(u.take(&f));
    if (f.site)
      return fail(BANG_E_BOUNDS, "index check failed in the %s kernels: %s, index %lld outside [0, %lld)", u.unit,
                  check_site_name((int)f.site - 1), f.index, f.bound);
  }
  return BANG_OK;
  }
}

}  // namespace bang

extern "C" {

const char* bang_last_error(void) { return g_last_error.c_str(); }

int bang_checked_build(void) { return bang::kChecked ? 1 : 0; }

bang_status bang_check_selftest(int device, long long index, long long bound) {
  g_last_error.clear();
  if constexpr (!bang::kChecked) {
    (void)device, (void)index, (void)bound;
    return fail(BANG_E_UNSUPPORTED, "bang_check_selftest: not the checked build");
  } else {
    BANG_CUDA(cudaSetDevice(device));
    BANG_CUDA(bang::launch_check_selftest(index, bound, nullptr));
    return bang::check_faults(nullptr);
  }
}

bang_status bang_model_create(const bang_galaxy_desc* gal, int n_gal, const bang_model_opts* opts, int device,
                              bang_model** out) {
  bang::NvtxRange nvtx("bang_model_create");
  g_last_error.clear();
  if (!gal || !opts || !out || n_gal < 1) return fail(BANG_E_INVALID_ARG, "bang_model_create: null argument or n_gal < 1");
  *out = nullptr;
  if (opts->n_discs != 1 && opts->n_discs != 2) return fail(BANG_E_INVALID_ARG, "n_discs must be 1 or 2");
  if (opts->n_quad != 64 && opts->n_quad != 128) return fail(BANG_E_INVALID_ARG, "n_quad must be 64 or 128");
  if (opts->bulge_kind < 0 || opts->bulge_kind > 2)
    return fail(BANG_E_UNSUPPORTED, "bulge_kind %d not available (0 Dehnen, 1 Hernquist, 2 Jaffe)", opts->bulge_kind);
  if (opts->bulge_kind != 0 && opts->bulge_table != 0)
    return fail(BANG_E_UNSUPPORTED, "the radial-table option applies to the Dehnen bulge (bulge_kind 0) only");
  if (opts->halo_kind != 0 && opts->halo_kind != 1)
    return fail(BANG_E_UNSUPPORTED, "halo_kind %d not available (0 NFW, 1 Hernquist)", opts->halo_kind);
  if (opts->psf_mode < 0 || opts->psf_mode > (BANG_PSF_CIRCLE | BANG_PSF_CENTRE | BANG_PSF_FLUX))
    return fail(BANG_E_INVALID_ARG, "psf_mode %d: a sum of BANG_PSF_CIRCLE, BANG_PSF_CENTRE, BANG_PSF_FLUX",
                opts->psf_mode);
  if (opts->bulge_table != 0 && (opts->bulge_table < 256 || opts->bulge_table > 4096))
    return fail(BANG_E_INVALID_ARG, "bulge_table must be 0 or in [256, 4096]");
  for (int g = 0; g < n_gal; ++g) {
    bang_status s = validate_desc(gal[g], g);
    if (s != BANG_OK) return s;
  }
  int ndev = 0;
  BANG_CUDA(cudaGetDeviceCount(&ndev));
  if (device < 0 || device >= ndev) return fail(BANG_E_INVALID_ARG, "device %d out of range (%d devices)", device, ndev);
  BANG_CUDA(cudaSetDevice(device));

  std::unique_ptr<bang_model> m(new bang_model());
  m->device = device;
  m->opts = *opts;
  m->P = opts->n_discs == 2 ? 19 : 15;
  BANG_CUDA(cudaDeviceGetAttribute(&m->num_sms, cudaDevAttrMultiProcessorCount, device));
  BANG_CUDA(cudaDeviceGetAttribute(&m->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device));
  {
    std::vector<float> cm1, lc, ws, wq;
    node_tables(cm1, lc, ws, wq);
    BANG_CUDA(bang::upload_nodes_forward(cm1.data(), lc.data(), ws.data(), wq.data()));
    BANG_CUDA(bang::upload_nodes_adjoint(cm1.data(), lc.data(), ws.data(), wq.data()));
    BANG_CUDA(bang::upload_nodes_plain(cm1.data(), lc.data(), ws.data(), wq.data()));
  }
  for (int g = 0; g < n_gal; ++g) {
    const bang_galaxy_desc& d = gal[g];
    bang::GalDev G{};
    G.nx = d.nx;
    G.ny = d.ny;
    G.os = d.oversample;
    const double pitch = d.spaxel_arcsec / d.oversample;
    G.h = psf_halfwidth(d.psf_fwhm_arcsec, pitch);
    G.L = G.os + 2 * G.h;
    G.W = G.os * G.nx + 2 * G.h;
    G.H = G.os * G.ny + 2 * G.h;
    G.psf_kind = (d.psf_kind == 1 || (opts->psf_mode & BANG_PSF_CIRCLE)) ? 1 : 0;   // two-dimensional taps
    G.flux = (opts->psf_mode & BANG_PSF_FLUX) ? 1 : 0;
    G.bulge_kind = opts->bulge_kind;
    G.pitch_kpa = (float)(pitch * d.kpc_per_arcsec);
    // sky x of padded fine column q: s ((q - h + 1/2) / os - nx / 2)
    G.xoff_kpa = d.spaxel_arcsec * ((0.5 - G.h) / d.oversample - 0.5 * d.nx) * d.kpc_per_arcsec;
    G.yoff_kpa = d.spaxel_arcsec * ((0.5 - G.h) / d.oversample - 0.5 * d.ny) * d.kpc_per_arcsec;
    const size_t n = (size_t)4 * d.nx * d.ny;
    std::vector<float> data(n), iv(n);
    std::vector<double> iv64(n, 0.0);
    double nc = 0.0;
    for (size_t s = 0; s < n; ++s) {
      const bool used = !d.mask || d.mask[s];
      data[s] = used ? d.data[s] : 0.f;
      if (used) {
        const double e = (double)d.err[s];
        iv64[s] = 1.0 / (e * e);
        iv[s] = (float)iv64[s];
        nc += std::log(std::sqrt(2.0 * kPiD) * e);
      } else {
        iv[s] = 0.f;
      }
    }
    G.norm_const = nc;
    bang_status st;
    if ((st = upload(m.get(), data, &G.data)) != BANG_OK) return st;
    if ((st = upload(m.get(), iv, &G.iv)) != BANG_OK) return st;
    const std::vector<float> taps =
        make_taps(d.psf_kind, d.psf_fwhm_arcsec, d.moffat_beta, G.os, G.h, pitch, opts->psf_mode);
    if (G.psf_kind == 1) {
      // the forward kernel keeps one quadrant of the two-dimensional taps: every window here
      // is even in dx and dy, so the mirrored taps agree (to float64 summation order)
      const int L = G.L;
      float tmax = 0.f;
      for (float t : taps) tmax = std::max(tmax, std::fabs(t));
      for (int cy = 0; cy < L; ++cy)
        for (int cx = 0; cx < L; ++cx) {
          const float t = taps[(size_t)cy * L + cx];
          if (std::fabs(t - taps[(size_t)(L - 1 - cy) * L + cx]) > 1e-6f * tmax ||
              std::fabs(t - taps[(size_t)cy * L + (L - 1 - cx)]) > 1e-6f * tmax)
            return fail(BANG_E_UNSUPPORTED, "galaxy %d: two-dimensional PSF taps are not mirror-symmetric", g);
        }
    }
    if ((st = upload(m.get(), taps, &G.taps)) != BANG_OK) return st;
    m->gals.push_back(G);
    m->desc.push_back(d);
    m->h_of.push_back(G.h);
    m->iv64.push_back(std::move(iv64));
    m->taps64.push_back(make_taps_d(d.psf_kind, d.psf_fwhm_arcsec, d.moffat_beta, G.os, G.h, pitch, opts->psf_mode));
    m->pitch64.push_back(pitch * d.kpc_per_arcsec);
  }
  BANG_CUDA(copy_vec(m->d_gals, m->gals));
  BANG_CUDA(cudaStreamCreateWithFlags(&m->capture_stream, cudaStreamNonBlocking));
  BANG_CUDA(cudaEventCreateWithFlags(&m->last_work, cudaEventDisableTiming));
  *out = m.release();
  return BANG_OK;
}

bang_status bang_model_destroy(bang_model* m) {
  if (!m) return BANG_OK;
  cudaSetDevice(m->device);
  cudaDeviceSynchronize();
  if (m->capture_stream) cudaStreamDestroy(m->capture_stream);
  if (m->last_work) cudaEventDestroy(m->last_work);
  delete m;
  return BANG_OK;
}

bang_status bang_model_set_scratch_limit(bang_model* m, int64_t bytes) {
  g_last_error.clear();
  if (!m) return fail(BANG_E_INVALID_ARG, "null model");
  if (bytes < 0) return fail(BANG_E_INVALID_ARG, "negative scratch limit");
  std::lock_guard<std::mutex> lock(m->mu);
  m->budget.limit = (size_t)bytes;
  return BANG_OK;
}

int64_t bang_model_scratch_bytes(const bang_model* m) { return m ? (int64_t)m->budget.used : -1; }

int bang_model_nparams(const bang_model* m) { return m ? m->P : -1; }
int bang_model_ngalaxies(const bang_model* m) { return m ? (int)m->gals.size() : -1; }
int bang_model_psf_halfwidth(const bang_model* m, int g) {
  if (!m || g < 0 || g >= (int)m->gals.size()) return -1;
  return m->h_of[g];
}

int64_t bang_model_maps_size(const bang_model* m, const int32_t* gal_idx, int B) {
  if (!m || B < 0) return -1;
  if (gal_idx_place(gal_idx, m->device) != 0) return -1;   // a host array only
  int64_t n = 0;
  for (int b = 0; b < B; ++b) {
    const int g = gal_idx ? gal_idx[b] : 0;
    if (g < 0 || g >= (int)m->gals.size()) return -1;
    n += (int64_t)4 * m->gals[g].nx * m->gals[g].ny;
  }
  return n;
}

}  // extern "C"

namespace {

// Common driver of the forward-type entry points: stages host buffers, runs (or replays)
// the persistent launch and the finalisation, copies results back for host buffers.
// Orders a call's device work after the previous call's on the same model, whatever streams
// the callers use: the model's staging buffers, scratch and plans are shared by its calls
// (the host side is already serialised by the model's mutex).
struct CallOrder {
  bang_model* m;
  cudaStream_t st;
  CallOrder(bang_model* m_, cudaStream_t s) : m(m_), st(s) { cudaStreamWaitEvent(st, m->last_work, 0); }
  ~CallOrder() { cudaEventRecord(m->last_work, st); }
};

bang_status run_forward(bang_model* m, const float* theta, const int32_t* gal_idx, int B, double* logL, float* maps,
                        int mode, void* stream) {
  g_last_error.clear();
  if (!m) return fail(BANG_E_INVALID_ARG, "null model");
  if (!theta || B < 1) return fail(BANG_E_INVALID_ARG, "theta is null or B < 1");
  if (mode == bang::kModeLogL && !logL) return fail(BANG_E_INVALID_ARG, "logL is null");
  if (mode == bang::kModeMaps && !maps) return fail(BANG_E_INVALID_ARG, "maps is null");
  std::lock_guard<std::mutex> lock(m->mu);
  ScratchScope scope(&m->budget);
  BANG_CUDA(cudaSetDevice(m->device));
  const int gplace = gal_idx_place(gal_idx, m->device);
  if (gplace < 0) return fail(BANG_E_INVALID_ARG, "gal_idx is device memory of another device");
  if (gplace > 0 && mode == bang::kModeMaps)
    return fail(BANG_E_UNSUPPORTED, "bang_model_maps: gal_idx must be host memory (the output packing depends on it)");
  const int* dgal = gplace > 0 ? gal_idx : nullptr;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  CallOrder order(m, st);
  Plan* p = nullptr;
  bang_status s = dgal ? get_dplan(m, B, mode, &p) : get_plan(m, gal_idx, B, mode, &p);
  if (s != BANG_OK) return s;

  const bool th_dev = is_device_pointer(theta);
  const bool out_dev = mode == bang::kModeLogL ? is_device_pointer(logL) : is_device_pointer(maps);
  const float* d_theta = theta;
  const size_t th_bytes = sizeof(float) * (size_t)B * m->P;
  if (!th_dev) {
    BANG_CUDA(m->stage_theta.reserve(th_bytes));
    BANG_CUDA(cudaMemcpyAsync(m->stage_theta.p, theta, th_bytes, cudaMemcpyHostToDevice, st));
    d_theta = m->stage_theta.as<float>();
  }
  double* d_logL = logL;
  float* d_maps = maps;
  const size_t out_bytes = mode == bang::kModeLogL ? sizeof(double) * B : sizeof(float) * (size_t)p->out_total;
  if (!out_dev) {
    BANG_CUDA(m->stage_out.reserve(out_bytes));
    if (mode == bang::kModeLogL) d_logL = m->stage_out.as<double>();
    else d_maps = m->stage_out.as<float>();
  }

  if (m->use_graphs && mode == bang::kModeLogL) {
    if (!p->graph || p->g_theta != d_theta || p->g_out != d_logL || p->g_gal != dgal) {
      if (p->graph) {
        cudaGraphExecDestroy(p->graph);
        p->graph = nullptr;
      }
      cudaGraph_t g = nullptr;
      BANG_CUDA(cudaStreamBeginCapture(m->capture_stream, cudaStreamCaptureModeThreadLocal));
      cudaError_t e = enqueue_forward(m, p, d_theta, mode, d_logL, nullptr, m->capture_stream, nullptr, dgal);
      cudaError_t e2 = cudaStreamEndCapture(m->capture_stream, &g);
      if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return fail(BANG_E_CUDA, "graph capture failed: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
      }
      e = cudaGraphInstantiate(&p->graph, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) return fail(BANG_E_CUDA, "graph instantiate failed: %s", cudaGetErrorString(e));
      p->g_theta = d_theta;
      p->g_out = d_logL;
      p->g_gal = dgal;
    }
    BANG_CUDA(cudaGraphLaunch(p->graph, st));
  } else {
    BANG_CUDA(enqueue_forward(m, p, d_theta, mode, mode == bang::kModeLogL ? d_logL : nullptr, d_maps, st, nullptr,
                              dgal));
  }
  if (!out_dev) {
    BANG_CUDA(cudaMemcpyAsync(mode == bang::kModeLogL ? (void*)logL : (void*)maps, m->stage_out.p, out_bytes,
                              cudaMemcpyDeviceToHost, st));
    BANG_CUDA(cudaStreamSynchronize(st));
  } else if (!th_dev) {
    BANG_CUDA(cudaStreamSynchronize(st));   // the staged theta buffer is reused by the next call
  }
  return bang::check_faults(st);
}

}  // namespace

extern "C" {

bang_status bang_loglike_batch(bang_model* m, const float* theta, const int32_t* gal_idx, int B, double* logL,
                               void* stream) {
  bang::NvtxRange nvtx("bang_loglike_batch");
  return run_forward(m, theta, gal_idx, B, logL, nullptr, bang::kModeLogL, stream);
}

bang_status bang_model_maps(bang_model* m, const float* theta, const int32_t* gal_idx, int B, float* maps,
                            void* stream) {
  bang::NvtxRange nvtx("bang_model_maps");
  return run_forward(m, theta, gal_idx, B, nullptr, maps, bang::kModeMaps, stream);
}

bang_status bang_loglike_grad_batch(bang_model* m, const float* theta, const int32_t* gal_idx, int B, double* logL,
                                    float* grad, void* stream) {
  bang::NvtxRange nvtx("bang_loglike_grad_batch");
  g_last_error.clear();
  if (!m) return fail(BANG_E_INVALID_ARG, "null model");
  if (!theta || !logL || !grad || B < 1) return fail(BANG_E_INVALID_ARG, "theta, logL or grad is null, or B < 1");
  std::lock_guard<std::mutex> lock(m->mu);
  ScratchScope scope(&m->budget);
  BANG_CUDA(cudaSetDevice(m->device));
  const int gplace = gal_idx_place(gal_idx, m->device);
  if (gplace < 0) return fail(BANG_E_INVALID_ARG, "gal_idx is device memory of another device");
  const int* dgal = gplace > 0 ? gal_idx : nullptr;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  CallOrder order(m, st);
  Plan* p = nullptr;
  bang_status s = dgal ? get_dplan(m, B, bang::kModeSeed, &p) : get_plan(m, gal_idx, B, bang::kModeSeed, &p);
  if (s != BANG_OK) return s;
  const size_t th_bytes = sizeof(float) * (size_t)B * m->P;
  const bool th_dev = is_device_pointer(theta), l_dev = is_device_pointer(logL), g_dev = is_device_pointer(grad);
  const float* d_theta = theta;
  if (!th_dev) {
    BANG_CUDA(m->stage_theta.reserve(th_bytes));
    BANG_CUDA(cudaMemcpyAsync(m->stage_theta.p, theta, th_bytes, cudaMemcpyHostToDevice, st));
    d_theta = m->stage_theta.as<float>();
  }
  double* d_logL = logL;
  float* d_grad = grad;
  if (!l_dev || !g_dev) {
    BANG_CUDA(m->stage_out.reserve(sizeof(double) * B + th_bytes + 16));
    if (!l_dev) d_logL = m->stage_out.as<double>();
    if (!g_dev) d_grad = reinterpret_cast<float*>(m->stage_out.as<char>() + sizeof(double) * B);
  }
  BANG_CUDA(m->scratch_seed.reserve(sizeof(float) * (size_t)std::max<int64_t>(p->out_total, 4)));
  BANG_CUDA(m->scratch_grad.reserve(grad_scratch_bytes(p)));
  BANG_CUDA(enqueue_grad(m, p, d_theta, d_logL, m->scratch_seed.as<float>(), m->scratch_grad.as<double>(), d_grad, st,
                         dgal));
  if (!l_dev) BANG_CUDA(cudaMemcpyAsync(logL, d_logL, sizeof(double) * B, cudaMemcpyDeviceToHost, st));
  if (!g_dev) BANG_CUDA(cudaMemcpyAsync(grad, d_grad, th_bytes, cudaMemcpyDeviceToHost, st));
  if (!th_dev || !l_dev || !g_dev) BANG_CUDA(cudaStreamSynchronize(st));
  return bang::check_faults(st);
}

bang_status bang_loglike_grids(bang_model* m, const float* theta, int B, const int32_t* grids, int n_grids,
                               double* logL, float* grad, void* stream) {
  bang::NvtxRange nvtx("bang_loglike_grids");
  g_last_error.clear();
  if (!m) return fail(BANG_E_INVALID_ARG, "null model");
  if (!theta || !logL || !grids || B < 1 || n_grids < 1)
    return fail(BANG_E_INVALID_ARG, "theta, logL or grids is null, or B < 1, or n_grids < 1");
  for (int k = 0; k < n_grids; ++k)
    if (grids[k] < 0 || grids[k] >= (int)m->gals.size())
      return fail(BANG_E_INVALID_ARG, "grids[%d] = %d out of range", k, grids[k]);
  if ((int64_t)B * n_grids > (int64_t)1 << 30) return fail(BANG_E_INVALID_ARG, "B x n_grids too large");
  std::lock_guard<std::mutex> lock(m->grids_mu);
  BANG_CUDA(cudaSetDevice(m->device));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int P = m->P, BX = B * n_grids;
  const size_t th_bytes = sizeof(float) * (size_t)B * P, thx_bytes = sizeof(float) * (size_t)BX * P;
  const float* d_theta = theta;
  if (!is_device_pointer(theta)) {
    BANG_CUDA(m->grids_in.reserve(th_bytes));
    BANG_CUDA(cudaMemcpyAsync(m->grids_in.p, theta, th_bytes, cudaMemcpyHostToDevice, st));
    d_theta = m->grids_in.as<float>();
  }
  // expanded rows, their logL and gradients, and the sums (when the caller's buffers are on the host)
  const size_t lx = sizeof(double) * (size_t)BX, gx = grad ? thx_bytes : 0;
  const size_t sl = sizeof(double) * (size_t)B, sg = grad ? th_bytes : 0;
  BANG_CUDA(m->grids_theta.reserve(thx_bytes));
  BANG_CUDA(m->grids_out.reserve(lx + gx + sl + sg + 64));
  double* logL_x = m->grids_out.as<double>();
  float* grad_x = grad ? reinterpret_cast<float*>(m->grids_out.as<char>() + lx) : nullptr;
  const bool l_dev = is_device_pointer(logL), g_dev = !grad || is_device_pointer(grad);
  double* d_logL = l_dev ? logL : reinterpret_cast<double*>(m->grids_out.as<char>() + lx + gx);
  float* d_grad = !grad ? nullptr : (g_dev ? grad : reinterpret_cast<float*>(m->grids_out.as<char>() + lx + gx + sl));
  BANG_CUDA(bang::launch_expand_rows(d_theta, P, B, n_grids, m->grids_theta.as<float>(), st));
  std::vector<int32_t> gal_x((size_t)BX);
  for (int b = 0; b < B; ++b)
    for (int k = 0; k < n_grids; ++k) gal_x[(size_t)b * n_grids + k] = grids[k];
  bang_status s = grad ? bang_loglike_grad_batch(m, m->grids_theta.as<float>(), gal_x.data(), BX, logL_x, grad_x, stream)
                       : bang_loglike_batch(m, m->grids_theta.as<float>(), gal_x.data(), BX, logL_x, stream);
  if (s != BANG_OK) return s;
  BANG_CUDA(bang::launch_sum_rows(logL_x, grad_x, P, B, n_grids, d_logL, d_grad, st));
  if (!l_dev) BANG_CUDA(cudaMemcpyAsync(logL, d_logL, sl, cudaMemcpyDeviceToHost, st));
  if (!g_dev) BANG_CUDA(cudaMemcpyAsync(grad, d_grad, sg, cudaMemcpyDeviceToHost, st));
  BANG_CUDA(cudaStreamSynchronize(st));   // the staged and expanded buffers are reused by the next call
  return bang::check_faults(st);
}

bang_status bang_loglike_plain(bang_model* m, const float* theta, const int32_t* gal_idx, int B, double* logL,
                               void* stream) {
  bang::NvtxRange nvtx("bang_loglike_plain");
  g_last_error.clear();
  if (!m) return fail(BANG_E_INVALID_ARG, "null model");
  if (!theta || !logL || B < 1) return fail(BANG_E_INVALID_ARG, "theta or logL is null, or B < 1");
  if (m->opts.bulge_table) return fail(BANG_E_UNSUPPORTED, "bang_loglike_plain: no radial-table mode (bulge_table)");
  std::lock_guard<std::mutex> lock(m->mu);
  ScratchScope scope(&m->budget);
  BANG_CUDA(cudaSetDevice(m->device));
  std::vector<int32_t> gal_host;
  {
    bang_status gs = host_gal_idx(gal_idx, B, m->device, gal_host, &gal_idx);
    if (gs != BANG_OK) return gs;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  CallOrder order(m, st);
  size_t need = 0;
  for (int b = 0; b < B; ++b) {
    const int g = gal_idx ? gal_idx[b] : 0;
    if (g < 0 || g >= (int)m->gals.size()) return fail(BANG_E_INVALID_ARG, "gal_idx[%d] = %d out of range", b, g);
    const bang::GalDev& G = m->gals[g];
    need = std::max(need, bang::plain_scratch_bytes(G.W * G.H, G.nx * G.ny));
  }
  BANG_CUDA(m->scratch_plain.reserve(need));
  const size_t th_bytes = sizeof(float) * (size_t)B * m->P;
  const bool th_dev = is_device_pointer(theta), l_dev = is_device_pointer(logL);
  const float* d_theta = theta;
  if (!th_dev) {
    BANG_CUDA(m->stage_theta.reserve(th_bytes));
    BANG_CUDA(cudaMemcpyAsync(m->stage_theta.p, theta, th_bytes, cudaMemcpyHostToDevice, st));
    d_theta = m->stage_theta.as<float>();
  }
  double* d_logL = logL;
  if (!l_dev) {
    BANG_CUDA(m->stage_out.reserve(sizeof(double) * B));
    d_logL = m->stage_out.as<double>();
  }
  for (int b = 0; b < B; ++b) {
    const int g = gal_idx ? gal_idx[b] : 0;
    BANG_CUDA(bang::launch_plain_row(d_theta + (size_t)b * m->P, m->P, m->opts.n_quad, m->opts.n_discs, m->opts.halo_kind,
                                     m->d_gals.as<bang::GalDev>() + g, m->gals[g], m->scratch_plain.p, d_logL + b, st));
  }
  if (!l_dev) BANG_CUDA(cudaMemcpyAsync(logL, d_logL, sizeof(double) * B, cudaMemcpyDeviceToHost, st));
  if (!th_dev || !l_dev) BANG_CUDA(cudaStreamSynchronize(st));
  return bang::check_faults(st);
}

}  // extern "C"

namespace {

// The parameter domain of theta_in_domain (bang_device.cuh), in float64, for the radial-rule
// bulge.
bool in_domain64(const double* th, int nd, int halo_kind) {
  const int np = nd == 2 ? 19 : 15;
  for (int i = 0; i < np; ++i)
    if (!std::isfinite(th[i])) return false;
  if (!(th[3] >= 0.0 && th[3] < 0.5 * kPiD)) return false;
  if (!(th[6] >= 0.0 && th[6] < 3.0)) return false;
  if (!(std::fabs(th[9]) <= 1.0)) return false;
  if (!(th[10] > 0.0 && th[11] > 0.0)) return false;
  if (halo_kind == 0 && !(th[13] > 0.0)) return false;
  if (nd == 2 && !(std::fabs(th[17]) <= 1.0 && th[18] > 0.0)) return false;
  return true;
}

// Device copies of the float64 check path's tables (first call only).
bang_status fp64_prepare(bang_model* m) {
  if (!m->g64.empty()) return BANG_OK;
  std::vector<double> ch, th2, w;
  node_tables64(ch, th2, w);
  std::vector<double> all(ch);
  all.insert(all.end(), th2.begin(), th2.end());
  all.insert(all.end(), w.begin(), w.end());
  BANG_CUDA(copy_vec(m->nodes64, all));
  std::vector<bang::Gal64> g64;
  for (size_t gi = 0; gi < m->gals.size(); ++gi) {
    const bang::GalDev& G = m->gals[gi];
    bang::Gal64 g{};
    g.nx = G.nx;
    g.ny = G.ny;
    g.os = G.os;
    g.h = G.h;
    g.L = G.L;
    g.W = G.W;
    g.H = G.H;
    g.psf2d = G.psf_kind;
    g.pitch = m->pitch64[gi];
    g.xoff = G.xoff_kpa;
    g.yoff = G.yoff_kpa;
    g.norm_const = G.norm_const;
    g.data = G.data;
    bang_status s;
    if ((s = upload(m, m->taps64[gi], &g.taps)) != BANG_OK) return s;
    if ((s = upload(m, m->iv64[gi], &g.iv)) != BANG_OK) return s;
    g64.push_back(g);
  }
  m->g64 = std::move(g64);
  return BANG_OK;
}

}  // namespace

extern "C" {

bang_status bang_loglike_fp64(bang_model* m, const double* theta, const int32_t* gal_idx, int B, double* logL,
                              void* stream) {
  bang::NvtxRange nvtx("bang_loglike_fp64");
  g_last_error.clear();
  if (!m) return fail(BANG_E_INVALID_ARG, "null model");
  if (!theta || !logL || B < 1) return fail(BANG_E_INVALID_ARG, "theta or logL is null, or B < 1");
  if (m->opts.bulge_kind != 0)
    return fail(BANG_E_UNSUPPORTED, "bang_loglike_fp64: radial-rule bulge only (bulge_kind 0)");
  if (m->opts.psf_mode & BANG_PSF_FLUX) return fail(BANG_E_UNSUPPORTED, "bang_loglike_fp64: no flux-weighted PSF mode");
  BANG_CUDA(cudaSetDevice(m->device));
  std::vector<int32_t> gal_host;
  {
    bang_status gs = host_gal_idx(gal_idx, B, m->device, gal_host, &gal_idx);
    if (gs != BANG_OK) return gs;
  }
  for (int b = 0; b < B; ++b) {
    const int g = gal_idx ? gal_idx[b] : 0;
    if (g < 0 || g >= (int)m->gals.size()) return fail(BANG_E_INVALID_ARG, "gal_idx[%d] = %d out of range", b, g);
  }
  std::lock_guard<std::mutex> lock(m->fp64_mu);
  BANG_CUDA(cudaSetDevice(m->device));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  bang_status s = fp64_prepare(m);
  if (s != BANG_OK) return s;
  const int P = m->P;
  const size_t th_bytes = sizeof(double) * (size_t)B * P;
  std::vector<double> th((size_t)B * P), out((size_t)B, 0.0);
  if (is_device_pointer(theta)) {
    BANG_CUDA(cudaMemcpyAsync(th.data(), theta, th_bytes, cudaMemcpyDeviceToHost, st));
    BANG_CUDA(cudaStreamSynchronize(st));
  } else {
    std::memcpy(th.data(), theta, th_bytes);
  }
  size_t need = 16;
  for (int b = 0; b < B; ++b) {
    const bang::Gal64& g = m->g64[gal_idx ? gal_idx[b] : 0];
    need = std::max(need, bang::fp64_scratch_bytes(g.W * g.H, g.nx * g.ny));
  }
  BANG_CUDA(m->fp64_scratch.reserve(need));
  BANG_CUDA(m->fp64_theta.reserve(th_bytes));
  BANG_CUDA(m->fp64_out.reserve(sizeof(double) * B));
  BANG_CUDA(cudaMemcpyAsync(m->fp64_theta.p, th.data(), th_bytes, cudaMemcpyHostToDevice, st));
  const int base = m->opts.n_quad == 64 ? 0 : 64;
  const double* nd64 = m->nodes64.as<double>();
  const bang::Nodes64 nodes{nd64 + base, nd64 + 192 + base, nd64 + 384 + base, m->opts.n_quad};
  std::vector<char> ok((size_t)B);
  for (int b = 0; b < B; ++b) {
    ok[b] = in_domain64(th.data() + (size_t)b * P, m->opts.n_discs, m->opts.halo_kind);
    if (!ok[b]) continue;
    BANG_CUDA(bang::launch_fp64_row(m->fp64_theta.as<double>() + (size_t)b * P, m->opts.n_discs, m->opts.halo_kind,
                                    nodes, m->g64[gal_idx ? gal_idx[b] : 0], m->fp64_scratch.p,
                                    m->fp64_out.as<double>() + b, st));
  }
  BANG_CUDA(cudaMemcpyAsync(out.data(), m->fp64_out.p, sizeof(double) * B, cudaMemcpyDeviceToHost, st));
  BANG_CUDA(cudaStreamSynchronize(st));
  for (int b = 0; b < B; ++b)
    if (!ok[b]) out[b] = -INFINITY;
  if (is_device_pointer(logL)) {
    BANG_CUDA(cudaMemcpyAsync(logL, out.data(), sizeof(double) * B, cudaMemcpyHostToDevice, st));
    BANG_CUDA(cudaStreamSynchronize(st));
  } else {
    std::memcpy(logL, out.data(), sizeof(double) * B);
  }
  return bang::check_faults(st);
}

// The launch shape a call would use (plans are built, nothing is launched).
bang_status bang_model_launch_info(bang_model* m, const int32_t* gal_idx, int B, int grad, int32_t* info) {
  g_last_error.clear();
  if (!m || !info) return fail(BANG_E_INVALID_ARG, "null model or info");
  if (B < 1) return fail(BANG_E_INVALID_ARG, "B < 1");
  std::lock_guard<std::mutex> lock(m->mu);
  ScratchScope scope(&m->budget);
  BANG_CUDA(cudaSetDevice(m->device));
  const int gplace = gal_idx_place(gal_idx, m->device);
  if (gplace < 0) return fail(BANG_E_INVALID_ARG, "gal_idx is device memory of another device");
  const int mode = grad ? bang::kModeSeed : bang::kModeLogL;
  Plan* p = nullptr;
  bang_status s = gplace > 0 ? get_dplan(m, B, mode, &p) : get_plan(m, gal_idx, B, mode, &p);
  if (s != BANG_OK) return s;
  const int32_t v[13] = {p->G, p->bands, p->blocks_per_sm, p->grid, p->n_items, (int32_t)p->smem,
                         grad ? p->adj_G : 0, grad ? p->adj_grid : 0, grad ? p->adj_items : 0, p->implicit ? 1 : 0,
                         p->kmode == bang::kModeLogL2 ? 2 : 1, grad ? p->adj_blocks_per_sm : 0, p->col_lanes};
  std::memcpy(info, v, sizeof v);
  return BANG_OK;
}

// Autotuner: times the forward launch for every (kernel form, fine rows per block step G,
// spaxel-row bands per row) candidate on this batch shape, then logL + gradient calls for
// the seed pass's rows per step and the adjoint's band height, and keeps the fastest for
// later calls.
namespace {
bang_status tune_paths(bang_model* m, const int32_t* gal_idx, int B, bool grad);
}  // namespace

bang_status bang_model_tune(bang_model* m, const int32_t* gal_idx, int B) {
  bang::NvtxRange nvtx("bang_model_tune");
  return tune_paths(m, gal_idx, B, false);
}

bang_status bang_model_tune_grad(bang_model* m, const int32_t* gal_idx, int B) {
  bang::NvtxRange nvtx("bang_model_tune_grad");
  return tune_paths(m, gal_idx, B, true);
}

}  // extern "C"

namespace {

bang_status tune_paths(bang_model* m, const int32_t* gal_idx, int B, bool grad) {
  g_last_error.clear();
  if (!m) return fail(BANG_E_INVALID_ARG, "null model");
  if (B < 1) return fail(BANG_E_INVALID_ARG, "B < 1");
  std::lock_guard<std::mutex> lock(m->mu);
  ScratchScope scope(&m->budget);
  BANG_CUDA(cudaSetDevice(m->device));
  // a device gal_idx is tuned on the device-index launch (implicit work items) that later
  // calls with a device gal_idx of B rows take; its contents are read here only to check them
  const int gplace = gal_idx_place(gal_idx, m->device);
  const int* dgal = gplace > 0 ? gal_idx : nullptr;
  std::vector<int32_t> gal_host;
  const int32_t* hgal = gal_idx;
  {
    bang_status gs = host_gal_idx(gal_idx, B, m->device, gal_host, &hgal);
    if (gs != BANG_OK) return gs;
  }
  int ny_max = 1;
  for (int b = 0; b < B; ++b) {
    const int g = hgal ? hgal[b] : 0;
    if (g < 0 || g >= (int)m->gals.size()) return fail(BANG_E_INVALID_ARG, "gal_idx[%d] = %d out of range", b, g);
    ny_max = std::max(ny_max, m->gals[g].ny);
  }
  if (dgal)
    for (const bang::GalDev& G : m->gals) ny_max = std::max(ny_max, G.ny);
  // in-domain parameter vectors of typical size (the cost does not depend on the values)
  static const float kTypical[19] = {0.02f, -0.03f, 0.5f, 0.9f, 10.0f, 0.0f, 1.0f, 10.5f, 0.5f, 0.5f,
                                     4.0f, 2.5f, 12.5f, 10.0f, 0.0f, 10.2f, 0.6f, 0.6f, 2.5f};
  std::vector<float> th((size_t)B * m->P);
  for (int b = 0; b < B; ++b)
    for (int k = 0; k < m->P; ++k) th[(size_t)b * m->P + k] = kTypical[k] + (k == 2 ? 0.001f * (b % 97) : 0.f);
  BANG_CUDA(cudaEventSynchronize(m->last_work));   // earlier calls may still read the staging buffers
  BANG_CUDA(m->stage_theta.reserve(th.size() * sizeof(float)));
  BANG_CUDA(cudaMemcpy(m->stage_theta.p, th.data(), th.size() * sizeof(float), cudaMemcpyHostToDevice));
  BANG_CUDA(m->stage_out.reserve(sizeof(double) * B));
  const uint64_t skey = dgal ? device_key(B) : shape_key(hgal, B);
  bang_model::Tuning prior;   // an earlier gradient choice survives a forward-only tuning
  {
    auto t = m->tuned.find(skey);
    if (t != m->tuned.end()) prior = t->second;
  }
  std::vector<int> bands = {0};
  if (B < 4 * m->num_sms)
    for (int nb : {1, 2, 4, 8, 16})
      if (nb <= ny_max) bands.push_back(nb);
  cudaStream_t st = m->capture_stream;
  CallOrder order(m, st);
  cudaEvent_t e0, e1;
  BANG_CUDA(cudaEventCreate(&e0));
  BANG_CUDA(cudaEventCreate(&e1));
  float best = 1e30f;
  bang_model::Tuning best_t;
  bool any = false;
  bool separable = false;   // the lanes-per-column choice applies to Gaussian-PSF galaxies
  for (const bang::GalDev& g : m->gals) separable |= g.psf_kind == 0;
  for (int lanes : {0, 1}) {
  if (lanes && !separable) continue;
  for (int pair : {0, 1}) {
  if (lanes && pair) continue;   // the two-point form has one thread per spaxel column
  for (int G : {1, 2, 4, 8}) {
    for (int nb : bands) {
      bang_model::Tuning cand{G, nb, 0, pair};
      cand.lanes = lanes;
      m->tuned[skey] = cand;
      m->plans.clear();
      Plan* p = nullptr;
      if ((dgal ? get_dplan(m, B, bang::kModeLogL, &p) : get_plan(m, hgal, B, bang::kModeLogL, &p)) != BANG_OK)
        continue;
      if (p->G != G) continue;   // shared memory forced a smaller step
      float t_min = 1e30f;
      for (int rep = 0; rep < 4; ++rep) {
        BANG_CUDA(cudaEventRecord(e0, st));
        BANG_CUDA(enqueue_forward(m, p, m->stage_theta.as<float>(), bang::kModeLogL, m->stage_out.as<double>(), nullptr,
                                  st, nullptr, dgal));
        BANG_CUDA(cudaEventRecord(e1, st));
        BANG_CUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        BANG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        if (rep > 0) t_min = std::min(t_min, ms);
      }
      if (t_min < best) {
        best = t_min;
        best_t = cand;
        any = true;
      }
    }
  }
  }
  }
  if (!any) {
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    m->plans.clear();
    m->tuned.erase(skey);
    return fail(BANG_E_UNSUPPORTED, "no launch configuration fits this batch");
  }
  // the gradient path: the forward seed pass's rows per step, then the adjoint's band height
  // (fine rows per work item), then (one-disc quadrature form) the adjoint's blocks per SM,
  // each timed on whole logL + gradient calls
  if (grad) {
    float best_g = 1e30f;
    int best_rows = 0, best_sg = best_t.G, best_minb = 0, best_sb = 0, best_sl = 0;
    struct Cand {
      int sb, sg, rows, minb, sl;   // -1: the best value so far
    };
    std::vector<Cand> cands;
    // the seed pass's bands (0: the logL launch's), chosen for its own kernel form, whose
    // blocks per SM can differ from the tuned logL form's
    for (int sb : {0, 1, 2, 3, 4, 6, 8})
      if (sb <= ny_max && (sb == 0 || B < 2 * m->num_sms)) cands.push_back({sb, best_t.G, 0, 0, 0});
    for (int sg : {1, 2, 4}) cands.push_back({-1, sg, 0, 0, 0});
    for (int rows : {4, 8, 16, 24, 32}) cands.push_back({-1, -1, rows, 0, 0});
    if (m->opts.n_discs == 1 && m->opts.bulge_table == 0) cands.push_back({-1, -1, -1, 3, 0});   // 4 is the default
    if (separable) cands.push_back({-1, -1, -1, -1, 1});   // several lanes per column in the seed pass
    for (const Cand& c : cands) {
      const int sb = c.sb < 0 ? best_sb : c.sb;
      const int sg = c.sg < 0 ? best_sg : c.sg;
      const int rows = c.rows < 0 ? best_rows : c.rows;
      const int minb = c.minb < 0 ? best_minb : c.minb;
      const int sl = c.sl < 0 ? best_sl : c.sl;
      bang_model::Tuning tg = best_t;
      tg.seed_bands = sb;
      tg.seed_G = sg;
      tg.adj_G = rows;
      tg.adj_minb = minb;
      tg.seed_lanes = sl;
      m->tuned[skey] = tg;
      m->plans.clear();
      Plan* p = nullptr;
      if ((dgal ? get_dplan(m, B, bang::kModeSeed, &p) : get_plan(m, hgal, B, bang::kModeSeed, &p)) != BANG_OK)
        continue;
      if (p->G != sg) continue;
      if (m->scratch_seed.reserve(sizeof(float) * (size_t)std::max<int64_t>(p->out_total, 4)) != cudaSuccess ||
          m->scratch_grad.reserve(grad_scratch_bytes(p)) != cudaSuccess ||
          m->stage_out2.reserve(sizeof(float) * (size_t)B * m->P) != cudaSuccess) {
        cudaGetLastError();
        continue;
      }
      float t_min = 1e30f;
      for (int rep = 0; rep < 3; ++rep) {
        BANG_CUDA(cudaEventRecord(e0, st));
        BANG_CUDA(enqueue_grad(m, p, m->stage_theta.as<float>(), m->stage_out.as<double>(), m->scratch_seed.as<float>(),
                               m->scratch_grad.as<double>(), m->stage_out2.as<float>(), st, dgal));
        BANG_CUDA(cudaEventRecord(e1, st));
        BANG_CUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        BANG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        if (rep > 0) t_min = std::min(t_min, ms);
      }
      if (t_min < best_g) {
        best_g = t_min;
        best_sb = sb;
        best_rows = rows;
        best_sg = sg;
        best_minb = minb;
        best_sl = sl;
      }
    }
    best_t.seed_bands = best_sb;
    best_t.adj_G = best_rows;
    best_t.seed_G = best_sg;
    best_t.adj_minb = best_minb;
    best_t.seed_lanes = best_sl;
  } else {
    best_t.seed_bands = prior.seed_bands;
    best_t.adj_G = prior.adj_G;
    best_t.seed_G = prior.seed_G;
    best_t.adj_minb = prior.adj_minb;
    best_t.seed_lanes = prior.seed_lanes;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  m->plans.clear();
  m->tuned[skey] = best_t;
  return bang::check_faults(st);
}

}  // namespace
