// Index checks of the checked build (compiled with -DBANG_CHECKED; see build.py).
//
// compute-sanitizer is not available where this library is tested, so the kernels check
// their own indexes instead: BANG_IN(i, n, site) is true when 0 <= i < n.  When it is not,
// the first failing check of the launch records (site, i, n) in a device word of its
// translation unit and the caller skips the access; the kernel never traps.  After each
// call the host reads and clears the words (take_fault_*) and returns BANG_E_BOUNDS with
// the site's name.  In the normal build BANG_IN is the constant true and the index
// expressions are not evaluated, so the checks cost nothing.
#pragma once

#include <cuda_runtime.h>

namespace bang {

// Check sites (the value recorded is the site + 1; 0 means no fault).
enum CheckSite {
  kSiteSelftest = 0,
  kSiteFwdItem,        // forward: work item id against n_items
  kSiteFwdRow,         // forward: the item's row against B
  kSiteFwdGal,         // forward: the item's galaxy against n_gal
  kSiteFwdSmem,        // forward: end of the shared-memory layout against the dynamic size
  kSiteFwdStage,       // forward: points of a chunk against the stage
  kSiteFwdStencil,     // forward: stencil reads of a fine row against the row width W
  kSiteFwdTap,         // forward: tap index against L (or L * L)
  kSiteFwdSpaxel,      // forward: spaxel index against nx * ny
  kSiteFwdOut,         // forward: end of a row's maps / seeds against the output size
  kSiteFwdTable,       // forward: a row's radial table against the table buffer
  kSiteDecodeGal,      // decode / finalize / gradient: a row's galaxy against n_gal
  kSiteFinalizeItem,   // finalize / gradient: a row's items against n_items
  kSiteAdjItem,        // adjoint: work item id against n_items
  kSiteAdjRow,         // adjoint: the item's row against B
  kSiteAdjGal,         // adjoint: the item's galaxy against n_gal
  kSiteAdjSmem,        // adjoint: end of the shared-memory layout against the dynamic size
  kSiteAdjSeed,        // adjoint: seed reads against the row's seed block
  kSiteAdjLam,         // adjoint: spaxel-row buffer index against its size
  kSiteAdjTap,         // adjoint: tap index against L (or L * L)
  kSiteAdjV,           // adjoint: vertical-pass buffer index against G * nx
  kSiteAdjOut,         // adjoint: the item's accumulator slots against the partial buffer
  kSiteAdjTable,       // adjoint: a row's radial table against the table buffer
  kSitePlain,          // plain kernels: fine-grid, map and tap indexes
  kSiteTable,          // radial-table kernel: table index against the row's table
  kSiteCount
};

inline const char* check_site_name(int site) {
  static const char* names[kSiteCount] = {
      "selftest",        "forward item",      "forward row",     "forward galaxy",     "forward shared memory",
      "forward stage",   "forward stencil",   "forward tap",     "forward spaxel",     "forward output",
      "forward table",   "row galaxy",        "row items",       "adjoint item",       "adjoint row",
      "adjoint galaxy",  "adjoint shared memory", "adjoint seed", "adjoint spaxel rows", "adjoint tap",
      "adjoint vertical pass", "adjoint partials", "adjoint table", "plain kernels",   "table kernel"};
  return site >= 0 && site < kSiteCount ? names[site] : "unknown";
}

// Recorded fault: site + 1 (0 = none), the index and the bound.
struct Fault {
  long long site, index, bound;
};

#ifdef BANG_CHECKED
// One record per translation unit (no relocatable device code): the first fault wins.
static __device__ long long g_fault[3];

static __device__ __noinline__ void record_fault(int site, long long i, long long n) {
  if (atomicCAS(reinterpret_cast<unsigned long long*>(&g_fault[0]), 0ull, (unsigned long long)(site + 1)) == 0ull) {
    g_fault[1] = i;
    g_fault[2] = n;
  }
}

static __device__ __forceinline__ bool in_range(long long i, long long n, int site) {
  if (i >= 0 && i < n) return true;
  record_fault(site, i, n);
  return false;
}

#define BANG_IN(i, n, site) (::bang::in_range((long long)(i), (long long)(n), (site)))

// Reads this translation unit's record and clears it (synchronous).
#define BANG_DEFINE_FAULT_TAKER(fn)                                                  \
  cudaError_t fn(Fault* f) {                                                         \
    long long r[3] = {0, 0, 0};                                                      \
    cudaError_t e = cudaMemcpyFromSymbol(r, g_fault, sizeof(r));                     \
    f->site = r[0];                                                                  \
    f->index = r[1];                                                                 \
    f->bound = r[2];                                                                 \
    if (e == cudaSuccess && r[0]) {                                                  \
      const long long z[3] = {0, 0, 0};                                              \
      e = cudaMemcpyToSymbol(g_fault, z, sizeof(z));                                 \
    }                                                                                \
    return e;                                                                        \
  }
constexpr bool kChecked = true;
#else
#define BANG_IN(i, n, site) true
#define BANG_DEFINE_FAULT_TAKER(fn) \
  cudaError_t fn(Fault* f) {        \
    f->site = f->index = f->bound = 0; \
    return cudaSuccess;             \
  }
constexpr bool kChecked = false;
#endif

// Dynamic shared memory of the running launch, in bytes.
static __device__ __forceinline__ unsigned dynamic_smem_bytes() {
  unsigned r;
  asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(r));
  return r;
}

}  // namespace bang
