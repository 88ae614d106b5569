// Internal interfaces between the host library (bang_api.cu) and the kernel translation units.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/bang.h"
#include "bang_check.cuh"

#ifndef BANG_NO_NVTX
#include <nvtx3/nvToolsExt.h>
#endif

namespace bang {

struct GalDev;
struct WorkItem;
struct ModelConst;

// NVTX range over one entry point (shown by nsys and usable as an ncu --nvtx filter); a
// push and a pop through a function pointer that does nothing when no tool is attached.
struct NvtxRange {
#ifndef BANG_NO_NVTX
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
#else
  explicit NvtxRange(const char*) {}
#endif
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// Gradient accumulator row: adjoints of the per-model constants (slots 0..23, the second
// disc's unused for one-disc models) and d logL / d v_sys (slot 24).
constexpr int kAdjSlots = 24;   // constant adjoints per adjoint work item (the adjoint kernel's accumulators)
constexpr int kVsysSlot = 24;   // index of d logL / d v_sys among a row's summed adjoints (from the forward seed pass)

// Forward kernel modes: logL only, model maps, adjoint seeds; kModeLogL2 is logL with two
// fine points per thread at 3 blocks per SM (80 registers), an alternative launch form the
// autotuner may choose for logL batches.
enum { kModeLogL = 0, kModeMaps = 1, kModeSeed = 2, kModeLogL2 = 3 };

// Arguments of the fused forward kernel.
struct FwdArgs {
  const float* theta;       // [B][P]
  int P;
  int halo_kind;            // 0 NFW, 1 Hernquist (used when consts is NULL)
  const GalDev* gals;
  const ModelConst* consts; // [B] decoded rows (NULL: warp 0 of the block decodes the item's row)
  ModelConst* consts_out;   // with consts NULL (may be NULL): each row's constants, stored by its first band
  double l10k;              // log10(3 / (4 pi 200 rho_c)), for the decode when consts is NULL
  const WorkItem* items;    // [n_items], items of one row contiguous, rows in order; NULL: implicit items,
                            // item i is band i % nb of row i / nb against galaxy gal_idx[i / nb]
  const int* gal_idx;       // implicit items: device [B] galaxy of each row (NULL = galaxy 0)
  int nb;                   // implicit items: bands per row
  const int* order;         // execution order of items (NULL = table order)
  int n_items;
  int* queue;               // dynamic item counter, zeroed before the launch (NULL = static striding)
  int G;                    // fine rows per block step (at least)
  int chunk_pts;            // > 0: a narrower galaxy's items take chunk_pts / W rows per step, as shared memory allows
  int col_lanes;            // separable stencil: 1 = several lanes per spaxel column share its taps
  double* partial;          // [n_items] chi^2 of each item (NaN for an out-of-domain row)
  float* maps;              // kModeMaps: model maps, row b at out_off[b]
  float* seed;              // kModeSeed: d logL / dF per spaxel, row b at out_off[b]
  double* vsys_partial;     // kModeSeed: [n_items] d logL / d v_sys of each work item
  const int64_t* out_off;   // [B] float offsets of each row's [4][ny][nx] block (NULL: b * out_stride)
  int64_t out_stride;       // floats per row's block when out_off is NULL
  const float* tables;      // radial tables, row b at b * table_stride (NULL: quadrature per point)
  int table_T;              // radii per table
  int64_t table_stride;     // floats per row's table
  // sizes for the checked build's index checks
  int B, n_gal;             // rows of the batch, galaxies of the model
  int64_t out_total;        // floats of maps / seed
};

// Arguments of the adjoint sweep.
struct AdjArgs {
  const float* theta;
  int P;
  const GalDev* gals;
  const ModelConst* consts; // [B] decoded rows
  const WorkItem* items;    // fine-row bands (j0/j1 hold fine padded rows [y0, y1)); NULL: implicit items,
                            // item i is fine rows [k rows_per_item, (k + 1) rows_per_item) of row i / nb,
                            // k = i % nb, against galaxy gal_idx[i / nb] (empty past the galaxy's last row)
  const int* gal_idx;       // implicit items: device [B] galaxy of each row (NULL = galaxy 0)
  int nb, rows_per_item;    // implicit items: bands per row and fine rows per band
  const int* order;
  int n_items;
  int* queue;               // dynamic item counter, zeroed before the launch (NULL = static striding)
  int G;                    // fine rows per block step (at least)
  int chunk_pts;            // > 0: a narrower galaxy's items take chunk_pts / W rows per step, as shared memory allows
  int col_lanes;            // separable stencil: 1 = several lanes per spaxel column share its taps
  const float* seed;        // d logL / dF at the spaxels, row b at out_off[b] (NULL: b * out_stride)
  const int64_t* out_off;
  int64_t out_stride;
  double* acc_partial;      // [n_items][kAdjSlots] float64 constant adjoints of each work item
  const float* tables;      // radial tables with slopes, row b at b * table_stride (NULL: quadrature)
  int table_T;
  int64_t table_stride;
  // sizes for the checked build's index checks
  int B, n_gal;             // rows of the batch, galaxies of the model
  int64_t seed_total;       // floats of seed
};

// Read-only view of a model's immutable device state (for entry points defined outside
// bang_api.cu).
struct ModelView {
  int device, n_gal, n_quad, n_discs, halo_kind, P, num_sms, smem_optin, bulge_table;
  const GalDev* h_gals;   // host copies (device pointers inside)
  const GalDev* d_gals;   // device array [n_gal]
};
bool model_view(const bang_model* m, ModelView* v);
// Records a message for bang_last_error() on this thread and returns s.
bang_status set_error(bang_status s, const char* fmt, ...);

int forward_threads();
size_t forward_smem_bytes(int L, int os, int nx, int W, int G, int psf2d, int table_T = 0);
const void* forward_kernel_ptr(int n_quad, int n_discs, int psf2d, int mode);
cudaError_t launch_forward(const FwdArgs& a, int n_quad, int n_discs, int psf2d, int mode, int grid, size_t smem,
                           cudaStream_t st);
cudaError_t launch_expand_rows(const float* theta, int P, int B, int n, float* theta_x, cudaStream_t st);
cudaError_t launch_sum_rows(const double* logL_x, const float* grad_x, int P, int B, int n, double* logL, float* grad,
                            cudaStream_t st);
// row_first NULL: row b's items are [b nb, (b + 1) nb); row_g NULL: galaxy 0.  With
// check_gal, a row whose galaxy index is outside [0, n_gal) gets logL = NaN.
cudaError_t launch_finalize(const double* partial, const int* row_first, const int* row_g, const GalDev* gals, int B,
                            int n_items, int n_gal, double* logL, cudaStream_t st, int nb = 1, int check_gal = 0);
// Execution order of implicit work items, longest first: items of rows whose galaxy has a
// lower rank (gal_rank[g], 0 = the most costly item) come first; n_rank ranks.  One block.
cudaError_t launch_order(const int* gal_idx, const int* gal_rank, int n_gal, int n_rank, int B, int nb, int* order,
                         cudaStream_t st);
cudaError_t upload_nodes_forward(const float* cm1, const float* lc, const float* ws, const float* wq);

int adjoint_threads();
size_t adjoint_smem_bytes(int L, int os, int nx, int G, int psf2d, int table_T = 0);
// Radial tables of the bulge (see bang_device.cuh): floats per row, and the table kernel
// (one block per row; slopes only when `derivs`).
int64_t table_row_floats(int T, int derivs);
cudaError_t launch_tables(const ModelConst* consts, const GalDev* gals, const int* row_g, int n_gal, int B, int n_quad,
                          int T, int derivs, float* tables, int64_t stride, cudaStream_t st);
// The adjoint kernel a launch uses (its blocks-per-SM bound depends on the radial-table mode).
// Blocks per SM the adjoint kernel instance is built for: `want` (3 or 4) for the one-disc
// quadrature form, otherwise its fixed value (3)
int adjoint_minb(int n_discs, int table, int want);
const void* adjoint_kernel_ptr(int n_quad, int n_discs, int psf2d, int table, int minb);
cudaError_t launch_adjoint(const AdjArgs& a, int n_quad, int n_discs, int psf2d, int minb, int grid, size_t smem,
                           cudaStream_t st);
// adj_row_first / row_first NULL: implicit items, adj_nb / nb per row; gal_idx (device, may be
// NULL) marks rows with a galaxy index outside [0, n_gal) as invalid (zero gradient).
cudaError_t launch_grad_out(const float* theta, int P, int n_discs, int halo_kind, int bulge_kind,
                            const double* acc_partial, const int* adj_row_first, const double* vsys_partial,
                            const int* row_first, int B, int n_items, int adj_items, float* grad, cudaStream_t st,
                            int adj_nb = 1, int nb = 1, const int* gal_idx = nullptr, int n_gal = 0);
size_t model_const_bytes();
// row_g NULL: galaxy 0 for every row; a galaxy index outside [0, n_gal) makes the row invalid.
double decode_l10k_host();   // log10(3 / (4 pi 200 rho_c)), the r_200 decode term's offset
cudaError_t launch_decode(const float* theta, int P, int n_discs, int halo_kind, const GalDev* gals, const int* row_g,
                          int n_gal, int B, ModelConst* out, cudaStream_t st);
cudaError_t upload_nodes_adjoint(const float* cm1, const float* lc, const float* ws, const float* wq);

// Checked build: each kernel translation unit's fault record, read and cleared (synchronous).
cudaError_t take_fault_forward(Fault* f);
cudaError_t take_fault_adjoint(Fault* f);
cudaError_t take_fault_plain(Fault* f);
// Checked build: synchronises st, reads and clears the fault records of every kernel
// translation unit, and returns BANG_E_BOUNDS (with the site in the error message) if one
// was set; BANG_OK otherwise and always in the normal build (which does not synchronise).
bang_status check_faults(cudaStream_t st);
// Checked build: one in-range check of i against n run on the device (the selftest site).
cudaError_t launch_check_selftest(long long i, long long n, cudaStream_t st);

// Float64 check path (bang_loglike_fp64): one galaxy as that path reads it.
struct Gal64 {
  int nx, ny, os, h, L, W, H;
  int psf2d;                // taps: 0 separable [L], 1 two-dimensional [L][L]
  double pitch, xoff, yoff; // kpc: x of padded fine column q is xoff + q pitch
  double norm_const;
  const double* taps;       // float64 taps (the float32 kernels' taps before rounding)
  const float* data;        // [4][ny][nx], the model's data maps
  const double* iv;         // [4][ny][nx], mask / delta^2 in float64
};
// Radial rule in float64: cosh t_k, tanh^2 t_k and the weights w_k of n_quad nodes.
struct Nodes64 {
  const double* ch;
  const double* th2;
  const double* w;
  int n;
};
size_t fp64_scratch_bytes(int N, int n);
// logL of one row (theta float64 [P] on the device, already inside the parameter domain).
cudaError_t launch_fp64_row(const double* theta, int nd, int halo_kind, const Nodes64& nodes, const Gal64& g,
                            void* scratch, double* logL, cudaStream_t st);

size_t plain_scratch_bytes(int N, int n);
int plain_launches_per_row();
cudaError_t launch_plain_row(const float* theta, int P, int n_quad, int n_discs, int halo_kind, const GalDev* d_gal,
                             const GalDev& h_gal, void* scratch, double* logL, cudaStream_t st);
cudaError_t upload_nodes_plain(const float* cm1, const float* lc, const float* ws, const float* wq);

}  // namespace bang
