/* bang.h - C ABI of the GB300 galaxy-model log-likelihood library (libbang.so).
 *
 * The library evaluates, for a batch of parameter vectors, the log-likelihood of the
 * disc-galaxy model of Rigamonti et al. (2022), "Maximally informed Bayesian modelling of
 * disc galaxies", against integral-field maps of surface brightness B, line-of-sight
 * velocity v, velocity dispersion sigma and mass-to-light ratio M/L (Sec. 2.5.1, Eq. 18),
 * and its gradient with respect to the parameters.
 *
 * Model (Sec. 2.1-2.4): a spherical bulge of the Dehnen gamma family (Sec. 2.2; gamma = 1 is
 * the Hernquist bulge of Eq. 1, gamma = 2 the Jaffe bulge of Eq. B1) with its isotropic
 * projected dispersion (Eq. 6) from a fixed n_quad-node radial quadrature, one or two
 * razor-thin exponential discs (Eqs. 7-12) with the Freeman circular velocity
 * v^2 = (2 G M_d / R_d) y^2 [I0 K0 - I1 K1](y), y = r / (2 R_d) (Eq. 9, Binney & Tremaine
 * form), and an NFW halo given by M200 and concentration c.  The four light-weighted
 * observables (Eqs. 13-15 and 19) are evaluated on an os x os oversampled sub-grid of every
 * spaxel, padded by the PSF half-width, convolved with the normalised PSF of Eq. 21
 * (Gaussian, or Moffat), averaged per spaxel, and compared with the data through Gaussian
 * terms: logL = -chi^2 / 2 - sum ln(sqrt(2 pi) delta).
 *
 * Parameter vector theta (float32, row-major [B][P], P = 15 for one disc, 19 for two):
 *   0 x0, 1 y0 [kpc], 2 P.A. [rad], 3 i [rad, 0 <= i < pi/2],
 *   4 log10 Mb [Msun], 5 log10 Rb [kpc], 6 gamma [0 <= gamma < 3],
 *   7 log10 Md1, 8 log10 Rd1, 9 k1 [|k| <= 1], 10 (M/L)b, 11 (M/L)d1 [> 0],
 *   12 log10 M200 (NFW) or log10 M_h (Hernquist halo), 13 c [> 0] (NFW) or log10 R_h [kpc]
 *   (Hernquist halo), 14 v_sys [km/s],
 *   15 log10 Md2, 16 log10 Rd2, 17 k2, 18 (M/L)d2   (two-disc models only).
 * A row that is not finite or lies outside those ranges gets logL = -INFINITY and a zero
 * gradient; that is not an error (samplers propose such points).
 *
 * Sky grid: spaxel (i, j) is centred at x = (i - (nx-1)/2) s, y = (j - (ny-1)/2) s arcsec
 * (s = spaxel_arcsec); maps are stored [4][ny][nx] with i fastest, channels B [Lsun/pc^2],
 * v [km/s], sigma [km/s], M/L [Msun/Lsun].
 *
 * Pointers: every array argument of a compute entry point may be host memory (pageable or
 * pinned) or device memory of the model's device; the library asks the CUDA runtime which.
 * Host arrays are staged through library-owned device buffers on the given stream and the
 * call then returns only after the results are back in host memory.  With device arrays the
 * call is asynchronous on `stream` (a cudaStream_t passed as void*, NULL = legacy default).
 *
 * Errors: functions return a bang_status; on failure bang_last_error() gives a message
 * (per calling thread).  No entry point aborts the process.
 */
#ifndef BANG_H
#define BANG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bang_model bang_model; /* opaque; owns all device state of one model */

typedef enum {
  BANG_OK = 0,
  BANG_E_INVALID_ARG = 1, /* null pointer, bad size, index out of range, bad descriptor */
  BANG_E_CUDA = 2,        /* a CUDA runtime call failed; see bang_last_error() */
  BANG_E_OOM = 3,         /* device or host allocation failed */
  BANG_E_UNSUPPORTED = 4, /* option not implemented (e.g. Hernquist halo kind) */
  BANG_E_TIMEOUT = 5,     /* a bounded device-side wait gave up (reserved: no kernel of this
                             library waits on another block, so none is returned) */
  BANG_E_BOUNDS = 6       /* checked build only: a kernel's index check failed (see
                             bang_checked_build); bang_last_error() names the check site */
} bang_status;

/* One observed galaxy (Sec. 3.1).  The arrays are read during bang_model_create only and
 * are copied to the device; the caller keeps ownership. */
typedef struct {
  int nx, ny;               /* spaxels along x and y, >= 1 */
  int oversample;           /* os >= 1: os x os sub-points per spaxel */
  double spaxel_arcsec;     /* spaxel size s > 0 */
  double kpc_per_arcsec;    /* distance scale (53 Mpc -> 0.25695) */
  int psf_kind;             /* 0 Gaussian (Eq. 21), 1 Moffat */
  double psf_fwhm_arcsec;   /* >= 0; 0 means no PSF.  Window half-width h = floor(3 sigma os / s)
                               fine pixels with sigma = FWHM / 2.35482 for both kinds */
  double moffat_beta;       /* Moffat exponent (> 0), ignored for the Gaussian */
  const float *data;        /* host, [4][ny][nx]: B, v, sigma, M/L */
  const float *err;         /* host, [4][ny][nx]: delta > 0 where the mask is set */
  const uint8_t *mask;      /* host, [4][ny][nx], nonzero = used; NULL = all used */
} bang_galaxy_desc;

/* bits of bang_model_opts.psf_mode (no counterpart names in the paper) */
#define BANG_PSF_CIRCLE 1
#define BANG_PSF_CENTRE 2
#define BANG_PSF_FLUX 4

typedef struct {
  int n_discs;     /* 1 or 2 */
  int bulge_kind;  /* 0: Dehnen gamma family, projected by the radial quadrature (default).
                      1: Hernquist (gamma = 1, Eqs. 1-6), 2: Jaffe (gamma = 2, Eqs. B1-B5): the
                      projected density and dispersion from float32 fits of the closed forms'
                      universal profiles (about 2e-7 relative); the gamma slot of theta is then
                      not used and its gradient is 0.  Not with bulge_table. */
  int halo_kind;   /* 0: NFW (M200, c); 1: Hernquist (M_h, R_h), the paper's halo (Sec. 2.2):
                      v^2 = G M_h r / (r + R_h)^2, Eq. 2 with the halo's mass and radius */
  int n_quad;      /* radial quadrature nodes: 64 or 128 */
  int psf_mode;    /* 0 (default): square window |dx|, |dy| <= 3 sigma, each spaxel the mean over its
                      os x os fine points of the PSF-weighted average around each, and B, v,
                      sigma and <L/M> convolved each on its own (Sec. 3.1).  Or any sum of:
                      BANG_PSF_CIRCLE - the window is the circle of radius 3 sigma (Eq. 21);
                      BANG_PSF_CENTRE - each spaxel is the PSF-weighted average of the fine
                        points around its centre (App. A), without the os x os mean;
                      BANG_PSF_FLUX - B, B v, B (sigma^2 + v^2) and the surface mass are
                        convolved; v = C1/C0, sigma^2 = C2/C0 - v^2, M/L = C3/C0 per spaxel. */
  int bulge_table; /* 0: the radial quadrature at every fine point (default).  N in [256, 4096]:
                      per parameter vector, the same n_quad-node quadrature at N radii spaced
                      uniformly in log R between the 1e-6 kpc floor and the farthest fine point,
                      then 4-point Lagrange interpolation in log R of each fine point's bulge
                      density and dispersion (of values and log-ratios, so float32 keeps ~1e-7);
                      the interpolation error is ~1e-9 relative at N = 1024.  Not available to
                      bang_loglike_batch_noalloc and bang_loglike_plain (BANG_E_UNSUPPORTED). */
} bang_model_opts;

/* Creates a model for n_gal galaxies on CUDA device `device`: copies data, errors, masks
 * and PSF taps to the device (allocation happens once, as in App. A) and precomputes the
 * normalisation constant of each galaxy.  *out receives the handle.  Synchronous. */
bang_status bang_model_create(const bang_galaxy_desc *gal, int n_gal, const bang_model_opts *opts,
                              int device, bang_model **out);

/* Frees all device and host state of the model.  NULL is accepted.  Synchronises. */
bang_status bang_model_destroy(bang_model *m);

/* Caps the device memory the model may allocate while serving calls (work-item tables,
 * staging of host arrays, gradient and table scratch), beyond the resident data copied by
 * bang_model_create; bytes = 0 removes the cap.  A call that would go over the cap
 * returns BANG_E_OOM before launching anything and leaves the buffers it already had.
 * Also the host-side way to test allocation failure. */
bang_status bang_model_set_scratch_limit(bang_model *m, int64_t bytes);

/* Device bytes the model currently holds as call scratch; -1 for a NULL model. */
int64_t bang_model_scratch_bytes(const bang_model *m);

/* Parameters per row: 15 (one disc) or 19 (two discs); -1 for a NULL model. */
int bang_model_nparams(const bang_model *m);

/* Number of galaxies of the model; -1 for a NULL model. */
int bang_model_ngalaxies(const bang_model *m);

/* PSF window half-width h (fine pixels) of galaxy g, or -1 if g is out of range. */
int bang_model_psf_halfwidth(const bang_model *m, int g);

/* logL[b] (float64) of row b of theta ([B][P] float32) against galaxy gal_idx[b] (Eq. 18 on
 * the model of Sec. 2.1-2.4).  One persistent launch handles all rows, whatever their grid
 * sizes (Sec. 2.5, App. A).  gal_idx: int32 [B] in [0, n_gal), or NULL for galaxy 0 for every
 * row, in either memory:
 *  - a HOST array: the host reads it to build the launch's work items (cached per distinct
 *    gal_idx contents and B); an index out of range returns BANG_E_INVALID_ARG;
 *  - a DEVICE array of the model's device: nothing is read on the host and the call stays
 *    asynchronous (no host synchronisation once the batch size has been seen).  The kernels
 *    derive each row's work from its galaxy; the launch is sized for every galaxy of the
 *    model (shared memory, bands for the tallest grid), and the model's galaxies must share
 *    one PSF kind (Gaussian, or two-dimensional taps), else BANG_E_UNSUPPORTED.  A row whose
 *    index is out of range gets logL = NaN (and a zero gradient); the other rows are
 *    unaffected.  Results equal the host-array path's bit for bit.
 * Device memory of another device gives BANG_E_INVALID_ARG. */
bang_status bang_loglike_batch(bang_model *m, const float *theta, const int32_t *gal_idx, int B,
                               double *logL, void *stream);

/* As bang_loglike_batch (gal_idx host or device memory as described there), plus
 * grad[b][p] = d logL[b] / d theta[b][p] (float32, [B][P]): the gradient of Eq. 18's
 * log-likelihood through the discrete model of Sec. 2.1-2.4 and the PSF and binning of
 * Eq. 21, by a hand-written adjoint that re-evaluates the radial quadrature instead of
 * storing it.  (The paper samples without gradients; this serves gradient-based samplers
 * and optimisers the same likelihood.) */
bang_status bang_loglike_grad_batch(bang_model *m, const float *theta, const int32_t *gal_idx, int B,
                                    double *logL, float *grad, void *stream);

/* Model maps for every row: maps[b] is [4][ny][nx] float32 of galaxy gal_idx[b] (B, v_los +
 * v_sys, sigma_los, M/L = 1/<L/M>); rows are packed back to back, each with its own galaxy's
 * size.  Out-of-domain rows get NaN maps.  gal_idx must be host memory (the packing depends
 * on it; a device array gives BANG_E_UNSUPPORTED). */
bang_status bang_model_maps(bang_model *m, const float *theta, const int32_t *gal_idx, int B, float *maps,
                            void *stream);

/* Total floats bang_model_maps writes for this gal_idx (host memory, may be NULL) and B;
 * -1 for a NULL model, an index out of range or a device gal_idx. */
int64_t bang_model_maps_size(const bang_model *m, const int32_t *gal_idx, int B);

/* The paper's execution form (Alg. 2 of App. A): for each row, a serial chain of one kernel
 * per task (coordinates, bulge, circular velocities, discs, combination, PSF + binning,
 * chi-square), 64 threads per block, intermediate arrays in device memory.  Same model and
 * arithmetic as bang_loglike_batch; used as the comparison baseline.  A device gal_idx is
 * copied to the host first (this entry point schedules row by row on the host). */
bang_status bang_loglike_plain(bang_model *m, const float *theta, const int32_t *gal_idx, int B,
                               double *logL, void *stream);

/* One galaxy observed on several spaxel grids (the paper's tool takes maps with different
   numbers of pixels, Sec. 3.2): galaxies grids[0 .. n_grids) of the model are grids of the
   same galaxy (sky coordinates centred on the same point), each usually masked to the maps
   it holds (e.g. B on a fine photometric grid, v and sigma on a coarse kinematic one).
   Every parameter vector is evaluated against each of them:
     logL[b] = sum_k logL(theta_b, grids[k]),   grad[b] = sum_k d logL(theta_b, grids[k]) / d theta.
   theta [B][P] f32, logL [B] f64 and grad [B][P] f32 (NULL: no gradient) are host or device
   pointers; grids is a host array of n_grids galaxy indices (repeats allowed).  The B x
   n_grids rows run as one batch of bang_loglike_batch / bang_loglike_grad_batch; the sums
   are formed by a kernel.  Returns BANG_E_INVALID_ARG for null pointers, B < 1, n_grids < 1
   or an index out of range; scratch of about B x n_grids x (4 P + 8) bytes is kept by the
   model between calls. */
bang_status bang_loglike_grids(bang_model *m, const float *theta, int B, const int32_t *grids, int n_grids,
                               double *logL, float *grad, void *stream);

/* No-allocation variant of bang_loglike_batch.  The paper has no counterpart: this entry
 * point exists for callers that must not allocate device memory while they run.
 *
 * bang_loglike_batch allocates per-batch scratch (its work-item table and per-item chi^2
 * partial sums) with cudaMalloc the first time it meets a batch shape, and stages host
 * arrays through library-owned buffers.  Some callers cannot allow that: a program whose
 * device memory is handed in full to another allocator (for example a framework's caching
 * allocator that has reserved the GPU), a sampler loop that cannot take the device-wide
 * synchronisation cudaMalloc and cudaFree may cause, or an application that must know the
 * library's device footprint before it starts.  This call makes no cudaMalloc, cudaFree or
 * other allocating call.  Its scratch is one fixed array of about 1.2 MB compiled into the
 * library's device code; every GPU that loads the library holds it until the process exits.
 *
 * theta [B][P] float32 and logL [B] float64 must be device memory of the model's device
 * (host pointers give BANG_E_INVALID_ARG; there is no staging).  gal_idx is a HOST array
 * [B] of galaxy indices or NULL (galaxy 0 for every row); it is copied on `stream`, so a
 * pinned gal_idx must stay unchanged until the stream has passed this call.  Under stream
 * capture that copy becomes a node of the graph: gal_idx must then be pinned, and every
 * replay reads the array again at the time it runs (its contents are validated only when
 * the call is made).  B is at most
 * 32768 (the size the scratch was built for); a larger B returns BANG_E_INVALID_ARG and
 * launches nothing.  Each row is one work item (no bands), so logL equals
 * bang_loglike_batch's result up to the order of float64 additions.
 *
 * The first call on a device looks up the scratch's device address (cudaGetSymbolAddress,
 * with that device current) and keeps it; make that first call before any stream capture.
 * All calls share the one scratch array, which keeps what the last call wrote; every entry
 * a call reads is written earlier in the same call, so nothing has to be cleared between
 * calls.  Two calls that overlap on the GPU (two streams, or two host threads) race on the
 * scratch: serialise them.  Asynchronous on `stream`. */
bang_status bang_loglike_batch_noalloc(bang_model *m, const float *theta, const int32_t *gal_idx, int B,
                                       double *logL, void *stream);

/* Float64 check path: logL of B rows computed with every step in float64 (Sec. 2.1-2.4,
 * Eq. 18, Eq. 21) in the plainest form (one kernel per step: fine points, spaxels, sum),
 * on the same discretisation as bang_loglike_batch: padded fine grid, the fixed radial
 * rule in float64 (n_quad nodes, t in [0, 16]), the float64 PSF (x) box taps, 1/delta^2 in
 * float64, the data maps as given.  The disc velocity uses the modified Bessel functions
 * themselves up to r / (2 R_d) = 25 and their products' large-argument expansion beyond.  For comparisons with a float64 reference,
 * not for speed.  theta [B][P] float64 and logL [B] float64 may each be host or device
 * memory; gal_idx is an array [B] (host memory, or device memory copied to the host) or
 * NULL.  Rows outside the parameter domain give
 * -inf.  Supported: bulge_kind 0 (radial rule; bulge_table is ignored), psf_mode without
 * BANG_PSF_FLUX; otherwise BANG_E_UNSUPPORTED.  Synchronous on `stream`. */
bang_status bang_loglike_fp64(bang_model *m, const double *theta, const int32_t *gal_idx, int B, double *logL,
                              void *stream);

/* Chooses the launch parameters of bang_loglike_batch (kernel form, fine rows per block
 * step, spaxel-row bands per row, lanes per spaxel column of the separable stencil) for
 * batches of B rows by timing candidates on the device;
 * the choice is cached in the model.
 * With a host gal_idx (or NULL: galaxy 0 for every row) it applies to later calls with that
 * same gal_idx and B; with a device gal_idx (read here, this call being synchronous) it
 * applies to every later call of B rows with a device gal_idx. */
bang_status bang_model_tune(bang_model *m, const int32_t *gal_idx, int B);

/* As bang_model_tune, and then the launch parameters of bang_loglike_grad_batch for the same
 * batches (the forward seed pass's spaxel-row bands, fine rows per block step and stencil
 * lanes per spaxel column, the adjoint's fine rows per work item and, for the one-disc
 * model without the radial table, the adjoint's blocks per SM, 3 or 4), timed on whole
 * logL + gradient calls.  Synchronous; a gradient call costs a
 * few times a logL call, so this takes correspondingly longer. */
bang_status bang_model_tune_grad(bang_model *m, const int32_t *gal_idx, int B);

/* The launch shape bang_loglike_batch (grad = 0) or bang_loglike_grad_batch (grad = 1)
 * would use for (gal_idx, B), after any bang_model_tune: info[13] (host) receives
 *   0 fine rows per block step of the forward kernel, 1 spaxel-row bands per batch row,
 *   2 forward blocks per SM, 3 forward grid, 4 forward work items, 5 forward dynamic shared
 *   memory per block (bytes), 6 fine rows per adjoint work item, 7 adjoint grid,
 *   8 adjoint work items (6-8 zero when grad = 0), 9 1 when the work items are derived on
 *   the device (device gal_idx), else 0, 10 fine points per thread of the forward kernel
 *   (2: the two-point form the autotuner may choose for logL batches, 3 blocks per SM),
 *   11 adjoint blocks per SM (zero when grad = 0), 12 1 when the forward kernel's separable
 *   stencil gives each spaxel column several lanes (an autotuner choice), else 0.
 * Builds (and caches) the batch's plan like a call; launches nothing.  Synchronous.  For
 * diagnostics (the paper has no counterpart). */
bang_status bang_model_launch_info(bang_model *m, const int32_t *gal_idx, int B, int grad, int32_t *info);

/* Message of the last failed call on this thread ("" if none). */
const char *bang_last_error(void);

/* 1 when this library is the checked build, else 0.  In the checked build every kernel
 * checks the indexes it computes (work items, rows, galaxies, shared-memory layout, stencil
 * and tap indexes, spaxels, output blocks, radial tables) against the sizes of their
 * buffers; an index out of range is not used, and the first such index of a call is
 * recorded on the device (site, index, bound) instead of trapping.  Each compute entry
 * point then synchronises its stream after its launches, reads and clears the records, and
 * returns BANG_E_BOUNDS with the site in bang_last_error().  The records are per library,
 * not per model: run checked calls one at a time.  The normal build compiles the checks
 * out and never returns BANG_E_BOUNDS. */
int bang_checked_build(void);

/* Checked build: one device-side index check of `index` against [0, bound) on `device`,
 * reported like a kernel's (BANG_E_BOUNDS when out of range; nothing is read or written at
 * the index), so that the recording and reporting path can be tested without an
 * out-of-range access.  Synchronous.  The normal build returns BANG_E_UNSUPPORTED. */
bang_status bang_check_selftest(int device, long long index, long long bound);

#ifdef __cplusplus
}
#endif

#endif /* BANG_H */
