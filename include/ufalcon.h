/*
 * ufalcon.h -- C ABI of the GB300 lightcone library (libufalcon_gb300.so).
 *
 * The library computes the data-parallel hot path of the UFalcon
 * multi-lens-plane method (Sgier, Refregier, Amara & Nicola, "Fast
 * Generation of Covariance Matrices for Weak Lensing"):
 *
 *   particles of nested simulation boxes, observer at the centre (Sec. 2.4)
 *     -> comoving shell (Eq. 8) and HEALPix RING pixel (Sec. 2.4)
 *     -> per-shell count maps n_p(pix, Delta chi_b)          (Eq. 5)
 *     -> Born-approximation convergence map kappa            (Eq. 2, 3, 6)
 *     -> moments, variance of the variance and a PDF         (Eq. 12, 13, Sec. 3.3)
 *     -> covariance and correlation over realisations        (Eq. 10, 11)
 *   plus the adjoint of kappa's statistics with respect to (Omega_m, h, and
 *   the n(z) parameters alpha, beta, z0), with the counts held fixed.
 *
 * Conventions shared by every call:
 *  - Pointers named *_dev are device memory of the context's device;
 *    all others are host memory.  The caller owns every buffer it passes;
 *    the library never frees or retains them after the call returns.
 *  - Device work is enqueued on the context's stream (ufc_set_stream) and is
 *    asynchronous unless a call says it synchronises.  Host outputs of a
 *    call that enqueues device work are valid when the call returns.
 *  - Positions are FP32 x,y,z triples (array of structures, 12 bytes per
 *    particle) in the box's coordinates, lengths in Mpc/h (or Mpc when
 *    ufc_cosmo.units_mpc_over_h = 0).
 *  - Count maps are int32 [nshell][12*nside^2], shell-major, RING order.
 *  - Every call returns UFC_OK or an error status; ufc_last_error() then
 *    holds a one-line message.  Invalid arguments never reach the GPU.
 *  - A context is not thread-safe: use one per host thread.
 */
#ifndef UFALCON_H
#define UFALCON_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define UFC_MAX_SHELLS 256     /* shells per map                         */
#define UFC_MAX_NSIDE 8192     /* HEALPix resolution (power of two)      */
#define UFC_MAX_REPLICATE 8    /* periodic image layers per axis         */
#define UFC_NMOMENTS 10        /* length of the moments vector           */

typedef enum {
  UFC_OK = 0,
  UFC_ERR_ARG = 1,          /* invalid argument (nothing was enqueued)    */
  UFC_ERR_CUDA = 2,         /* a CUDA runtime call failed                 */
  UFC_ERR_ALLOC = 3,        /* device workspace could not be allocated    */
  UFC_ERR_TIMEOUT = 4,      /* a device-side bounded wait ran out         */
  UFC_ERR_UNSUPPORTED = 5,  /* valid request this build does not handle   */
  UFC_ERR_CAPACITY = 6,     /* a caller-sized or fixed buffer is too small */
  UFC_ERR_INTERNAL = 7      /* an index test of a checked build failed    */
} ufc_status;

typedef struct ufc_ctx ufc_ctx;

/* Flat LambdaCDM cosmology (the paper uses h = 0.7, Omega_m = 0.276, Table 1).
 * E(z) = sqrt(Omega_m (1+z)^3 + 1 - Omega_m).  units_mpc_over_h = 1: lengths
 * in Mpc/h, c/H0 = 2997.92458 Mpc/h; 0: lengths in Mpc, c/H0 = 2997.92458/h.
 * density_volume selects the density factor F_b of Eq. 6 and 7: 0 (as
 * printed) F_b = N_pix V / (4 pi N chi_b^2) at the shell's lower edge;
 * 1 its average over the shell volume,
 * F_b = 3 N_pix V Delta chi_b / (4 pi N (chi_{b+1}^3 - chi_b^3)),
 * for which the expected kappa and delta of a uniform field are exactly 0. */
typedef struct {
  double omega_m;
  double h;
  int32_t units_mpc_over_h;
  int32_t density_volume;
} ufc_cosmo;

/* One simulation box of the nesting scheme (Sec. 2.4).  obs is the observer
 * (the paper places it at the box centre).  The box owns the shells
 * [shell_lo, shell_hi): a particle of this box is counted only when its
 * radius falls in one of them.  n_total is the particle count of the whole
 * simulation box, which sets the mean density rho = m_p N / V of Eq. 6.
 * replicate = R adds the periodic images (i,j,k) in [-R,R]^3 (the paper
 * avoids replication; R = 0 reproduces that). */
typedef struct {
  double L;
  double obs[3];
  int64_t n_total;
  int32_t shell_lo;
  int32_t shell_hi;
  int32_t replicate;
} ufc_box;

/* Lensing source (Sec. 2.3-2.4): kind 0 = single plane at z_s (Eq. 3);
 * kind 1 = n(z) proportional to z^alpha exp(-(z/z0)^beta) on [0, z_max]. */
typedef struct {
  int32_t kind;
  double z_s;
  double alpha, beta, z0, z_max;
} ufc_source;

/* ---- context -------------------------------------------------------------- */

/* Creates a context on CUDA device `device`; the context owns its device
 * workspace, which grows on demand and is freed by ufc_destroy. */
ufc_status ufc_create(ufc_ctx **ctx, int32_t device);
ufc_status ufc_destroy(ufc_ctx *ctx);
/* Sets the CUDA stream (a cudaStream_t, NULL = legacy default stream). */
ufc_status ufc_set_stream(ufc_ctx *ctx, void *stream);
/* Waits for all work enqueued by this context; reports device-side errors:
 * UFC_ERR_TIMEOUT when a bounded wait of the fast binning stage (on its
 * particle copies) ran out since the last report, in which case that
 * binning call's counts are incomplete; else UFC_ERR_INTERNAL when an index
 * test failed since the last report (checked builds, and
 * ufc_check_selftest).  The context stays usable. */
ufc_status ufc_synchronize(ufc_ctx *ctx);
/* Self-test of the device-side failure report (no counterpart in the
 * paper): one kernel waits on a barrier that nothing completes, gives up
 * after `limit` polls (1 <= limit <= 2^28) and reports it; the next
 * ufc_synchronize returns UFC_ERR_TIMEOUT.  Faults nothing and leaves the
 * context usable.  Asynchronous. */
ufc_status ufc_wait_selftest(ufc_ctx *ctx, int64_t limit);
/* Message of the last error on this context ("" if none). */
const char *ufc_last_error(const ufc_ctx *ctx);

/* Index tests.  A library built with -DUFC_CHECKED (build.py checked=True,
 * libufalcon_gb300_checked.so; the Python binding loads it when the
 * environment sets UFC_CHECKED=1) tests the computed indices of the binning
 * kernels (count-map cells, buckets, bucket groups, scatter destinations,
 * histogram offsets) and of the batched kernel's count maps before each
 * access; a failed test records its site, index and bound, skips the access
 * and lets the kernel finish.  ufc_synchronize then returns
 * UFC_ERR_INTERNAL with the first failure in ufc_last_error.  Other builds
 * compile the tests away.  The record is one per device, shared by the
 * contexts on it.  ufc_check_selftest fails one test on purpose (index
 * against bound, in every build; nothing is accessed) so that the report
 * path can be exercised.  Asynchronous. */
ufc_status ufc_check_selftest(ufc_ctx *ctx, int64_t index, int64_t bound);
/* Device bytes the context holds (workspace, counters and the workspace of
 * its batched-call lanes) in *bytes.  Host only; enqueues nothing. */
ufc_status ufc_workspace_bytes(const ufc_ctx *ctx, int64_t *bytes);
/* Pre-allocates the workspace of a ufc_bin call with up to two boxes and up
 * to n_max particle images (particles times images) at (nside, nshell), so
 * that such calls allocate nothing. */
ufc_status ufc_reserve(ufc_ctx *ctx, int32_t nside, int32_t nshell, int64_t n_max);

/* Kernel timing (tracing; the paper has no counterpart).  While enabled,
 * each kernel the library launches is bracketed by CUDA events on the
 * context's stream (a few microseconds of overhead per launch). */
ufc_status ufc_profile_enable(ufc_ctx *ctx, int32_t on);
/* Synchronises, then reports the launches recorded since the last read,
 * aggregated by kernel name: up to `max` entries of names (char[max][32],
 * NUL-terminated), total milliseconds ms[max] and launch counts
 * launches[max]; *n_out receives the number of distinct kernels (which may
 * exceed max).  Clears the record. */
ufc_status ufc_profile_read(ufc_ctx *ctx, int32_t max, char *names, double *ms,
                            int64_t *launches, int32_t *n_out);

/* ---- host cosmology (Eq. 1-3, Eq. 6, Eq. 8) -------------------------------- */

/* Comoving distances chi(z) = (c/H0) int_0^z dz'/E(z') of the nshell+1 shell
 * edges z_edges (Delta chi_b of Sec. 2.4).  z_edges must be increasing, >= 0. */
ufc_status ufc_chi_edges(const ufc_cosmo *cosmo, const double *z_edges,
                         int32_t nshell, double *chi_out);
/* Inverse of chi(z) for n values (for shells of equal comoving thickness). */
ufc_status ufc_z_of_chi(const ufc_cosmo *cosmo, const double *chi, int32_t n,
                        double *z_out);
/* Coefficients of kappa_p = sum_b A_b n_bp - C (Eq. 6):
 *   A_b = 3/2 Omega_m W_b (H0/c) F_b,  F_b = N_pix V_k / (4 pi N_k chi_b^2),
 *   B_b = 3/2 Omega_m W_b (H0/c) Delta chi_b,  C = sum_b B_b,
 * with W_b from Eq. 3 (plane) or its n(z) average, chi_b the shell's lower
 * edge (or F_b over the shell volume, ufc_cosmo.density_volume) and
 * (V_k = L^3, N_k = n_total) of the box owning shell b.  Every shell
 * must be owned by exactly one box and z_edges[0] > 0.
 * Optional dA [5][nshell] and dC [5] receive the derivatives with respect to
 * theta = (Omega_m, h, alpha, beta, z0) (NULL to skip). */
ufc_status ufc_kappa_coeffs(const ufc_cosmo *cosmo, const ufc_box *boxes,
                            int32_t nbox, const double *z_edges, int32_t nshell,
                            int32_t nside, const ufc_source *src, double *A,
                            double *B, double *C, double *dA, double *dC);

/* Coefficients of the overdensity map of Eq. 7,
 *   delta_p = sum_b [F_b n_bp - Delta chi_b] / sum_b Delta chi_b
 *           = sum_b A_b n_bp - C,   A_b = F_b / sum_b Delta chi_b,  C = 1,
 * with F_b the density factor of Eq. 6 (ufc_kappa_coeffs, including the
 * density_volume reading; (V_k, N_k) of the owning box).  The map,
 * its moments and PDF come from ufc_kappa_stats with these coefficients,
 * gradients from ufc_kappa_backward with dA [5][nshell] and dC [5] (theta as
 * for kappa; the n(z) parameters do not enter, their columns are 0).
 * Arguments and errors as for ufc_kappa_coeffs (no source). */
ufc_status ufc_delta_coeffs(const ufc_cosmo *cosmo, const ufc_box *boxes,
                            int32_t nbox, const double *z_edges, int32_t nshell,
                            int32_t nside, double *A, double *C, double *dA,
                            double *dC);

/* ---- binning (Eq. 5, Eq. 8, HEALPix pixelisation) ------------------------- */

/* Shell and pixel of every particle of one box without replication:
 * keys_dev[i] = shell * 12 nside^2 + pix, -1 when the radius is outside the
 * box's shells, -2 when the particle is invalid (non-finite, or r == 0).
 * chi_edges: nshell+1 increasing FP64 radii (host).  Membership is
 * chi_b <= r < chi_{b+1} (Eq. 8 read half-open); the pixel is the RING pixel
 * of the fixed FP64 procedure documented with the library (bit-exact). */
ufc_status ufc_keys(ufc_ctx *ctx, const float *xyz_dev, int64_t n,
                    const ufc_box *box, const double *chi_edges, int32_t nshell,
                    int32_t nside, int32_t *keys_dev);

#define UFC_BIN_ACCUMULATE 1   /* add to counts_dev instead of overwriting */
#define UFC_BIN_FORCE_DIRECT 2 /* L2-atomic path regardless of map size      */
#define UFC_BIN_FORCE_DENSE 4  /* dense-key path (needs nside >= 64, no
                                  replication, 16-byte aligned counts)       */

/* Count maps of one lightcone made of nbox boxes: box k's particles are
 * xyz_dev[k] (n[k] of them).  counts_dev [nshell][12 nside^2] is overwritten
 * (or added to with UFC_BIN_ACCUMULATE).  nshell * 12 nside^2 < 2^31 (the
 * paper's 140 shells at Nside 1024 included).
 * The library picks the output path (L2 atomics for maps up to 32 MB, the
 * dense-key scatter and shared-memory histograms above); the FORCE flags
 * override the choice (used by the autotuner).  Results are identical. */
ufc_status ufc_bin(ufc_ctx *ctx, const float *const *xyz_dev, const int64_t *n,
                   const ufc_box *boxes, int32_t nbox, const double *chi_edges,
                   int32_t nshell, int32_t nside, int32_t flags,
                   int32_t *counts_dev);
/* ufc_bin with the positions in host memory (end-to-end use; the paper's
 * particles arrive from the simulation's output on the host).  Box k's
 * xyz_host[k] (n[k] particles, 12 bytes each) is copied into a device
 * staging buffer owned by the context (grown on demand, kept for later
 * calls) in chunks of 2^25 particles on a second stream of the
 * context; the fast stage of each chunk starts on the context stream as
 * soon as the chunk has landed, so transfer and binning overlap.  Results
 * are identical to ufc_bin's.  Page-locked host memory (cudaHostAlloc,
 * cudaHostRegister) lets the copies run asynchronously; pageable memory
 * works, the copies then serialise with the host.  The host buffers must
 * not change until the call's work has finished (ufc_synchronize).
 * UFC_ERR_UNSUPPORTED while the context stream is capturing a graph.
 * Asynchronous otherwise, like ufc_bin. */
ufc_status ufc_bin_host(ufc_ctx *ctx, const float *const *xyz_host, const int64_t *n,
                        const ufc_box *boxes, int32_t nbox, const double *chi_edges,
                        int32_t nshell, int32_t nside, int32_t flags,
                        int32_t *counts_dev);
/* ufc_bin from host memory for particle sets of any size (beyond device
 * memory): each box's particles are cut into chunks of at most `chunk`
 * particles, copied into one of two device buffers owned by the context
 * while the previous chunk is binned from the other, and every chunk is
 * binned into counts_dev like a ufc_bin call (accumulating after the
 * first; UFC_BIN_ACCUMULATE adds the first chunk too).  Device memory held:
 * 2 x 12 chunk bytes plus one chunk's binning workspace.  Counts equal
 * ufc_bin's.  Larger chunks amortise the per-chunk work (at large maps each
 * chunk's histogram pass touches the whole map).  ufc_bin_info then
 * describes the last chunk.  Host buffers as for ufc_bin_host.
 * UFC_ERR_UNSUPPORTED while the context stream is capturing. */
ufc_status ufc_bin_host_stream(ufc_ctx *ctx, const float *const *xyz_host,
                               const int64_t *n, const ufc_box *boxes,
                               int32_t nbox, const double *chi_edges,
                               int32_t nshell, int32_t nside, int32_t flags,
                               int64_t chunk, int32_t *counts_dev);

/* ---- snapshot-mode lightcone (Sec. 2.1, Sec. 2.4) -------------------------- */

/* Which snapshot fills each shell when the simulation wrote snapshots (all
 * particles at one redshift) instead of a lightcone output.  Shell b is
 * filled from the snapshot at its redshift z_b, the lower edge (Sec. 2.4);
 * with snapshots sparser than shells (the paper's snapshots are spaced
 * dz = 0.02, its shells 0.01) shell b takes the last snapshot at or below
 * z_b: snap_of_shell[b] = max{s : z_snap[s] <= z_b + 1e-9 (1 + |z_b|)}, or
 * -1 when every snapshot lies above z_b.  The 1e-9 slack absorbs the last-bit
 * differences of redshift grids generated in different ways.
 * z_edges: nshell+1 finite, increasing; z_snap: nsnap finite, strictly
 * increasing (host arrays).  UFC_ERR_ARG otherwise.  Host only. */
ufc_status ufc_snapshot_assign(const double *z_edges, int32_t nshell,
                               const double *z_snap, int32_t nsnap,
                               int32_t *snap_of_shell);
/* Count maps of a snapshot-mode lightcone: shell b counts the particles of
 * snapshot s = snap_of_shell[b] (xyz_dev[s], n[s] of them, in the box
 * snap_geom[s]: L, obs, n_total and replicate are used, the shell range is
 * ignored) whose radius lies in shell b; a shell with s = -1 stays empty.
 * Each run of consecutive shells taken from one snapshot is one box of a
 * ufc_bin pass; a pass takes up to 16 runs and the later passes accumulate.
 * The dense path's histogram covers only the shells of the pass.  Flags and
 * output as for ufc_bin; ufc_bin_info describes the last pass. */
ufc_status ufc_bin_snapshots(ufc_ctx *ctx, const float *const *xyz_dev,
                             const int64_t *n, const ufc_box *snap_geom,
                             int32_t nsnap, const int32_t *snap_of_shell,
                             const double *chi_edges, int32_t nshell,
                             int32_t nside, int32_t flags, int32_t *counts_dev);
/* ufc_bin_snapshots from host memory, for snapshot sets beyond device
 * memory: each run's particles stream through two device buffers of at
 * most `chunk` particles as in ufc_bin_host_stream (copy of the next chunk
 * overlapped with the binning of the current one; device memory held:
 * 2 x 12 chunk bytes plus one chunk's binning workspace).  Counts equal
 * ufc_bin_snapshots'.  Host buffers as for ufc_bin_host;
 * UFC_ERR_UNSUPPORTED while the context stream is capturing. */
ufc_status ufc_bin_snapshots_host(ufc_ctx *ctx, const float *const *xyz_host,
                                  const int64_t *n, const ufc_box *snap_geom,
                                  int32_t nsnap, const int32_t *snap_of_shell,
                                  const double *chi_edges, int32_t nshell,
                                  int32_t nside, int32_t flags, int64_t chunk,
                                  int32_t *counts_dev);
/* Diagnostics of the last ufc_bin/ufc_keys call (synchronises):
 * info[0] invalid particles, info[1] particle-images with a key,
 * info[2] decisions refined past the FP32 stage, info[3] past the
 * float-float stage (resolved by the FP64 procedure itself). */
ufc_status ufc_bin_info(ufc_ctx *ctx, int64_t info[4]);

/* ---- kappa map, moments, PDF (Eq. 6, Eq. 12-13, Sec. 3.3) ------------------ */

/* kappa_p = sum_b A[b] n_bp - C accumulated to better than FP64's needs in
 * double-float arithmetic, rounded once to FP32 (kappa_dev, may be NULL).
 * moments_dev[10] (FP64): mean, mu2, mu3, mu4, skewness, excess kurtosis,
 * <s^2> = (N-1) mu2/N, sigma^2_{s^2} (Eq. 13), s^2/sigma^2_{s^2}, N, where
 * mu_k are the central moments of the FP32 map.  pdf_dev[nbins+3] (int64):
 * counts of bin = floor((kappa - lo) * nbins/(hi - lo)), then underflow
 * (kappa < lo), overflow (kappa >= hi) and NaN. A and C are host arrays. */
ufc_status ufc_kappa_stats(ufc_ctx *ctx, const int32_t *counts_dev,
                           int32_t nshell, int32_t nside, const double *A,
                           double C, double pdf_lo, double pdf_hi,
                           int32_t nbins, float *kappa_dev, double *moments_dev,
                           int64_t *pdf_dev);

/* Same results as ufc_kappa_stats, but the call allocates no device memory:
 * it is meant for callers that cannot call cudaMalloc, for example an
 * application whose device memory is owned by its own allocator (a caching
 * allocator or a fixed arena carved out at start-up), or a pipeline that must
 * not allocate once it runs because cudaMalloc may block and synchronise the
 * device.  The paper has no counterpart; this is a property of the library.
 *  - The caller passes every input and output: kappa_dev, moments_dev and
 *    pdf_dev are all required (none may be NULL).
 *  - Scratch (per-block partial sums) lives in one fixed device array of
 *    4096 doubles (32 KB) that every GPU loading the library holds until the
 *    process exits.  A launch that would need more returns UFC_ERR_CAPACITY.
 *  - The first call on a device looks up the array's device address (with
 *    that device current) and caches it; make that first call before any
 *    stream capture on the device.  A cudaDeviceReset unloads the library's
 *    device code and can move the array: after a reset this call must not
 *    be used again in the same process.
 *  - All calls on a device share the array, which keeps the last call's
 *    contents: calls that overlap on the GPU (different streams or contexts)
 *    race on it.  Serialise them.  pdf_dev is cleared by the call itself. */
ufc_status ufc_kappa_stats_noalloc(ufc_ctx *ctx, const int32_t *counts_dev,
                                   int32_t nshell, int32_t nside, const double *A,
                                   double C, double pdf_lo, double pdf_hi,
                                   int32_t nbins, float *kappa_dev,
                                   double *moments_dev, int64_t *pdf_dev);

/* ---- adjoint --------------------------------------------------------------- */

/* Gradient of L = w_var var(kappa) + w_skew skew(kappa) + sum_p g_p kappa_p
 * with respect to theta = (Omega_m, h, alpha, beta, z0), counts held fixed,
 * for the unrounded map kappa_p = sum_b A_b n_bp - C:
 *   dL/dtheta = sum_b dA_b/dtheta G_b - dC/dtheta H,
 *   G_b = sum_p gbar_p n_bp,  H = sum_p gbar_p,  gbar = dL/dkappa.
 * g_kappa_dev (FP32 [npix], 16-byte aligned) may be NULL.  counts_dev must
 * be 16-byte aligned; above 72 shells the counts are read once per window
 * of 72 shells (60 shells or fewer take one window).  dA [5][nshell], dC [5] come from ufc_kappa_coeffs (or
 * ufc_delta_coeffs).  grad_theta [5] (host) receives
 * dL/dtheta; G [nshell] and H (host) may be NULL.  The per-shell sums are
 * exact 128-bit fixed-point sums of the map quantised to 44 bits relative to
 * its maximum (|kappa_p| and |g_p| below 2^14, else UFC_ERR_UNSUPPORTED).
 * Synchronises. */
ufc_status ufc_kappa_backward(ufc_ctx *ctx, const int32_t *counts_dev,
                              int32_t nshell, int32_t nside, const double *A,
                              double C, double w_var, double w_skew,
                              const float *g_kappa_dev, const double *dA,
                              const double *dC, double *grad_theta, double *G,
                              double *H);

/* ufc_kappa_stats and ufc_kappa_backward in one read of the counts: the
 * adjoint's pass over the counts also rounds the unrounded map e_p (built in
 * the same shell order as the forward pass) to the FP32 kappa_dev
 * ([npix], 16-byte aligned, required), so kappa_dev, pdf_dev and the
 * gradient outputs equal those of the two separate calls bit for bit;
 * moments_dev equal them to the last bits only (the map's mean is summed
 * over a different grid of partial sums).  Arguments as for the two calls.
 * Synchronises. */
ufc_status ufc_kappa_stats_backward(ufc_ctx *ctx, const int32_t *counts_dev,
                                    int32_t nshell, int32_t nside, const double *A,
                                    double C, double pdf_lo, double pdf_hi,
                                    int32_t nbins, double w_var, double w_skew,
                                    const float *g_kappa_dev, const double *dA,
                                    const double *dC, float *kappa_dev,
                                    double *moments_dev, int64_t *pdf_dev,
                                    double *grad_theta, double *G, double *H);

/* ---- subvolume combination (Sec. 2.4) -------------------------------------- */

/* Sec. 2.4 processes subvolumes of a simulation independently and combines
 * their maps.  kappa_p = sum_b A_b n_bp - C is linear in the counts, so a
 * process that binned one subvolume contributes its partial sum
 *   partial_p = sum_b A_b n_bp        (no -C; A from ufc_kappa_coeffs with the
 *                                      WHOLE simulation's n_total per box)
 * accumulated in double-float over the shells in order (as ufc_kappa_stats)
 * and stored as FP64 in partial_dev ([12 nside^2], 16-byte aligned, 8 B per
 * pixel: 100 MB at Nside 1024, against 4 nshell B per pixel for the count
 * maps).  The partials of all subvolumes are summed in FP64 by the caller
 * (an all-reduce across processes), then ufc_kappa_stats_partial finishes
 * the map.  counts_dev 16-byte aligned.  Asynchronous. */
ufc_status ufc_kappa_partial(ufc_ctx *ctx, const int32_t *counts_dev,
                             int32_t nshell, int32_t nside, const double *A,
                             double *partial_dev);

/* The FP32 map kappa_p = E_p - C from the summed partials E (partial_dev,
 * the sum over subvolumes of ufc_kappa_partial), subtracted in double-float
 * and rounded once to FP32, with the moments and PDF of ufc_kappa_stats
 * (same definitions and outputs; kappa_dev 16-byte aligned, all three
 * outputs required).  The map equals ufc_kappa_stats' map of the summed
 * counts except where a value lies within about 2^-48 (relative) of an FP32
 * rounding boundary; there the two may differ by one FP32 unit.
 * Asynchronous. */
ufc_status ufc_kappa_stats_partial(ufc_ctx *ctx, const double *partial_dev,
                                   int32_t nside, double C, double pdf_lo,
                                   double pdf_hi, int32_t nbins,
                                   float *kappa_dev, double *moments_dev,
                                   int64_t *pdf_dev);

/* The adjoint of ufc_kappa_backward for a map combined from subvolumes.
 * The gradient of L needs G_b = sum_p gbar_p n_bp over the whole
 * simulation's counts, with gbar from the whole map; G_b is linear in the
 * counts, so each process forms its subvolume's share from its own counts
 * (counts_dev) and the summed partials (partial_dev, e_p = E_p - C):
 *   sums[4 b + 0..3] = sum_p e_p n_bp, sum_p e_p^2 n_bp, sum_p g_p n_bp,
 *                      sum_p n_bp                      (b < nshell; the
 *                                                      subvolume's share)
 *   sums[4 nshell + 0..3] = sum_p e_p, sum_p e_p^2, sum_p e_p^3, sum_p g_p
 *                                                      (whole map; the same
 *                                                      in every process)
 * (host array of 4 nshell + 4 FP64, exact fixed-point sums rounded once, as
 * in ufc_kappa_backward).  The caller sums the first 4 nshell entries over
 * the processes and passes the result to ufc_kappa_grad_from_sums.  With
 * kappa_dev non-NULL the same read of the counts also writes the FP32 map
 * (equal to ufc_kappa_stats_partial's bit for bit) with its moments and PDF
 * (moments_dev, pdf_dev then required).  g_kappa_dev as in
 * ufc_kappa_backward, may be NULL.  Synchronises. */
ufc_status ufc_kappa_adjoint_sums(ufc_ctx *ctx, const int32_t *counts_dev,
                                  int32_t nshell, int32_t nside,
                                  const double *partial_dev, double C,
                                  const float *g_kappa_dev, double pdf_lo,
                                  double pdf_hi, int32_t nbins,
                                  float *kappa_dev, double *moments_dev,
                                  int64_t *pdf_dev, double *sums);

/* dL/dtheta of ufc_kappa_backward from adjoint sums (layout of
 * ufc_kappa_adjoint_sums, the per-shell entries summed over subvolumes):
 * the central moments of the map from its power sums, then
 *   G_b = w_var dvar_b + w_skew dskew_b + sum_p g_p n_bp,  H = sum_p g_p,
 *   grad_theta[j] = sum_b dA[j][b] G_b - dC[j] H.
 * Host only (no device, no context); G [nshell] and H may be NULL.
 * UFC_ERR_ARG for NULL inputs, bad sizes or non-finite sums. */
ufc_status ufc_kappa_grad_from_sums(const double *sums, int32_t nshell,
                                    int32_t nside, double w_var, double w_skew,
                                    const double *dA, const double *dC,
                                    double *grad_theta, double *G, double *H);

/* ---- full-sky power spectrum (Sec. 3.2, Eq. 10-11) ------------------------- */

/* Spherical-harmonic coefficients of a RING map (FP32 [12 nside^2], e.g.
 * kappa or delta from ufc_kappa_stats):
 *   a_lm = (4 pi / N_pix) sum_p map_p Y*_lm(theta_p, phi_p),  0 <= m <= l <= lmax,
 * at the pixel centres, Y_lm orthonormal with the Condon-Shortley phase.
 * alm_dev: FP64 (re, im) pairs, m-major (index m (2 lmax + 1 - m)/2 + l),
 * (lmax+1)(lmax+2)/2 of them, 16-byte aligned.  nside a power of two
 * <= 1024 (UFC_ERR_UNSUPPORTED above), 0 <= lmax <= 4 nside (the usual
 * choice is 3 nside - 1).  Workspace about 16 (lmax+1)(4 nside) + 12 (lmax+1)
 * (2 nside) + 16 (lmax+1)(lmax+2)/2 ceil(nside/512) bytes.  Asynchronous. */
ufc_status ufc_map2alm(ufc_ctx *ctx, const float *map_dev, int32_t nside,
                       int32_t lmax, double *alm_dev);
/* Angular power spectrum of a real map from its a_lm (layout as above):
 * cl_dev[l] = (|a_l0|^2 + 2 sum_{m=1..l} |a_lm|^2) / (2l + 1), l = 0..lmax.
 * Its covariance over realisations: ufc_welford_update on (binned) C_l. */
ufc_status ufc_alm2cl(ufc_ctx *ctx, const double *alm_dev, int32_t lmax,
                      double *cl_dev);
/* Band powers for the binned C_l covariance (the paper bins with
 * Delta l = 4, 10, 24): out_dev[b] = mean of cl_dev[l] over
 * l in [lmin + b dl, lmin + (b+1) dl), b < nbins; the bins must lie in
 * [0, lmax].  Feed them to ufc_welford_update for their covariance. */
ufc_status ufc_cl_bin(ufc_ctx *ctx, const double *cl_dev, int32_t lmax,
                      int32_t lmin, int32_t dl, int32_t nbins, double *out_dev);

/* ---- smoothed maps (Sec. 3.3, Eq. 12-13) ----------------------------------- */

/* Gaussian beam in harmonic space: alm_out[l, m] = alm_in[l, m] b_l,
 * b_l = exp(-l(l+1) sigma^2 / 2), sigma the beam's r.m.s. radius in
 * radians (the paper smooths with 10.8 arcmin).  In place allowed. */
ufc_status ufc_alm_beam(ufc_ctx *ctx, const double *alm_in_dev, int32_t lmax,
                        double sigma, double *alm_out_dev);
/* The real field with coefficients a_lm (layout of ufc_map2alm) at the RING
 * pixel centres: map_p = sum_l sum_{m>=0} (2 - delta_m0) Re(a_lm Y_lm(p)),
 * written as FP32 [12 nside^2].  Same nside and lmax limits as ufc_map2alm. */
ufc_status ufc_alm2map(ufc_ctx *ctx, const double *alm_dev, int32_t nside,
                       int32_t lmax, float *map_dev);
/* Moments (the 10 of ufc_kappa_stats, including s^2 and sigma^2_{s^2} of
 * Eq. 12-13) and PDF of any FP32 RING map (16-byte aligned), e.g. a map
 * smoothed with ufc_alm_beam + ufc_alm2map. */
ufc_status ufc_map_stats(ufc_ctx *ctx, const float *map_dev, int32_t nside,
                         double pdf_lo, double pdf_hi, int32_t nbins,
                         double *moments_dev, int64_t *pdf_dev);

/* ---- covariance over realisations (Eq. 10-11) ------------------------------ */

#define UFC_BATCH_GRAPH 1      /* capture the whole batch into one CUDA graph */
#define UFC_BATCH_LAUNCHES 2   /* one launch sequence per realisation, never the
                                  persistent kernel                           */

/* Statistics of nreal realisations in one call (Sec. 3.2 averages over 150
 * realisations).  Realisation r has nbox particle sets xyz_dev[r*nbox + k]
 * with n[r*nbox + k] particles in boxes[r*nbox + k]; the shell edges, nside
 * and PDF range are shared; A [nreal][nshell] and C [nreal] are that
 * realisation's kappa coefficients (they depend on its n_total).  For each r
 * the library bins, builds kappa in kappa_dev (scratch, [npix]) from
 * counts_dev (scratch, [nshell][npix]), writes moments_dev[r][10],
 * pdf_dev[r][nbins+3] and stats_dev[r][6 + nbins] (ufc_stats_vector), and
 * finally adds all nreal vectors to the Welford state state_dev in order.
 * Count maps of up to 64 MB whose boxes have no periodic images, and whose
 * per-realisation maps fit in 4 GB of workspace together, run as ONE
 * persistent kernel (unless UFC_BATCH_LAUNCHES): a device work queue of
 * (realisation, particle chunk) tasks; the block that finishes a
 * realisation's last chunk builds its kappa map, moments, PDF and
 * statistics vector, and the block that finishes the last realisation runs
 * the Welford update in realisation order.  No block waits for another
 * (completion is counted with atomics).  Its chunk size and blocks per SM
 * come from ufc_set_tuning.  Results equal the one-at-a-time calls bit for
 * bit; counts_dev and kappa_dev are then not used (the kernel keeps one map
 * per realisation in the workspace).  Otherwise count maps of up to 64 MB
 * run on up to 8 concurrent lanes: realisation r on lane r mod 8, lane 0
 * being this context with counts_dev and kappa_dev, the others extra
 * contexts owned by this one, each with its own count and kappa maps,
 * workspace and stream (forked from and joined back to the context stream
 * by events); results do not depend on the lanes.
 * The workspace is grown once up front; with UFC_BATCH_GRAPH the per-
 * realisation work is captured into one CUDA graph and launched once (the
 * context stream must not be capturing already; on the legacy default
 * stream the graph is captured and launched on a stream of the context,
 * ordered after earlier work and before later work by events).  The
 * executable graph stays in the context: a call whose host arguments
 * (pointers, sizes, boxes, shell edges, coefficients, PDF range) equal the
 * previous graph call's relaunches it without capture, reading the particle
 * buffers' current contents; other calls update or rebuild it.
 * Asynchronous. */
ufc_status ufc_batched_stats(ufc_ctx *ctx, int32_t nreal, int32_t nbox,
                             const float *const *xyz_dev, const int64_t *n,
                             const ufc_box *boxes, const double *chi_edges,
                             int32_t nshell, int32_t nside, const double *A,
                             const double *C, double pdf_lo, double pdf_hi,
                             int32_t nbins, int32_t *counts_dev, float *kappa_dev,
                             double *moments_dev, int64_t *pdf_dev,
                             double *stats_dev, double *state_dev, int32_t flags);

/* Tuning of a context (no counterpart in the paper; an autotuner picks the
 * values by timing candidates): batch_chunk = particles per task of the
 * persistent batch kernel (0: 8192), batch_blocks_per_sm = its resident
 * blocks per SM (0: 2; at most 2).  Host only. */
typedef struct {
  int32_t batch_chunk;
  int32_t batch_blocks_per_sm;
} ufc_tuning;
ufc_status ufc_set_tuning(ufc_ctx *ctx, const ufc_tuning *t);
ufc_status ufc_get_tuning(const ufc_ctx *ctx, ufc_tuning *t);

/* Statistics vector of one map, the quantity whose covariance over
 * realisations is estimated: v_dev[6 + nbins] = (mean, mu2, mu3, mu4, skew,
 * excess kurtosis, pdf[0..nbins-1] / N) from ufc_kappa_stats's outputs. */
ufc_status ufc_stats_vector(ufc_ctx *ctx, const double *moments_dev,
                            const int64_t *pdf_dev, int32_t nbins, double *v_dev);

/* A Welford state for d-dimensional vectors is 1 + d + d*d doubles:
 * count, mean[d], M2[d][d].  ufc_welford_update adds the nvec vectors
 * v_dev [nvec][d] in order (Welford/Chan update in FP64, device memory);
 * ufc_welford_merge adds state b into state a (Chan et al. pairwise
 * formula); ufc_welford_finalize writes mean, cov = M2/(n - ddof) and
 * corr = cov_ij / sqrt(cov_ii cov_jj) (0 where a variance is 0), all device
 * memory.  Zero a state (all doubles 0) before its first update. */
ufc_status ufc_welford_update(ufc_ctx *ctx, const double *v_dev, int32_t nvec,
                              int32_t d, double *state_dev);
ufc_status ufc_welford_merge(ufc_ctx *ctx, double *state_a_dev,
                             const double *state_b_dev, int32_t d);
ufc_status ufc_welford_finalize(ufc_ctx *ctx, const double *state_dev,
                                int32_t d, int32_t ddof, double *mean_dev,
                                double *cov_dev, double *corr_dev);
/* The same update and merge on host memory (no context, no GPU): the
 * realisation-sharded path of Eq. 10, where processes that hold their own
 * states (for example ranks exchanging them over a CPU transport) combine
 * them in rank order.  Same formulas and order as the device calls. */
ufc_status ufc_welford_update_host(const double *v, int32_t nvec, int32_t d,
                                   double *state);
ufc_status ufc_welford_merge_host(double *state_a, const double *state_b,
                                  int32_t d);

#ifdef __cplusplus
}
#endif
#endif /* UFALCON_H */
