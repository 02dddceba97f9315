/*
 * Plain, slow FP64 CPU oracle for the UFalcon lightcone hot path
 * (Sgier, Refregier, Amara & Nicola, "Fast Generation of Covariance
 * Matrices for Weak Lensing", sections 2.3-2.4 and 3.2-3.3).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or constant generator with the CUDA library; the two meet
 * only through the seeded input generator and through the results they are
 * compared on.
 *
 * Compiled with -O2 -ffp-contract=off (no fused multiply-add, no fast-math),
 * so every floating-point step below is one IEEE-754 binary64 operation in
 * round-to-nearest, in the order written.
 *
 * Functions whose result cannot be pinned to anything other than itself are
 * marked "parity unpinned" at their definition.  None are at present.
 */
#ifndef UFALCON_ORACLE_H
#define UFALCON_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* A simulation box (Table 1; nesting scheme, Sec. 2.4).  The observer sits
 * at obs (normally the box centre).  The box owns the shells
 * [shell_lo, shell_hi) of the global shell table.  n_total is the number of
 * particles of the whole simulation box (mean density rho = m_p N / V,
 * Sec. 2.3).  replicate = R >= 0 adds the periodic images i,j,k in [-R, R]. */
typedef struct {
  double L;
  double obs[3];
  int64_t n_total;
  int32_t shell_lo, shell_hi;
  int32_t replicate;
} or_box;

/* ---- HEALPix RING geometry (pixelisation, Sec. 2.4) ---------------------- */
int64_t or_nside2npix(int64_t nside);
/* Fixed FP64 procedure mapping an observer-relative vector to its RING pixel
 * (tie rule in healpix.c).  r must be the FP64 radius of (dx,dy,dz) computed
 * as sqrt((dx*dx + dy*dy) + dz*dz).  Returns -1 if r == 0. */
int64_t or_vec2pix_ring(int64_t nside, double dx, double dy, double dz, double r);
void or_vec2pix_batch(int64_t nside, const double *d, int64_t n, int64_t *pix);
/* The quarter-turn azimuth t = 2*phi/pi in [0,4) of the same procedure. */
double or_azimuth_t(double dx, double dy);
/* Centre of a RING pixel as (z = cos theta, phi). */
void or_pix2ang_ring(int64_t nside, int64_t pix, double *z, double *phi);

/* ---- Lightcone binning (Eq. 5 and Eq. 8) -------------------------------- */
/* Key of one particle: shell*npix + pix, or -1 (outside the box's shells),
 * or -2 (invalid: non-finite or r == 0).  Replication must be 0. */
void or_keys(const float *xyz, int64_t n, const or_box *box,
             const double *chi_edges, int32_t nshell, int64_t nside,
             int64_t *keys_out);
/* Adds every in-cone particle (and image) to counts[nshell][npix];
 * returns the number of invalid particles. */
int64_t or_bin(const float *xyz, int64_t n, const or_box *box,
               const double *chi_edges, int32_t nshell, int64_t nside,
               int32_t *counts);
/* or_bin on all host cores (OpenMP, atomic increments): same counts. */
int64_t or_bin_omp(const float *xyz, int64_t n, const or_box *box,
                   const double *chi_edges, int32_t nshell, int64_t nside,
                   int32_t *counts, int32_t *threads_out);
/* Snapshot mode: the snapshot of each shell (last one at or below the
 * shell's lower-edge redshift, -1 if none), and the count maps with shell b
 * taken from snapshot snap_of_shell[b] (added to counts). */
void or_snapshot_assign(const double *z_edges, int32_t nshell, const double *z_snap,
                        int32_t nsnap, int32_t *snap_of_shell);
int64_t or_bin_snapshots(const float *const *xyz, const int64_t *n, const or_box *geom,
                         const int32_t *snap_of_shell, const double *chi_edges,
                         int32_t nshell, int64_t nside, int32_t *counts);

/* ---- Cosmology and shell weights (Eq. 1-3, Eq. 6) ------------------------ */
/* Source: kind 0 = single plane at z_s (Eq. 3); kind 1 = n(z) proportional to
 * z^alpha exp(-(z/z0)^beta) on [0, z_max]. */
typedef struct {
  int32_t kind;
  double z_s, alpha, beta, z0, z_max;
} or_source;
/* theta = (omega_m, h, alpha, beta, z0); units_mpc_over_h = 1 means lengths
 * in Mpc/h (c/H0 = 2997.92458), 0 means Mpc (c/H0 = 2997.92458/h). */
double or_comoving_distance(double omega_m, double h, int units_mpc_over_h, double z);
void or_chi_edges(double omega_m, double h, int units_mpc_over_h,
                  const double *z_edges, int32_t nshell, double *chi_out);
double or_z_of_chi(double omega_m, double h, int units_mpc_over_h, double chi);
/* Per-shell weight W_b (Eq. 3 for a plane, its n(z) average otherwise). */
void or_shell_weights(double omega_m, const double *z_edges, int32_t nshell,
                      const or_source *src, double *w_out);
/* A_b, B_b and C of kappa_p = sum_b A_b n_bp - C (Eq. 6).  dens_volume
 * selects the density factor: 0 at the shell's lower edge (as printed),
 * 1 averaged over the shell volume. */
void or_kappa_coeffs(double omega_m, double h, int units_mpc_over_h, int dens_volume,
                     const or_box *boxes, int32_t nbox,
                     const double *z_edges, int32_t nshell, int64_t nside,
                     const or_source *src, double *A_out, double *B_out,
                     double *C_out);

/* A_b and C of the overdensity map delta_p = sum_b A_b n_bp - C (Eq. 7). */
void or_delta_coeffs(double omega_m, double h, int units_mpc_over_h, int dens_volume,
                     const or_box *boxes, int32_t nbox,
                     const double *z_edges, int32_t nshell, int64_t nside,
                     double *A_out, double *C_out);

/* ---- Map statistics (Eq. 6, Eq. 12-13, PDF of Sec. 3.3) ------------------ */
void or_kappa_map(const int32_t *counts, int32_t nshell, int64_t npix,
                  const double *A, double C, float *kappa_out);
/* moments_out[10]: mean, mu2, mu3, mu4, skew, excess kurtosis, <s^2>,
 * sigma^2_{s^2}, s^2/sigma^2_{s^2}, N. */
void or_moments(const float *kappa, int64_t npix, double *moments_out);
/* pdf_out[nbins+3]: bins, underflow, overflow, NaN. */
void or_pdf(const float *kappa, int64_t npix, double lo, double hi,
            int32_t nbins, int64_t *pdf_out);
/* Covariance and correlation over realisations (Eq. 10-11). */
void or_covariance(const double *v, int64_t nreal, int32_t d, int32_t ddof,
                   double *mean_out, double *cov_out, double *corr_out);

/* ---- Gradients by the complex-step method -------------------------------- */
/* d(var, skew, <g,kappa>)/d theta_j for theta = (omega_m, h, alpha, beta, z0)
 * with the counts held fixed; grad_out[3][5].  g may be NULL. */
void or_kappa_stat_grads(const int32_t *counts, int32_t nshell, int64_t nside,
                         double omega_m, double h, int units_mpc_over_h,
                         const or_box *boxes, int32_t nbox,
                         const double *z_edges, const or_source *src,
                         const float *g, double *grad_out);
/* The same statistics in FP64 without rounding kappa to FP32: out[3]. */
void or_kappa_stats_f64(const int32_t *counts, int32_t nshell, int64_t nside,
                        double omega_m, double h, int units_mpc_over_h,
                        const or_box *boxes, int32_t nbox,
                        const double *z_edges, const or_source *src,
                        const float *g, double *out);

/* ---- Spherical-harmonic analysis (full-sky C_l of Sec. 3.2) ----------------- */
/* a_lm index m (2 lmax + 1 - m) / 2 + l, 0 <= m <= l <= lmax. */
int64_t or_alm_index(int32_t lmax, int32_t l, int32_t m);
/* Orthonormal associated Legendre functions lambda_lm(z), s = sqrt(1 - z^2). */
void or_lambda_lm(double z, double s, int32_t lmax, double *lam);
/* a_lm = (4 pi / N_pix) sum_p map_p Y*_lm at the RING pixel centres. */
void or_map2alm(const float *map, int64_t nside, int32_t lmax, double *alm_re, double *alm_im);
/* C_l = (|a_l0|^2 + 2 sum_{m>0} |a_lm|^2) / (2l + 1). */
void or_alm2cl(const double *alm_re, const double *alm_im, int32_t lmax, double *cl);
/* map_p = sum_l sum_{m>=0} (2 - delta_m0) Re(a_lm Y_lm) at the RING pixel centres. */
void or_alm2map(const double *alm_re, const double *alm_im, int64_t nside, int32_t lmax,
                double *map);
/* Gaussian beam b_l = exp(-l(l+1) sigma^2 / 2), sigma the r.m.s. radius (radians). */
void or_gauss_beam(double sigma, int32_t lmax, double *b);

#ifdef __cplusplus
}
#endif
#endif
