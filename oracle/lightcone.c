/*
 * Oracle: assignment of lightcone particles to shells and pixels, and the
 * per-shell count maps n_p(pix, Delta chi_b).  TEST INFRASTRUCTURE ONLY.
 *
 * Shell membership (Eq. 8) is written with <= at both ends in the paper, so
 * a particle on an edge would belong to two shells; it is read here as the
 * half-open chi_b <= r < chi_{b+1}.  Radii outside [chi_lo, chi_hi) of the
 * particle's box are dropped (nesting scheme, Sec. 2.4: each box owns the
 * shells [shell_lo, shell_hi)).  The observer-relative vector is formed in
 * FP64 as d = x + (i L - o) for the periodic image (i, j, k); without
 * replication that is x - o.  r = sqrt((dx*dx + dy*dy) + dz*dz).  A particle
 * with a non-finite coordinate, or an image with r == 0, is invalid.
 */
#include <math.h>
#include <omp.h>
#include <stdlib.h>
#include "oracle.h"

static int shell_of(double r, const double *chi, int32_t lo, int32_t hi) {
  if (!(r >= chi[lo]) || !(r < chi[hi])) return -1;
  int b = lo;
  while (!(r < chi[b + 1])) ++b;
  return b;
}

/* Key of one observer-relative vector, or -1 (outside) / -2 (r == 0). */
static int64_t key_of(double dx, double dy, double dz, const or_box *box,
                      const double *chi, int64_t nside) {
  double r = sqrt((dx * dx + dy * dy) + dz * dz);
  if (r == 0.0) return -2;
  int b = shell_of(r, chi, box->shell_lo, box->shell_hi);
  if (b < 0) return -1;
  int64_t pix = or_vec2pix_ring(nside, dx, dy, dz, r);
  return (int64_t)b * or_nside2npix(nside) + pix;
}

void or_keys(const float *xyz, int64_t n, const or_box *box,
             const double *chi_edges, int32_t nshell, int64_t nside,
             int64_t *keys_out) {
  (void)nshell;
  double sx = 0.0 - box->obs[0], sy = 0.0 - box->obs[1], sz = 0.0 - box->obs[2];
  for (int64_t p = 0; p < n; ++p) {
    float x = xyz[3 * p], y = xyz[3 * p + 1], z = xyz[3 * p + 2];
    if (!isfinite(x) || !isfinite(y) || !isfinite(z)) { keys_out[p] = -2; continue; }
    keys_out[p] = key_of((double)x + sx, (double)y + sy, (double)z + sz, box,
                         chi_edges, nside);
  }
}

int64_t or_bin(const float *xyz, int64_t n, const or_box *box,
               const double *chi_edges, int32_t nshell, int64_t nside,
               int32_t *counts) {
  (void)nshell;
  int R = box->replicate;
  int64_t invalid = 0;
  for (int64_t p = 0; p < n; ++p) {
    float x = xyz[3 * p], y = xyz[3 * p + 1], z = xyz[3 * p + 2];
    if (!isfinite(x) || !isfinite(y) || !isfinite(z)) { ++invalid; continue; }
    for (int i = -R; i <= R; ++i)
      for (int j = -R; j <= R; ++j)
        for (int k = -R; k <= R; ++k) {
          double sx = (double)i * box->L - box->obs[0];
          double sy = (double)j * box->L - box->obs[1];
          double sz = (double)k * box->L - box->obs[2];
          int64_t key = key_of((double)x + sx, (double)y + sy, (double)z + sz,
                               box, chi_edges, nside);
          if (key >= 0) counts[key] += 1;
          else if (key == -2) ++invalid;
        }
  }
  return invalid;
}

/*
 * Snapshot-mode lightcone (Sec. 2.1: snapshot outputs at redshift spacing
 * 0.02; Sec. 2.4: the particles of shell b are those of the snapshot at
 * z_b).  Reading for snapshots sparser than shells: shell b takes the last
 * snapshot whose redshift is at most z_b, with a slack of 1e-9 (1 + |z_b|)
 * for grids that differ in the last bit; -1 when every snapshot lies above.
 * Written as the definition: for each shell, every snapshot is examined.
 */
void or_snapshot_assign(const double *z_edges, int32_t nshell, const double *z_snap,
                        int32_t nsnap, int32_t *snap_of_shell) {
  for (int32_t b = 0; b < nshell; ++b) {
    const double zb = z_edges[b];
    int32_t best = -1;
    for (int32_t s = 0; s < nsnap; ++s)
      if (z_snap[s] <= zb + 1e-9 * (1.0 + fabs(zb)) && s > best) best = s;
    snap_of_shell[b] = best;
  }
}

/* Count maps of a snapshot-mode lightcone, one shell at a time: shell b is
 * binned from snapshot snap_of_shell[b] as a box owning that shell alone
 * (geometry from geom[s]).  Adds to counts; returns the invalid particles
 * of the passes made. */
int64_t or_bin_snapshots(const float *const *xyz, const int64_t *n, const or_box *geom,
                         const int32_t *snap_of_shell, const double *chi_edges,
                         int32_t nshell, int64_t nside, int32_t *counts) {
  int64_t invalid = 0;
  for (int32_t b = 0; b < nshell; ++b) {
    const int32_t s = snap_of_shell[b];
    if (s < 0) continue;
    or_box box = geom[s];
    box.shell_lo = b;
    box.shell_hi = b + 1;
    invalid += or_bin(xyz[s], n[s], &box, chi_edges, nshell, nside, counts);
  }
  return invalid;
}

/*
 * The same binning spread over the host's cores with OpenMP (used to time
 * the CPU baseline on all cores): particles are independent, each adds its
 * images to the shared count maps with atomic increments, so the counts
 * equal or_bin's.  Returns the invalid particles; *threads_out is the
 * number of threads that ran.
 */
int64_t or_bin_omp(const float *xyz, int64_t n, const or_box *box,
                   const double *chi_edges, int32_t nshell, int64_t nside,
                   int32_t *counts, int32_t *threads_out) {
  (void)nshell;
  const int R = box->replicate;
  int64_t invalid = 0;
  int threads = 1;
#pragma omp parallel reduction(+ : invalid)
  {
#pragma omp single
    threads = omp_get_num_threads();
#pragma omp for schedule(static)
    for (int64_t p = 0; p < n; ++p) {
      const float x = xyz[3 * p], y = xyz[3 * p + 1], z = xyz[3 * p + 2];
      if (!isfinite(x) || !isfinite(y) || !isfinite(z)) { ++invalid; continue; }
      for (int i = -R; i <= R; ++i)
        for (int j = -R; j <= R; ++j)
          for (int k = -R; k <= R; ++k) {
            const double sx = (double)i * box->L - box->obs[0];
            const double sy = (double)j * box->L - box->obs[1];
            const double sz = (double)k * box->L - box->obs[2];
            const int64_t key = key_of((double)x + sx, (double)y + sy, (double)z + sz,
                                       box, chi_edges, nside);
            if (key >= 0) {
#pragma omp atomic
              counts[key] += 1;
            } else if (key == -2) {
              ++invalid;
            }
          }
    }
  }
  if (threads_out) *threads_out = threads;
  return invalid;
}
