/*
 * Oracle (test infrastructure only): spherical-harmonic analysis of a HEALPix
 * RING map and its angular power spectrum, the full-sky C_l of Sec. 3.2
 * (the quantity the paper's covariance of Eq. 10-11 is taken of).  Plain
 * definitions, FP64, one pixel at a time:
 *
 *   a_lm = (4 pi / N_pix) sum_p map_p Y*_lm(theta_p, phi_p),   0 <= m <= l <= lmax,
 *   C_l  = (|a_l0|^2 + 2 sum_{m=1..l} |a_lm|^2) / (2l + 1)     (real maps),
 *
 * at the pixel centres of or_pix2ang_ring, with Y_lm = lambda_lm(cos theta)
 * e^{i m phi} and lambda_lm the orthonormal associated Legendre function with
 * the Condon-Shortley phase, from the textbook recurrences
 *   lambda_00 = 1/sqrt(4 pi),
 *   lambda_mm = -sqrt((2m+1)/(2m)) sin(theta) lambda_{m-1,m-1},
 *   lambda_{m+1,m} = sqrt(2m+3) cos(theta) lambda_mm,
 *   lambda_lm = sqrt((4l^2-1)/(l^2-m^2)) (cos(theta) lambda_{l-1,m}
 *               - sqrt(((l-1)^2-m^2)/(4(l-1)^2-1)) lambda_{l-2,m}).
 * a_lm is stored m-major: index m (2 lmax + 1 - m) / 2 + l.
 *
 * Synthesis (the inverse direction, for maps smoothed in harmonic space,
 * Sec. 3.3): map_p = sum_l sum_{m>=0} (2 - delta_m0) Re(a_lm Y_lm(theta_p, phi_p)),
 * the real field whose a_l,-m = (-1)^m conj(a_lm); the Gaussian beam of
 * r.m.s. radius sigma multiplies a_lm by b_l = exp(-l(l+1) sigma^2 / 2).
 */
#include <math.h>
#include <stdlib.h>

#include "oracle.h"

int64_t or_alm_index(int32_t lmax, int32_t l, int32_t m) {
  return (int64_t)m * (2 * lmax + 1 - m) / 2 + l;
}

/* lambda_lm(cos theta) for 0 <= m <= l <= lmax, m-major as a_lm. */
void or_lambda_lm(double z, double s, int32_t lmax, double *lam) {
  const double pi = 3.14159265358979323846264338327950288;
  double lmm = 1.0 / sqrt(4.0 * pi);
  for (int32_t m = 0; m <= lmax; ++m) {
    if (m > 0) lmm *= -sqrt((2.0 * m + 1.0) / (2.0 * m)) * s;
    double prev2 = 0.0, prev1 = lmm;
    lam[or_alm_index(lmax, m, m)] = lmm;
    for (int32_t l = m + 1; l <= lmax; ++l) {
      double cur;
      if (l == m + 1) {
        cur = sqrt(2.0 * m + 3.0) * z * lmm;
      } else {
        const double a = sqrt((4.0 * l * l - 1.0) / ((double)l * l - (double)m * m));
        const double b = sqrt(((double)(l - 1) * (l - 1) - (double)m * m) /
                              (4.0 * (double)(l - 1) * (l - 1) - 1.0));
        cur = a * (z * prev1 - b * prev2);
      }
      lam[or_alm_index(lmax, l, m)] = cur;
      prev2 = prev1;
      prev1 = cur;
    }
  }
}

void or_map2alm(const float *map, int64_t nside, int32_t lmax, double *alm_re, double *alm_im) {
  const double pi = 3.14159265358979323846264338327950288;
  const int64_t npix = or_nside2npix(nside);
  const int64_t nalm = (int64_t)(lmax + 1) * (lmax + 2) / 2;
  double *lam = (double *)malloc(sizeof(double) * nalm);
  for (int64_t i = 0; i < nalm; ++i) alm_re[i] = alm_im[i] = 0.0;
  const double w = 4.0 * pi / (double)npix;
  for (int64_t p = 0; p < npix; ++p) {
    double z, phi;
    or_pix2ang_ring(nside, p, &z, &phi);
    const double s = sqrt((1.0 - z) * (1.0 + z));
    or_lambda_lm(z, s, lmax, lam);
    const double v = w * (double)map[p];
    for (int32_t m = 0; m <= lmax; ++m) {
      const double c = cos(m * phi), sn = sin(m * phi);   /* e^{-i m phi} = c - i sn */
      for (int32_t l = m; l <= lmax; ++l) {
        const int64_t k = or_alm_index(lmax, l, m);
        alm_re[k] += v * lam[k] * c;
        alm_im[k] -= v * lam[k] * sn;
      }
    }
  }
  free(lam);
}

void or_alm2cl(const double *alm_re, const double *alm_im, int32_t lmax, double *cl) {
  for (int32_t l = 0; l <= lmax; ++l) {
    double s = 0.0;
    for (int32_t m = 0; m <= l; ++m) {
      const int64_t k = or_alm_index(lmax, l, m);
      const double p = alm_re[k] * alm_re[k] + alm_im[k] * alm_im[k];
      s += (m == 0) ? p : 2.0 * p;
    }
    cl[l] = s / (2.0 * l + 1.0);
  }
}

void or_alm2map(const double *alm_re, const double *alm_im, int64_t nside, int32_t lmax,
                double *map) {
  const int64_t npix = or_nside2npix(nside);
  const int64_t nalm = (int64_t)(lmax + 1) * (lmax + 2) / 2;
  double *lam = (double *)malloc(sizeof(double) * nalm);
  for (int64_t p = 0; p < npix; ++p) {
    double z, phi;
    or_pix2ang_ring(nside, p, &z, &phi);
    const double s = sqrt((1.0 - z) * (1.0 + z));
    or_lambda_lm(z, s, lmax, lam);
    double v = 0.0;
    for (int32_t m = 0; m <= lmax; ++m) {
      const double c = cos(m * phi), sn = sin(m * phi);   /* e^{i m phi} = c + i sn */
      double acc = 0.0;
      for (int32_t l = m; l <= lmax; ++l) {
        const int64_t k = or_alm_index(lmax, l, m);
        acc += lam[k] * (alm_re[k] * c - alm_im[k] * sn);
      }
      v += (m == 0) ? acc : 2.0 * acc;
    }
    map[p] = v;
  }
  free(lam);
}

void or_gauss_beam(double sigma, int32_t lmax, double *b) {
  for (int32_t l = 0; l <= lmax; ++l) b[l] = exp(-0.5 * (double)l * (l + 1) * sigma * sigma);
}
