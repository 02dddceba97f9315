/*
 * Oracle: kappa map (Eq. 6), moments (Eq. 12-13), PDF (Sec. 3.3) and the
 * covariance/correlation over realisations (Eq. 10-11).
 * TEST INFRASTRUCTURE ONLY.
 *
 * Readings:
 *  - kappa_p = sum_b A_b n_bp - C accumulated in FP64 in shell order, then
 *    rounded once to FP32;
 *  - Eq. 12 lacks the square of (q_i - mean); the population moments
 *    mu_k = (1/N) sum (q_i - mean)^k of the FP32 map promoted to FP64 are
 *    used, with s^2 = mu2, <s^2> = (N-1) mu2/N and sigma^2_{s^2} from the
 *    left-hand form of Eq. 13; skew = mu3/mu2^(3/2), kurtosis = mu4/mu2^2 - 3;
 *  - PDF: the paper histograms smoothed maps; here the unsmoothed map, with
 *    bin = floor((kappa - lo) * s), s = nbins/(hi - lo) in FP64, kappa < lo
 *    to underflow, kappa >= hi to overflow, NaN to its own slot;
 *  - Eq. 10 as printed is a product of two averages of deviations, which is
 *    zero; it is read as <(v - <v>)(v' - <v'>)>, divided by (R - ddof).
 */
#include <math.h>
#include <stdlib.h>
#include "oracle.h"

void or_kappa_map(const int32_t *counts, int32_t nshell, int64_t npix,
                  const double *A, double C, float *kappa_out) {
  for (int64_t p = 0; p < npix; ++p) {
    double s = 0.0;
    for (int b = 0; b < nshell; ++b) s += A[b] * (double)counts[(int64_t)b * npix + p];
    kappa_out[p] = (float)(s - C);
  }
}

/* Neumaier's compensated sum. */
typedef struct { double s, c; } nsum;
static void nadd(nsum *a, double x) {
  double t = a->s + x;
  if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
  else a->c += (x - t) + a->s;
  a->s = t;
}
static double nval(const nsum *a) { return a->s + a->c; }

void or_moments(const float *kappa, int64_t npix, double *m) {
  nsum s1 = {0, 0};
  for (int64_t p = 0; p < npix; ++p) nadd(&s1, (double)kappa[p]);
  double N = (double)npix;
  double mean = nval(&s1) / N;
  nsum s2 = {0, 0}, s3 = {0, 0}, s4 = {0, 0};
  for (int64_t p = 0; p < npix; ++p) {
    double d = (double)kappa[p] - mean;
    double d2 = d * d;
    nadd(&s2, d2);
    nadd(&s3, d2 * d);
    nadd(&s4, d2 * d2);
  }
  double mu2 = nval(&s2) / N, mu3 = nval(&s3) / N, mu4 = nval(&s4) / N;
  m[0] = mean;
  m[1] = mu2;
  m[2] = mu3;
  m[3] = mu4;
  m[4] = mu3 / (mu2 * sqrt(mu2));
  m[5] = mu4 / (mu2 * mu2) - 3.0;
  m[6] = (N - 1.0) * mu2 / N;
  double N3 = N * N * N;
  m[7] = (N - 1.0) * (N - 1.0) / N3 * mu4 - (N - 1.0) * (N - 3.0) / N3 * mu2 * mu2;
  m[8] = mu2 / m[7];
  m[9] = N;
}

void or_pdf(const float *kappa, int64_t npix, double lo, double hi,
            int32_t nbins, int64_t *pdf) {
  for (int i = 0; i < nbins + 3; ++i) pdf[i] = 0;
  double scale = (double)nbins / (hi - lo);
  for (int64_t p = 0; p < npix; ++p) {
    float k = kappa[p];
    if (isnan(k)) { pdf[nbins + 2]++; continue; }
    double x = (double)k;
    if (x < lo) { pdf[nbins]++; continue; }
    if (x >= hi) { pdf[nbins + 1]++; continue; }
    int64_t b = (int64_t)floor((x - lo) * scale);
    if (b >= nbins) b = nbins - 1;
    if (b < 0) b = 0;
    pdf[b]++;
  }
}

void or_covariance(const double *v, int64_t R, int32_t d, int32_t ddof,
                   double *mean, double *cov, double *corr) {
  for (int a = 0; a < d; ++a) {
    double s = 0.0;
    for (int64_t r = 0; r < R; ++r) s += v[r * d + a];
    mean[a] = s / (double)R;
  }
  for (int a = 0; a < d; ++a)
    for (int b = 0; b < d; ++b) {
      double s = 0.0;
      for (int64_t r = 0; r < R; ++r) s += (v[r * d + a] - mean[a]) * (v[r * d + b] - mean[b]);
      cov[a * d + b] = s / (double)(R - ddof);
    }
  for (int a = 0; a < d; ++a)
    for (int b = 0; b < d; ++b) {
      double den = sqrt(cov[a * d + a] * cov[b * d + b]);
      corr[a * d + b] = den > 0.0 ? cov[a * d + b] / den : 0.0;
    }
}
