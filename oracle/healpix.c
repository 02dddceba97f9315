/*
 * Oracle: HEALPix RING pixelisation (pixelisation step of Sec. 2.4; the
 * paper uses HEALPix with 12 Nside^2 pixels).  TEST INFRASTRUCTURE ONLY.
 *
 * The paper does not say which HEALPix numbering it uses; RING is taken.
 * Geometry (Gorski et al. 2005): rings i = 1 .. 4N-1 from the north pole.
 *   north cap   i <  N : 4i pixels, z = 1 - i^2/(3N^2), phi = (pi/2i)(j+1/2)
 *   equatorial  N <= i <= 3N : 4N pixels, z = 4/3 - 2i/(3N),
 *               phi = (pi/2N)(j + s/2), s = (i - N + 1) mod 2
 *   south cap mirrors the north cap;  j counts from 0 in increasing phi.
 * Pixel edges: in |z| <= 2/3 the curves N(1/2 + t -+ 3z/4) = integer, in the
 * caps N sqrt(3(1-|z|)) t_p = integer and N sqrt(3(1-|z|)) (1-t_p) = integer,
 * with t = 2 phi/pi and t_p = t - floor(t).
 *
 * Tie rule.  A direction is mapped by one fixed FP64 procedure made only of
 * IEEE +, -, *, /, sqrt in the order written here (no contraction), with the
 * azimuth taken from the series below rather than from a library atan2.
 * floor() is then applied to those FP64 values, so a value that lands on an
 * integer goes to the upper pixel (half-open [k, k+1)).  The CUDA library
 * implements the same procedure separately.
 */
#include <math.h>
#include "oracle.h"

int64_t or_nside2npix(int64_t nside) { return 12 * nside * nside; }

/* atan(u)*(2/pi) for u in [0,1]: two half-angle steps
 *   atan(u) = 2 atan(u / (1 + sqrt(1 + u^2)))
 * bring u below tan(pi/16); the Maclaurin series of atan(w)/w,
 * sum_k (-1)^k w^(2k) / (2k+1), k = 0..10, is summed by Horner's rule, and
 * the result 4 w p is scaled by 2/pi in one product with the double nearest
 * to 8/pi.  u = 1 returns exactly 1/2, so the diagonals |x| = |y| fall on
 * the exact pixel edge and the half-open rule decides them. */
static double atan_quarter_turns(double u) {
  if (u == 1.0) return 0.5;               /* atan(1) = pi/4 exactly */
  double v = u / (1.0 + sqrt(1.0 + u * u));
  double w = v / (1.0 + sqrt(1.0 + v * v));
  double s = w * w;
  double p = 1.0 / 21.0;
  for (int k = 9; k >= 0; --k) {
    double c = ((k & 1) ? -1.0 : 1.0) / (double)(2 * k + 1);
    p = p * s + c;
  }
  const double eight_over_pi = 2.5464790894703253723021402139602;
  return (w * p) * eight_over_pi;
}

double or_azimuth_t(double dx, double dy) {
  double ax = fabs(dx), ay = fabs(dy);
  if (ax == 0.0 && ay == 0.0) return 0.0;
  double tq;
  if (ay <= ax) tq = atan_quarter_turns(ay / ax);
  else tq = 1.0 - atan_quarter_turns(ax / ay);
  double t;
  if (dx >= 0.0) t = (dy >= 0.0) ? tq : 4.0 - tq;
  else t = (dy >= 0.0) ? 2.0 - tq : 2.0 + tq;
  if (t >= 4.0) t = t - 4.0;
  return t;
}

int64_t or_vec2pix_ring(int64_t N, double dx, double dy, double dz, double r) {
  if (!(r > 0.0)) return -1;
  const double two_thirds = 2.0 / 3.0;
  double z = dz / r;
  double za = fabs(z);
  double t = or_azimuth_t(dx, dy);
  if (za <= two_thirds) {
    double temp1 = (double)N * (0.5 + t);
    double temp2 = (double)N * (0.75 * z);
    int64_t jp = (int64_t)floor(temp1 - temp2);
    int64_t jm = (int64_t)floor(temp1 + temp2);
    int64_t ir = N + 1 + jp - jm;          /* ring counted from z = 2/3 */
    if (ir < 1) ir = 1;
    if (ir > 2 * N + 1) ir = 2 * N + 1;
    int64_t kshift = 1 - (ir & 1);
    int64_t ip = ((jp + jm - N + kshift + 1 + 8 * N) / 2) % (4 * N);
    return 2 * N * (N - 1) + (ir - 1) * 4 * N + ip;
  }
  double tp = t - floor(t);
  double s2 = dx * dx + dy * dy;
  double omz = s2 / (r * (r + fabs(dz)));   /* 1 - |z| without cancellation */
  double tmp = (double)N * sqrt(3.0 * omz);
  int64_t jp = (int64_t)floor(tp * tmp);
  int64_t jm = (int64_t)floor((1.0 - tp) * tmp);
  int64_t ir = jp + jm + 1;                 /* ring counted from the pole */
  if (ir > N) ir = N;
  int64_t ip = (int64_t)floor(t * (double)ir) % (4 * ir);
  if (z > 0.0) return 2 * ir * (ir - 1) + ip;
  return 12 * N * N - 2 * ir * (ir + 1) + ip;
}

void or_pix2ang_ring(int64_t N, int64_t pix, double *z, double *phi) {
  const double pi = 3.14159265358979323846264338327950288;
  int64_t npix = 12 * N * N, ncap = 2 * N * (N - 1);
  if (pix < ncap) {
    int64_t i = 1;
    while (2 * (i + 1) * i <= pix) ++i;     /* ring i holds [2i(i-1), 2i(i+1)) */
    int64_t j = pix - 2 * i * (i - 1);
    *z = 1.0 - (double)(i * i) / (3.0 * (double)(N * N));
    *phi = pi / (2.0 * (double)i) * ((double)j + 0.5);
  } else if (pix < npix - ncap) {
    int64_t k = pix - ncap;
    int64_t i = N + k / (4 * N);
    int64_t j = k % (4 * N);
    int64_t s = (i - N + 1) % 2;
    *z = 4.0 / 3.0 - 2.0 * (double)i / (3.0 * (double)N);
    *phi = pi / (2.0 * (double)N) * ((double)j + 0.5 * (double)s);
  } else {
    int64_t q = npix - pix;                 /* 1 .. ncap */
    int64_t i = 1;
    while (2 * i * (i + 1) < q) ++i;        /* ring i from the south pole */
    int64_t j = pix - (npix - 2 * i * (i + 1));
    *z = -(1.0 - (double)(i * i) / (3.0 * (double)(N * N)));
    *phi = pi / (2.0 * (double)i) * ((double)j + 0.5);
  }
}

/* Batch form of or_vec2pix_ring over FP64 vectors d[n][3]. */
void or_vec2pix_batch(int64_t N, const double *d, int64_t n, int64_t *pix) {
  for (int64_t i = 0; i < n; ++i) {
    double x = d[3 * i], y = d[3 * i + 1], z = d[3 * i + 2];
    double r = sqrt((x * x + y * y) + z * z);
    pix[i] = or_vec2pix_ring(N, x, y, z, r);
  }
}
