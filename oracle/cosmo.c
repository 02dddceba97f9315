/*
 * Oracle: cosmology, shell edges, shell weights and the kappa coefficients
 * of Eq. 6.  TEST INFRASTRUCTURE ONLY.
 *
 * Every quantity that depends on theta = (omega_m, h, alpha, beta, z0) is
 * carried as a complex double, so that derivatives can be taken by the
 * complex-step method f'(x) = Im f(x + i eps) / eps (Squire & Trapp 1998):
 * only analytic operations (+, -, *, /, csqrt, cexp, clog, cpow) touch those
 * values.
 *
 * Readings (the paper does not define E(z)):
 *  - flat LambdaCDM, E(z) = sqrt(omega_m (1+z)^3 + 1 - omega_m);
 *  - c/H0 = 2997.92458 Mpc/h, or 2997.92458/h Mpc;
 *  - D(z) = int_0^z dz'/E (the dimensionless distance of Eq. 1), chi = (c/H0) D;
 *  - D(z, z_s) = D(z_s) - D(z) (flat), 1/a = 1 + z;
 *  - Eq. 3 integrand is zero for z > z_s;
 *  - n(z) source: D(z,z_s)/D(z_s) of Eq. 3 is replaced by its average over
 *    n(z_s) = z_s^alpha exp(-(z_s/z0)^beta) normalised on [0, z_max];
 *  - Eq. 6: A_b = (3/2) omega_m W_b (H0/c) N_pix V/(4 pi N chi_b^2) with chi_b
 *    the shell's lower edge and (V, N) of the box that owns the shell,
 *    B_b = (3/2) omega_m W_b (H0/c) Delta chi_b, C = sum_b B_b.
 *
 * Quadrature: Fejer's first rule (Chebyshev points of the first kind, no end
 * points) on panels no wider than 1/8; panels shrink geometrically towards
 * z = 0 where n(z) has a z^alpha end-point behaviour.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include "oracle.h"

typedef double complex cx;

#define FEJER_N 24
static double fej_x[FEJER_N], fej_w[FEJER_N];
static int fej_ready = 0;

/* Fejer type-1 nodes and weights on [-1, 1]:
 * x_k = cos(theta_k), theta_k = (2k-1) pi/(2n),
 * w_k = (2/n) (1 - 2 sum_{j=1}^{floor(n/2)} cos(2 j theta_k)/(4 j^2 - 1)). */
static void fejer_init(void) {
  if (fej_ready) return;
  const double pi = 3.14159265358979323846264338327950288;
  for (int k = 1; k <= FEJER_N; ++k) {
    double th = (2.0 * k - 1.0) * pi / (2.0 * FEJER_N);
    double s = 0.0;
    for (int j = 1; j <= FEJER_N / 2; ++j) s += cos(2.0 * j * th) / (4.0 * j * j - 1.0);
    fej_x[k - 1] = cos(th);
    fej_w[k - 1] = (2.0 / FEJER_N) * (1.0 - 2.0 * s);
  }
  fej_ready = 1;
}

typedef struct {
  cx om, h, alpha, beta, z0;
  int units_mpc_over_h;
  int dens_volume;   /* density factor: 0 at the lower edge, 1 over the shell volume */
} theta_t;

static cx inv_E(const theta_t *th, double z) {
  double zp = 1.0 + z;
  return 1.0 / csqrt(th->om * (zp * zp * zp) + (1.0 - th->om));
}

/* Generic integral of f over [a,b] on panels no wider than 1/8. */
typedef cx (*integrand)(const theta_t *, double, const void *);
static cx integrate(integrand f, const theta_t *th, const void *ctx, double a, double b) {
  fejer_init();
  if (!(b > a)) return 0.0;
  int np = (int)ceil((b - a) * 8.0);
  if (np < 1) np = 1;
  double hw = (b - a) / np;
  cx total = 0.0;
  for (int p = 0; p < np; ++p) {
    double lo = a + p * hw, hi = (p == np - 1) ? b : a + (p + 1) * hw;
    double c = 0.5 * (lo + hi), r = 0.5 * (hi - lo);
    cx s = 0.0;
    for (int k = 0; k < FEJER_N; ++k) s += fej_w[k] * f(th, c + r * fej_x[k], ctx);
    total += r * s;
  }
  return total;
}

static cx f_invE(const theta_t *th, double z, const void *ctx) { (void)ctx; return inv_E(th, z); }
static cx D_of(const theta_t *th, double z) { return integrate(f_invE, th, NULL, 0.0, z); }

static cx c_over_H0(const theta_t *th) {
  return th->units_mpc_over_h ? (cx)2997.92458 : 2997.92458 / th->h;
}

/* ---- n(z) ---------------------------------------------------------------- */
static cx nz(const theta_t *th, double z) {
  if (!(z > 0.0)) return 0.0;
  return cexp(th->alpha * log(z) - cpow(z / th->z0, th->beta));
}
static cx f_nz(const theta_t *th, double z, const void *ctx) { (void)ctx; return nz(th, z); }
/* int_0^zmax n(z) dz on geometric panels [zmax 2^-(k+1), zmax 2^-k]. */
static cx nz_norm(const theta_t *th, double zmax) {
  cx s = 0.0;
  for (int k = 0; k < 60; ++k)
    s += integrate(f_nz, th, NULL, zmax * ldexp(1.0, -(k + 1)), zmax * ldexp(1.0, -k));
  return s;
}
typedef struct { double z; cx Dz; } q_ctx;
/* n(z') (D(z') - D(z)) / D(z') */
static cx f_q(const theta_t *th, double zp, const void *ctx) {
  const q_ctx *q = (const q_ctx *)ctx;
  cx Dp = D_of(th, zp);
  return nz(th, zp) * (Dp - q->Dz) / Dp;
}
static cx f_n_over_D(const theta_t *th, double zp, const void *ctx) {
  (void)ctx;
  return nz(th, zp) / D_of(th, zp);
}

/* ---- shell weights ------------------------------------------------------- */
/* For the n(z) source the average int_z^zmax n(z')(D(z')-D(z))/D(z') dz' is
 * split at the shell's upper edge zb: the part over [zb, zmax] is
 * In - D(z) InD with In = int n and InD = int n/D over [zb, zmax], computed
 * once per shell (linearity of the integral). */
typedef struct { cx Ds; double zmax, zb; cx norm, In, InD; int kind; } w_ctx;
static cx f_wnum(const theta_t *th, double z, const void *ctx) {
  const w_ctx *w = (const w_ctx *)ctx;
  cx D = D_of(th, z);
  cx lens;
  if (w->kind == 0) {
    lens = D * (w->Ds - D) / w->Ds;
  } else {
    q_ctx q = { z, D };
    double zt = w->zb < w->zmax ? w->zb : w->zmax;
    cx avg = integrate(f_q, th, &q, z, zt) + w->In - D * w->InD;
    lens = D * avg / w->norm;
  }
  return inv_E(th, z) * lens * (1.0 + z);
}

static void weights(const theta_t *th, const double *z_edges, int32_t nshell,
                    const or_source *src, cx *w_out) {
  w_ctx w;
  w.kind = src->kind;
  double zcut = (src->kind == 0) ? src->z_s : src->z_max;
  w.zmax = src->z_max;
  w.Ds = (src->kind == 0) ? D_of(th, src->z_s) : 0.0;
  w.norm = (src->kind == 0) ? 1.0 : nz_norm(th, src->z_max);
  for (int b = 0; b < nshell; ++b) {
    double za = z_edges[b], zb = z_edges[b + 1];
    double zt = zb < zcut ? zb : zcut;
    w.zb = zb;
    w.In = 0.0;
    w.InD = 0.0;
    if (src->kind == 1 && zb < src->z_max) {
      w.In = integrate(f_nz, th, NULL, zb, src->z_max);
      w.InD = integrate(f_n_over_D, th, NULL, zb, src->z_max);
    }
    cx num = integrate(f_wnum, th, &w, za, zt);
    cx den = integrate(f_invE, th, NULL, za, zb);
    w_out[b] = num / den;
  }
}

/* Density factor of Eq. 6 and 7: the expected count of a pixel on shell b
 * is rho/m_p times the pixel's share of the shell volume.  Reading 0 (the
 * printed Eq. 6): F_b = N_pix V / (4 pi N chi_b^2), chi_b the lower edge.
 * Reading 1: the mean of 1/chi^2 over the shell volume, so that F_b times
 * the expected count of a uniform field is exactly Delta chi_b:
 * F_b = 3 N_pix V Delta chi_b / (4 pi N (chi_{b+1}^3 - chi_b^3)). */
static cx density_factor(double npix, double V, int64_t n_total, cx lo, cx hi, int volume) {
  const double pi = 3.14159265358979323846264338327950288;
  if (volume) return 3.0 * npix * V * (hi - lo) / (4.0 * pi * (double)n_total * (hi * hi * hi - lo * lo * lo));
  return npix * V / (4.0 * pi * (double)n_total * lo * lo);
}

static void coeffs(const theta_t *th, const or_box *boxes, int32_t nbox,
                   const double *z_edges, int32_t nshell, int64_t nside,
                   const or_source *src, cx *A, cx *B, cx *C) {
  const double pi = 3.14159265358979323846264338327950288;
  cx *w = (cx *)malloc(sizeof(cx) * nshell);
  cx *chi = (cx *)malloc(sizeof(cx) * (nshell + 1));
  weights(th, z_edges, nshell, src, w);
  cx cH = c_over_H0(th);
  for (int b = 0; b <= nshell; ++b) chi[b] = cH * D_of(th, z_edges[b]);
  double npix = (double)or_nside2npix(nside);
  *C = 0.0;
  for (int b = 0; b < nshell; ++b) {
    const or_box *bx = NULL;
    for (int k = 0; k < nbox; ++k)
      if (b >= boxes[k].shell_lo && b < boxes[k].shell_hi) bx = &boxes[k];
    if (!bx) { A[b] = NAN; B[b] = NAN; continue; }
    double V = bx->L * bx->L * bx->L;
    cx F = density_factor(npix, V, bx->n_total, chi[b], chi[b + 1], th->dens_volume);
    A[b] = 1.5 * th->om * w[b] * F / cH;
    B[b] = 1.5 * th->om * w[b] * (chi[b + 1] - chi[b]) / cH;
    *C += B[b];
  }
  free(w);
  free(chi);
}

static theta_t make_theta(double om, double h, int units, const or_source *src) {
  theta_t th;
  th.om = om; th.h = h; th.units_mpc_over_h = units; th.dens_volume = 0;
  th.alpha = src ? src->alpha : 0.0;
  th.beta = src ? src->beta : 1.0;
  th.z0 = src ? src->z0 : 1.0;
  return th;
}

/* ---- public real-valued entry points ------------------------------------ */
double or_comoving_distance(double om, double h, int units, double z) {
  theta_t th = make_theta(om, h, units, NULL);
  return creal(c_over_H0(&th) * D_of(&th, z));
}

void or_chi_edges(double om, double h, int units, const double *z_edges,
                  int32_t nshell, double *chi_out) {
  for (int b = 0; b <= nshell; ++b) chi_out[b] = or_comoving_distance(om, h, units, z_edges[b]);
}

/* Inverse of chi(z) by bisection on [0, 64]. */
double or_z_of_chi(double om, double h, int units, double chi) {
  double lo = 0.0, hi = 64.0;
  for (int it = 0; it < 200; ++it) {
    double mid = 0.5 * (lo + hi);
    if (mid == lo || mid == hi) break;
    if (or_comoving_distance(om, h, units, mid) < chi) lo = mid; else hi = mid;
  }
  return 0.5 * (lo + hi);
}

void or_shell_weights(double om, const double *z_edges, int32_t nshell,
                      const or_source *src, double *w_out) {
  theta_t th = make_theta(om, 0.7, 1, src);
  cx *w = (cx *)malloc(sizeof(cx) * nshell);
  weights(&th, z_edges, nshell, src, w);
  for (int b = 0; b < nshell; ++b) w_out[b] = creal(w[b]);
  free(w);
}

void or_kappa_coeffs(double om, double h, int units, int dens_volume, const or_box *boxes,
                     int32_t nbox, const double *z_edges, int32_t nshell,
                     int64_t nside, const or_source *src, double *A_out,
                     double *B_out, double *C_out) {
  theta_t th = make_theta(om, h, units, src);
  th.dens_volume = dens_volume;
  cx *A = (cx *)malloc(sizeof(cx) * nshell), *B = (cx *)malloc(sizeof(cx) * nshell), C;
  coeffs(&th, boxes, nbox, z_edges, nshell, nside, src, A, B, &C);
  for (int b = 0; b < nshell; ++b) { A_out[b] = creal(A[b]); B_out[b] = creal(B[b]); }
  *C_out = creal(C);
  free(A); free(B);
}

/* Overdensity map, Eq. 7: delta_p = sum_b [F_b n_bp - dchi_b] / sum_b dchi_b,
 * returned as delta_p = sum_b A_b n_bp - C: A_b = F_b / sum_b dchi_b and
 * C = (sum_b dchi_b) / (sum_b dchi_b) = 1.  F_b is the density factor of
 * Eq. 6 (density_factor), with V, N of the box owning shell b;
 * dchi_b = chi_{b+1} - chi_b. */
void or_delta_coeffs(double om, double h, int units, int dens_volume, const or_box *boxes,
                     int32_t nbox, const double *z_edges, int32_t nshell,
                     int64_t nside, double *A_out, double *C_out) {
  double *chi = (double *)malloc(sizeof(double) * (nshell + 1));
  for (int b = 0; b <= nshell; ++b) chi[b] = or_comoving_distance(om, h, units, z_edges[b]);
  double total = 0.0;
  for (int b = 0; b < nshell; ++b) total += chi[b + 1] - chi[b];
  const double npix = (double)or_nside2npix(nside);
  for (int b = 0; b < nshell; ++b) {
    const or_box *bx = NULL;
    for (int k = 0; k < nbox; ++k)
      if (b >= boxes[k].shell_lo && b < boxes[k].shell_hi) bx = &boxes[k];
    if (!bx) { A_out[b] = NAN; continue; }
    const double V = bx->L * bx->L * bx->L;
    const double F = creal(density_factor(npix, V, bx->n_total, chi[b], chi[b + 1], dens_volume));
    A_out[b] = F / total;
  }
  *C_out = total / total;
  free(chi);
}

/* ---- statistics of the unrounded map, for gradients ---------------------- */
/* Pairwise sum, so that the relative error stays near log2(n) ulp. */
static cx psum(const cx *v, int64_t n) {
  if (n <= 8) { cx s = 0.0; for (int64_t i = 0; i < n; ++i) s += v[i]; return s; }
  int64_t h = n / 2;
  return psum(v, h) + psum(v + h, n - h);
}

/* var = mu2, skew = mu3/mu2^(3/2), and <g, kappa> = sum_p g_p kappa_p of
 * kappa_p = sum_b A_b n_bp - C evaluated at theta, all in complex FP64. */
static void stats_at(const theta_t *th, const int32_t *counts, int32_t nshell,
                     int64_t nside, const or_box *boxes, int32_t nbox,
                     const double *z_edges, const or_source *src,
                     const float *g, cx *out) {
  int64_t npix = or_nside2npix(nside);
  cx *A = (cx *)malloc(sizeof(cx) * nshell), *B = (cx *)malloc(sizeof(cx) * nshell), C;
  coeffs(th, boxes, nbox, z_edges, nshell, nside, src, A, B, &C);
  cx *k = (cx *)malloc(sizeof(cx) * npix), *tmp = (cx *)malloc(sizeof(cx) * npix);
  for (int64_t p = 0; p < npix; ++p) {
    cx s = 0.0;
    for (int b = 0; b < nshell; ++b) s += A[b] * (double)counts[(int64_t)b * npix + p];
    k[p] = s - C;
  }
  cx mean = psum(k, npix) / (double)npix;
  for (int64_t p = 0; p < npix; ++p) { cx d = k[p] - mean; tmp[p] = d * d; }
  cx mu2 = psum(tmp, npix) / (double)npix;
  for (int64_t p = 0; p < npix; ++p) { cx d = k[p] - mean; tmp[p] = d * d * d; }
  cx mu3 = psum(tmp, npix) / (double)npix;
  out[0] = mu2;
  out[1] = mu3 / cpow(mu2, 1.5);
  if (g) {
    for (int64_t p = 0; p < npix; ++p) tmp[p] = (double)g[p] * k[p];
    out[2] = psum(tmp, npix);
  } else {
    out[2] = 0.0;
  }
  free(A); free(B); free(k); free(tmp);
}

void or_kappa_stats_f64(const int32_t *counts, int32_t nshell, int64_t nside,
                        double om, double h, int units, const or_box *boxes,
                        int32_t nbox, const double *z_edges,
                        const or_source *src, const float *g, double *out) {
  theta_t th = make_theta(om, h, units, src);
  cx o[3];
  stats_at(&th, counts, nshell, nside, boxes, nbox, z_edges, src, g, o);
  for (int i = 0; i < 3; ++i) out[i] = creal(o[i]);
}

void or_kappa_stat_grads(const int32_t *counts, int32_t nshell, int64_t nside,
                         double om, double h, int units, const or_box *boxes,
                         int32_t nbox, const double *z_edges,
                         const or_source *src, const float *g, double *grad_out) {
  const double eps = 1e-30;
  for (int j = 0; j < 5; ++j) {
    theta_t th = make_theta(om, h, units, src);
    cx step = eps * I;
    if (j == 0) th.om += step;
    if (j == 1) th.h += step;
    if (j == 2) th.alpha += step;
    if (j == 3) th.beta += step;
    if (j == 4) th.z0 += step;
    cx o[3];
    stats_at(&th, counts, nshell, nside, boxes, nbox, z_edges, src, g, o);
    for (int s = 0; s < 3; ++s) grad_out[s * 5 + j] = cimag(o[s]) / eps;
  }
}
