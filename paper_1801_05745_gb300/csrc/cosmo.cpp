// Host cosmology of the library: comoving distances, shell weights and the
// kappa coefficients of Eq. 6, with their derivatives with respect to
// theta = (Omega_m, h, alpha, beta, z0) by forward-mode dual numbers.
//
// Readings of the paper (Sec. 2.3-2.4): flat LambdaCDM
// E(z) = sqrt(Omega_m (1+z)^3 + 1 - Omega_m); D(z) = int_0^z dz'/E;
// chi = (c/H0) D with c/H0 = 2997.92458 Mpc/h (or /h Mpc); Eq. 3 with
// D(z, z_s) = D(z_s) - D(z), 1/a = 1 + z and zero integrand beyond z_s; for
// an n(z) source the ratio D(z, z_s)/D(z_s) of Eq. 3 is averaged over
// n(z_s) = z_s^alpha exp(-(z_s/z0)^beta) normalised on [0, z_max]; Eq. 6
// uses chi of the shell's lower edge and (V, N) of the box owning the shell.
//
// Quadrature: composite 20-point Gauss-Legendre on panels of width <= 1/8
// (nodes from Newton's method on the Legendre recurrence), geometric panels
// towards z = 0 for the n(z) normalisation.
#include <array>
#include <cmath>
#include <vector>

#include "../../include/ufalcon.h"

namespace ufc {

constexpr int kNP = 5;   // parameters: Omega_m, h, alpha, beta, z0

struct Dual {
  double v = 0.0;
  std::array<double, kNP> d{};
  Dual() = default;
  Dual(double x) : v(x) {}
  static Dual var(double x, int i) { Dual r(x); r.d[i] = 1.0; return r; }
};
inline Dual operator+(const Dual& a, const Dual& b) { Dual r(a.v + b.v); for (int i = 0; i < kNP; ++i) r.d[i] = a.d[i] + b.d[i]; return r; }
inline Dual operator-(const Dual& a, const Dual& b) { Dual r(a.v - b.v); for (int i = 0; i < kNP; ++i) r.d[i] = a.d[i] - b.d[i]; return r; }
inline Dual operator-(const Dual& a) { Dual r(-a.v); for (int i = 0; i < kNP; ++i) r.d[i] = -a.d[i]; return r; }
inline Dual operator*(const Dual& a, const Dual& b) { Dual r(a.v * b.v); for (int i = 0; i < kNP; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i]; return r; }
inline Dual operator/(const Dual& a, const Dual& b) { Dual r(a.v / b.v); for (int i = 0; i < kNP; ++i) r.d[i] = (a.d[i] * b.v - a.v * b.d[i]) / (b.v * b.v); return r; }
inline Dual& operator+=(Dual& a, const Dual& b) { a = a + b; return a; }
inline Dual sqrt(const Dual& a) { double s = std::sqrt(a.v); Dual r(s); for (int i = 0; i < kNP; ++i) r.d[i] = a.d[i] / (2.0 * s); return r; }
inline Dual exp(const Dual& a) { double e = std::exp(a.v); Dual r(e); for (int i = 0; i < kNP; ++i) r.d[i] = a.d[i] * e; return r; }
inline Dual log(const Dual& a) { Dual r(std::log(a.v)); for (int i = 0; i < kNP; ++i) r.d[i] = a.d[i] / a.v; return r; }
// x^p for x > 0 (real) and dual exponent
inline Dual powr(double x, const Dual& p) { return exp(p * Dual(std::log(x))); }
inline Dual powd(const Dual& x, const Dual& p) { return exp(p * log(x)); }

// ---- Gauss-Legendre nodes -------------------------------------------------
constexpr int kGL = 20;
struct GL {
  double x[kGL], w[kGL];
  GL() {
    const double pi = 3.14159265358979323846;
    for (int i = 0; i < kGL; ++i) {
      double z = std::cos(pi * (i + 0.75) / (kGL + 0.5));
      for (int it = 0; it < 100; ++it) {
        double p0 = 1.0, p1 = z;
        for (int k = 2; k <= kGL; ++k) {
          double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
          p0 = p1;
          p1 = p2;
        }
        double dp = kGL * (z * p1 - p0) / (z * z - 1.0);
        double dz = p1 / dp;
        z -= dz;
        if (std::fabs(dz) < 1e-16) {
          // one more step with the converged value
          p0 = 1.0; p1 = z;
          for (int k = 2; k <= kGL; ++k) { double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k; p0 = p1; p1 = p2; }
          dp = kGL * (z * p1 - p0) / (z * z - 1.0);
          x[i] = z;
          w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
          break;
        }
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
      }
    }
  }
};
static const GL& gl() { static GL g; return g; }

template <class F>
static Dual integrate(F f, double a, double b) {
  if (!(b > a)) return Dual(0.0);
  const GL& g = gl();
  int np = (int)std::ceil((b - a) * 8.0);
  if (np < 1) np = 1;
  const double h = (b - a) / np;
  Dual tot(0.0);
  for (int p = 0; p < np; ++p) {
    const double lo = a + p * h, hi = (p == np - 1) ? b : a + (p + 1) * h;
    const double c = 0.5 * (lo + hi), r = 0.5 * (hi - lo);
    Dual s(0.0);
    for (int k = 0; k < kGL; ++k) s += Dual(g.w[k]) * f(c + r * g.x[k]);
    tot += Dual(r) * s;
  }
  return tot;
}

struct Theta {
  Dual om, h, alpha, beta, z0;
  int units;
  int vol;   // density factor over the shell volume (ufc_cosmo.density_volume)
};

static Dual invE(const Theta& t, double z) {
  const double zp = 1.0 + z;
  return Dual(1.0) / sqrt(t.om * Dual(zp * zp * zp) + Dual(1.0) - t.om);
}
static Dual Dist(const Theta& t, double z) {
  return integrate([&](double x) { return invE(t, x); }, 0.0, z);
}
static Dual cH0(const Theta& t) {
  return t.units ? Dual(2997.92458) : Dual(2997.92458) / t.h;
}
static Dual nz(const Theta& t, double z) {
  if (!(z > 0.0)) return Dual(0.0);
  return exp(t.alpha * Dual(std::log(z)) - powd(Dual(z) / t.z0, t.beta));
}

static Theta theta(const ufc_cosmo& c, const ufc_source* s, bool derivs) {
  Theta t;
  t.units = c.units_mpc_over_h;
  t.vol = c.density_volume;
  t.om = derivs ? Dual::var(c.omega_m, 0) : Dual(c.omega_m);
  t.h = derivs ? Dual::var(c.h, 1) : Dual(c.h);
  const double a = s ? s->alpha : 0.0, b = s ? s->beta : 1.0, z0 = s ? s->z0 : 1.0;
  t.alpha = derivs ? Dual::var(a, 2) : Dual(a);
  t.beta = derivs ? Dual::var(b, 3) : Dual(b);
  t.z0 = derivs ? Dual::var(z0, 4) : Dual(z0);
  return t;
}

// Density factor of Eq. 6 and 7 with k = N_pix V / (4 pi N): k / chi_lo^2
// (lower edge, as printed), or its mean over the shell volume,
// 3 k (chi_hi - chi_lo) / (chi_hi^3 - chi_lo^3).
static Dual density_factor(double k, const Dual& lo, const Dual& hi, int volume) {
  if (volume) return Dual(3.0 * k) * (hi - lo) / (hi * hi * hi - lo * lo * lo);
  return Dual(k) / (lo * lo);
}

// Shell weights W_b (Eq. 3 or its n(z) average).
static void weights(const Theta& t, const double* z, int S, const ufc_source& src,
                    std::vector<Dual>& W) {
  W.assign(S, Dual(0.0));
  const bool plane = src.kind == 0;
  const double zcut = plane ? src.z_s : src.z_max;
  Dual Ds = plane ? Dist(t, src.z_s) : Dual(0.0);
  Dual norm(1.0);
  if (!plane) {
    // geometric panels [zmax 2^-(k+1), zmax 2^-k]
    norm = Dual(0.0);
    for (int k = 0; k < 60; ++k)
      norm += integrate([&](double x) { return nz(t, x); }, src.z_max * std::ldexp(1.0, -(k + 1)),
                        src.z_max * std::ldexp(1.0, -k));
  }
  for (int b = 0; b < S; ++b) {
    const double za = z[b], zb = z[b + 1];
    const double zt = std::min(zb, zcut);
    const Dual Da = Dist(t, za);
    // D(z) inside the shell as D(z_a) + int_{z_a}^{z} dz'/E
    auto Din = [&](double x) {
      return Da + integrate([&](double y) { return invE(t, y); }, za, x);
    };
    Dual In(0.0), InD(0.0);
    if (!plane && zb < src.z_max) {
      In = integrate([&](double x) { return nz(t, x); }, zb, src.z_max);
      InD = integrate([&](double x) { return nz(t, x) / Dist(t, x); }, zb, src.z_max);
    }
    Dual num = integrate(
        [&](double x) {
          Dual D = Din(x);
          Dual lens;
          if (plane) {
            lens = D * (Ds - D) / Ds;
          } else {
            // average of (D(z') - D(z))/D(z') over z' in [z, z_max]
            Dual part = integrate(
                [&](double y) {
                  Dual Dy = Din(y);
                  return nz(t, y) * (Dy - D) / Dy;
                },
                x, std::min(zb, src.z_max));
            lens = D * (part + In - D * InD) / norm;
          }
          return invE(t, x) * lens * Dual(1.0 + x);
        },
        za, zt);
    Dual den = integrate([&](double x) { return invE(t, x); }, za, zb);
    W[b] = num / den;
  }
}

// ---- exported helpers (called from capi.cu) ----------------------------
ufc_status cosmo_chi_edges(const ufc_cosmo& c, const double* z, int n, double* chi) {
  Theta t = theta(c, nullptr, false);
  const Dual ch = cH0(t);
  for (int i = 0; i < n; ++i) chi[i] = (ch * Dist(t, z[i])).v;
  return UFC_OK;
}

ufc_status cosmo_z_of_chi(const ufc_cosmo& c, const double* chi, int n, double* zout) {
  Theta t = theta(c, nullptr, false);
  const double ch = cH0(t).v;
  for (int i = 0; i < n; ++i) {
    // Newton on chi(z) - chi = 0, chi'(z) = (c/H0)/E(z), started from the
    // low-redshift value and bracketed by bisection steps when it strays
    double lo = 0.0, hi = 64.0, z = chi[i] / ch;
    for (int it = 0; it < 100; ++it) {
      const double f = ch * Dist(t, z).v - chi[i];
      if (f < 0) lo = z; else hi = z;
      const double step = f / (ch * invE(t, z).v);
      double zn = z - step;
      if (!(zn > lo && zn < hi)) zn = 0.5 * (lo + hi);
      if (std::fabs(zn - z) <= 1e-16 * std::max(1.0, z)) { z = zn; break; }
      z = zn;
    }
    zout[i] = z;
  }
  return UFC_OK;
}

ufc_status cosmo_kappa_coeffs(const ufc_cosmo& c, const ufc_box* boxes, int nbox,
                              const double* z, int S, int nside, const ufc_source& src,
                              double* A, double* B, double* C, double* dA, double* dC) {
  const bool derivs = dA || dC;
  Theta t = theta(c, &src, derivs);
  std::vector<Dual> W;
  weights(t, z, S, src, W);
  const Dual ch = cH0(t);
  std::vector<Dual> chi(S + 1);
  for (int b = 0; b <= S; ++b) chi[b] = ch * Dist(t, z[b]);
  const double pi = 3.14159265358979323846;
  const double npix = 12.0 * nside * nside;
  Dual Ct(0.0);
  for (int b = 0; b < S; ++b) {
    const ufc_box* bx = nullptr;
    for (int k = 0; k < nbox; ++k)
      if (b >= boxes[k].shell_lo && b < boxes[k].shell_hi) bx = &boxes[k];
    const double V = bx->L * bx->L * bx->L;
    const Dual F = density_factor(npix * V / (4.0 * pi * (double)bx->n_total), chi[b], chi[b + 1],
                                  t.vol);
    Dual Ab = Dual(1.5) * t.om * W[b] * F / ch;
    Dual Bb = Dual(1.5) * t.om * W[b] * (chi[b + 1] - chi[b]) / ch;
    A[b] = Ab.v;
    if (B) B[b] = Bb.v;
    if (dA)
      for (int j = 0; j < kNP; ++j) dA[j * S + b] = Ab.d[j];
    Ct += Bb;
  }
  *C = Ct.v;
  if (dC)
    for (int j = 0; j < kNP; ++j) dC[j] = Ct.d[j];
  return UFC_OK;
}

// Overdensity map, Eq. 7: delta_p = sum_b [F_b n_bp - Delta chi_b] / sum_b Delta chi_b
// = sum_b A_b n_bp - C with A_b = F_b / sum_b Delta chi_b and C = 1; F_b is
// the density factor of Eq. 6 (N_pix V_k / (4 pi N_k chi_b^2), chi_b the
// shell's lower edge).  Derivatives with respect to theta as for kappa
// (only Omega_m and, in Mpc units, h enter, through chi).
ufc_status cosmo_delta_coeffs(const ufc_cosmo& c, const ufc_box* boxes, int nbox,
                              const double* z, int S, int nside, double* A, double* C,
                              double* dA, double* dC) {
  const bool derivs = dA || dC;
  Theta t = theta(c, nullptr, derivs);
  const Dual ch = cH0(t);
  std::vector<Dual> chi(S + 1);
  for (int b = 0; b <= S; ++b) chi[b] = ch * Dist(t, z[b]);
  Dual thick(0.0);
  for (int b = 0; b < S; ++b) thick += chi[b + 1] - chi[b];
  const double pi = 3.14159265358979323846;
  const double npix = 12.0 * nside * nside;
  for (int b = 0; b < S; ++b) {
    const ufc_box* bx = nullptr;
    for (int k = 0; k < nbox; ++k)
      if (b >= boxes[k].shell_lo && b < boxes[k].shell_hi) bx = &boxes[k];
    const double V = bx->L * bx->L * bx->L;
    const Dual Ab = density_factor(npix * V / (4.0 * pi * (double)bx->n_total), chi[b],
                                   chi[b + 1], t.vol) / thick;
    A[b] = Ab.v;
    if (dA)
      for (int j = 0; j < kNP; ++j) dA[j * S + b] = Ab.d[j];
  }
  *C = 1.0;
  if (dC)
    for (int j = 0; j < kNP; ++j) dC[j] = 0.0;
  return UFC_OK;
}

}  // namespace ufc
